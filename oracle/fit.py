"""Indirect-learning fit in float64 (oracle; test infrastructure).

Same procedure as the engine's fit: postdistorter P trained so that
P(y/G) ~ x (y = PA(x), G = small-signal gain), loss mean |P(y/G) - x|^2,
Adam from the identity.  Gradients come from the float64 adjoint
(dpd.dpd_stream_backward); Adam acts on the real and imaginary parts as
separate real parameters (bias-corrected first and second moments).

Pins: the update rule of :func:`adam_fit` against a hand-expanded recurrence on
a one-tap problem and against torch.optim.Adam in float64 (gradients from
torch autograd); the amplifier against the identities of the Saleh model; the
gradient against finite differences.  The paper prints no fit outcome, so the
final NMSE itself has no value to be compared with; the tests compare the
engine's loss curve with this one.
"""
from __future__ import annotations

import numpy as np

from . import dpd as D
from . import pa as PA


def adam_fit(u, target, h0, orders, steps, lr, betas=(0.9, 0.999), eps=1e-8):
    """Adam on the taps of P (real and imaginary parts as separate parameters) so that
    P(u) ~ target; loss mean |P(u) - target|^2.  Returns (h, losses)."""
    h = np.array(h0, np.complex128)
    m = np.zeros(h.shape + (2,))
    v = np.zeros(h.shape + (2,))
    losses = []
    N = len(u)
    for t in range(1, steps + 1):
        out = D.dpd_stream(u, h, orders)
        r = out - target
        losses.append(float(np.mean(r.real ** 2 + r.imag ** 2)))
        g = 2.0 * r / N                          # dL/dRe(out) + i dL/dIm(out)
        _, gh = D.dpd_stream_backward(u, h, orders, g)
        gr = np.stack([gh.real, gh.imag], axis=-1)
        m = betas[0] * m + (1 - betas[0]) * gr
        v = betas[1] * v + (1 - betas[1]) * gr * gr
        mh = m / (1 - betas[0] ** t)
        vh = v / (1 - betas[1] ** t)
        step = lr * mh / (np.sqrt(vh) + eps)
        h = h - (step[..., 0] + 1j * step[..., 1])
    return h, np.array(losses)


def ila_fit(x, orders=(1, 3, 5, 7), M=10, steps=200, lr=1e-3, betas=(0.9, 0.999), eps=1e-8,
            saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05)):
    x = np.asarray(x, np.complex128)
    K = len(orders)
    G = PA.small_signal_gain(saleh, memory)
    u = PA.pa(x, saleh, memory) / G
    h = np.zeros((K, M), np.complex128)
    h[0, 0] = 1
    return adam_fit(u, x, h, orders, steps, lr, betas, eps)


def ila_fit_iterative(x, iterations=3, orders=(1, 3, 5, 7), M=10, steps=200, lr=1e-3,
                      saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05)):
    """Iterative indirect learning: in iteration i the current predistorter P_i drives
    the amplifier with z = P_i(x); a postdistorter, started from P_i's taps, is
    trained so that P(PA(z)/G) ~ z and becomes P_{i+1}.  P_0 is the identity.
    Returns (h, loss curves per iteration, NMSE in dB of PA(P_{i+1}(x))/G against x
    after each iteration)."""
    x = np.asarray(x, np.complex128)
    K = len(orders)
    G = PA.small_signal_gain(saleh, memory)
    h = np.zeros((K, M), np.complex128)
    h[0, 0] = 1
    curves, nmse = [], []
    for _ in range(iterations):
        z = D.dpd_stream(x, h, orders)
        u = PA.pa(z, saleh, memory) / G
        h, losses = adam_fit(u, z, h, orders, steps, lr)
        curves.append(losses)
        e = PA.pa(D.dpd_stream(x, h, orders), saleh, memory) / G - x
        nmse.append(float(10 * np.log10(np.sum(np.abs(e) ** 2) / np.sum(np.abs(x) ** 2))))
    return h, curves, np.array(nmse)
