"""Dynamic predistortion arithmetic in float64 (oracle; test infrastructure).

Sec. 4.2 describes the predistorter as parallel FIR filters fed by a Poly
actor and summed by an Adder actor; the control actor picks, per block, which
branches are active.  The paper does not print the branch nonlinearity; the
reading adopted here is the memory-polynomial branch

    z_k[n] = |x[n]|^(o_k - 1) * x[n],      o_k odd,

followed by an M-tap complex FIR per branch, y_k[n] = sum_m h[k,m] z_k[n-m],
and out[n] = sum over active k (ascending) of y_k[n].

All arithmetic is complex128; complex64 inputs are promoted exactly.
"""
from __future__ import annotations

import numpy as np


def psi(x: np.ndarray, order: int) -> np.ndarray:
    """Branch nonlinearity |x|^(order-1) x, with u = |x|^2 raised by repeated products."""
    if order < 1 or order % 2 == 0:
        raise ValueError("branch order must be odd and >= 1")
    x = np.asarray(x, np.complex128)
    u = x.real * x.real + x.imag * x.imag
    p = np.ones_like(u)
    for _ in range((order - 1) // 2):
        p = p * u
    return p * x


def fir(h: np.ndarray, hist: np.ndarray, z: np.ndarray):
    """M-tap FIR over a stream, continuing from ``hist`` (the previous M-1 inputs).

    Returns (y, new_hist) with y[n] = sum_{m<M} h[m] * s[n-m] where s is the
    stream ``hist`` followed by ``z``.  Written as one shifted product per tap.
    """
    h = np.asarray(h, np.complex128)
    M = len(h)
    s = np.concatenate([np.asarray(hist, np.complex128), np.asarray(z, np.complex128)])
    L = len(z)
    y = np.zeros(L, np.complex128)
    for m in range(M):
        y += h[m] * s[M - 1 - m: M - 1 - m + L]
    return y, s[len(s) - (M - 1):].copy() if M > 1 else np.zeros(0, np.complex128)


def active_branches(mask: int, K: int):
    return [k for k in range(K) if (int(mask) >> k) & 1]


def dpd_stream(x: np.ndarray, h: np.ndarray, orders) -> np.ndarray:
    """All branches active on one contiguous signal, zero history (stateless form)."""
    x = np.asarray(x, np.complex128)
    K, M = h.shape
    y = np.zeros(len(x), np.complex128)
    for k in range(K):
        yk, _ = fir(h[k], np.zeros(M - 1, np.complex128), psi(x, orders[k]))
        y += yk
    return y


def dpd_stream_backward(x: np.ndarray, h: np.ndarray, orders, g: np.ndarray):
    """Adjoint of :func:`dpd_stream` for a real loss L.

    ``g`` is dL/dRe(y) + i dL/dIm(y) (PyTorch's convention for complex
    tensors).  Returns (grad_x, grad_h) in the same convention:

    * y_k = FIR(h_k, z_k) is linear in h_k:  grad_h[k,m] = sum_n g[n] conj(z_k[n-m]).
    * grad wrt z_k:  gz_k[j] = sum_m conj(h[k,m]) g[j+m]   (j+m within the signal).
    * z = u^q x with u = |x|^2, q = (o-1)/2 gives dz = (q+1) u^q dx + q u^(q-1) x^2 conj(dx),
      so grad_x += (q+1) u^q gz_k + q u^(q-1) x^2 conj(gz_k).
    """
    x = np.asarray(x, np.complex128)
    g = np.asarray(g, np.complex128)
    K, M = h.shape
    N = len(x)
    u = x.real * x.real + x.imag * x.imag
    grad_h = np.zeros((K, M), np.complex128)
    grad_x = np.zeros(N, np.complex128)
    for k in range(K):
        q = (orders[k] - 1) // 2
        z = psi(x, orders[k])
        for m in range(M):
            grad_h[k, m] = np.sum(g[m:] * np.conj(z[:N - m]))
        gz = np.zeros(N, np.complex128)
        for m in range(M):
            gz[:N - m] += np.conj(h[k, m]) * g[m:]
        uq = np.ones_like(u)
        for _ in range(q):
            uq = uq * u
        grad_x += (q + 1) * uq * gz
        if q > 0:
            uq1 = np.ones_like(u)
            for _ in range(q - 1):
                uq1 = uq1 * u
            grad_x += q * uq1 * x * x * np.conj(gz)
    return grad_x, grad_h


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2 (0 when both are zero)."""
    a = np.asarray(a, np.complex128)
    ref = np.asarray(ref, np.complex128)
    den = np.linalg.norm(ref)
    num = np.linalg.norm(a - ref)
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return float(num / den)
