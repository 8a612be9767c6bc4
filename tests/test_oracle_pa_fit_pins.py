"""Pins for the synthetic power amplifier (Saleh AM/AM and AM/PM, then the
memory FIR) and for the oracle's Adam update, at amplitudes and step counts
where every term matters.

The amplifier pins use identities the model implies rather than its formula:
the AM/AM curve takes equal values at r and 1/(beta_a r); the AM/PM phases at r
and 1/(beta_p r) add up to the saturation phase alpha_p / beta_p; the phase is
added (v / x turns counter-clockwise) and is a function of the input
amplitude; the memory taps act after the nonlinearity, which numpy.convolve
of the memoryless output checks.  The Adam pins compare the oracle with a
scalar recurrence expanded by hand on a one-tap problem and with
torch.optim.Adam (float64, real and imaginary parts as separate parameters,
gradients from torch autograd) on a two-branch problem.
"""
import numpy as np
import pytest

from oracle import fit as OF
from oracle import pa as PA

SALEH = (2.1587, 1.1517, 4.0033, 9.1040)


def _single(r, theta=0.7):
    """Output sample of a single input sample r e^{j theta} with no memory."""
    x = np.array([r * np.exp(1j * theta)])
    return PA.pa(x, SALEH, (1.0,))[0], x[0]


@pytest.mark.parametrize("r", [0.5, 1 / np.sqrt(SALEH[1]), 2.0, 0.05, 3.7])
def test_am_am_symmetry_under_r_to_one_over_beta_r(r):
    """A(r) = A(1/(beta_a r)): the AM/AM curve of the Saleh model is symmetric
    about its peak on a logarithmic amplitude axis."""
    ba = SALEH[1]
    v1, _ = _single(r)
    v2, _ = _single(1.0 / (ba * r))
    assert abs(abs(v1) - abs(v2)) < 1e-13 * max(1.0, abs(v1))


@pytest.mark.parametrize("r", [0.5, 1 / np.sqrt(SALEH[3]), 2.0, 0.1])
def test_am_pm_phases_add_to_saturation_phase(r):
    """Phi(r) + Phi(1/(beta_p r)) = alpha_p / beta_p, the phase shift the
    amplifier approaches in saturation; the shift is added to the input phase
    (a flipped sign gives -alpha_p / beta_p)."""
    ap, bp = SALEH[2], SALEH[3]
    v1, x1 = _single(r, 0.3)
    v2, x2 = _single(1.0 / (bp * r), -1.1)
    d = np.angle(v1 / x1) + np.angle(v2 / x2)
    assert abs(d - ap / bp) < 1e-12
    # at r = 1/sqrt(beta_p) the shift is half the saturation phase
    v, x = _single(1 / np.sqrt(bp), 2.0)
    assert abs(np.angle(v / x) - ap / (2 * bp)) < 1e-12


def test_am_pm_saturates_and_vanishes():
    """Large inputs approach the saturation phase, small ones no phase shift."""
    ap, bp = SALEH[2], SALEH[3]
    v, x = _single(1e4)
    assert abs(np.angle(v / x) - ap / bp) < 1e-7
    v, x = _single(1e-5)
    assert abs(np.angle(v / x)) < 1e-8


def test_memory_taps_follow_the_nonlinearity():
    """y = numpy.convolve(memoryless PA output, taps), truncated; a single impulse
    of non-small amplitude gives the taps times the compressed, rotated sample."""
    rng = np.random.default_rng(5)
    x = (rng.normal(0, 0.6, 64) + 1j * rng.normal(0, 0.6, 64))
    mem = (1.0, 0.1, -0.05)
    v = PA.pa(x, SALEH, (1.0,))
    y = PA.pa(x, SALEH, mem)
    np.testing.assert_allclose(y, np.convolve(v, mem)[:len(x)], rtol=0, atol=1e-14)
    imp = np.zeros(5, complex)
    imp[0] = 1.3 * np.exp(0.4j)
    yi = PA.pa(imp, SALEH, mem)
    v0, _ = _single(1.3, 0.4)
    np.testing.assert_allclose(yi[:3], v0 * np.array(mem), rtol=1e-14, atol=0)
    assert np.all(yi[3:] == 0)


def test_adam_one_tap_hand_expanded():
    """One branch of order 1, one tap: P(u) = h u, loss mean |h u - t|^2, whose
    gradients are dL/dRe h = 2/N sum Re(conj(u) (h u - t)) and
    dL/dIm h = 2/N sum Im(conj(u) (h u - t)).  Each part follows its own scalar
    Adam; three steps at a large learning rate, so that the bias correction and
    the placement of eps both show."""
    rng = np.random.default_rng(1)
    N = 16
    u = rng.normal(size=N) + 1j * rng.normal(size=N)
    t = (0.8 - 0.3j) * u + 0.01 * (rng.normal(size=N) + 1j * rng.normal(size=N))
    h0 = 1.0 + 0.0j
    lr = 0.05
    for steps in (1, 2, 3):
        h, losses = OF.adam_fit(u, t, np.array([[h0]]), (1,), steps, lr)
        # the two real parameters interact only through the residual; iterate them jointly
        hr, hi = h0.real, h0.imag
        m = np.zeros(2)
        v = np.zeros(2)
        for s in range(1, steps + 1):
            r = (hr + 1j * hi) * u - t
            g = np.array([2 / N * np.sum((np.conj(u) * r).real), 2 / N * np.sum((np.conj(u) * r).imag)])
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            step = lr * (m / (1 - 0.9 ** s)) / (np.sqrt(v / (1 - 0.999 ** s)) + 1e-8)
            hr, hi = hr - step[0], hi - step[1]
        assert abs(h[0, 0] - (hr + 1j * hi)) < 1e-13
        r0 = h0 * u - t
        assert abs(losses[0] - np.mean(np.abs(r0) ** 2)) < 1e-13
    # the first Adam step moves each part by lr (sign of its gradient), whatever its size
    h1, _ = OF.adam_fit(u, t, np.array([[h0]]), (1,), 1, lr)
    r0 = h0 * u - t
    gr = np.sum(np.conj(u) * r0)
    assert abs(abs(h1[0, 0].real - h0.real) - lr) < 1e-9
    assert abs(abs(h1[0, 0].imag - h0.imag) - lr) < 1e-9
    assert np.sign(h0.real - h1[0, 0].real) == np.sign(gr.real)
    assert np.sign(h0.imag - h1[0, 0].imag) == np.sign(gr.imag)


def test_adam_matches_torch_optim_two_branches():
    """Two branches (orders 1 and 3) of three taps: the oracle's Adam equals
    torch.optim.Adam in float64 over five steps, with the forward written as
    torch ops and the gradient from autograd (real and imaginary parts of the
    taps as one real (K, M, 2) parameter)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    N, K, M = 40, 2, 3
    orders = (1, 3)
    u = 0.5 * (rng.normal(size=N) + 1j * rng.normal(size=N))
    t = u + 0.2 * u * np.abs(u) ** 2 + 0.05 * (rng.normal(size=N) + 1j * rng.normal(size=N))
    h0 = np.zeros((K, M), complex)
    h0[0, 0] = 1.0
    h0[1, 1] = 0.1 - 0.05j
    steps, lr = 5, 0.02
    h_or, loss_or = OF.adam_fit(u, t, h0, orders, steps, lr)

    ut = torch.tensor(u, dtype=torch.complex128)
    tt = torch.tensor(t, dtype=torch.complex128)
    p = torch.tensor(np.stack([h0.real, h0.imag], -1), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        h = torch.complex(p[..., 0], p[..., 1])
        y = torch.zeros(N, dtype=torch.complex128)
        for k in range(K):
            z = ut * (ut.abs() ** (orders[k] - 1))
            for m in range(M):
                y = y + h[k, m] * torch.cat([torch.zeros(m, dtype=torch.complex128), z[:N - m]])
        loss = ((y - tt).abs() ** 2).mean()
        losses.append(loss.item())
        loss.backward()
        opt.step()
    h_t = (p[..., 0] + 1j * p[..., 1]).detach().numpy()
    np.testing.assert_allclose(h_or, h_t, rtol=0, atol=1e-12)
    np.testing.assert_allclose(loss_or, losses, rtol=1e-12, atol=0)
