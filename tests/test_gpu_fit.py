"""The differentiable predistorter: torch.autograd.gradcheck of DPDFunction and
the indirect-learning fit against the float64 oracle fit."""
import numpy as np
import pytest

import synth
from oracle import fit as OF
from oracle import pa as OPA

pytestmark = pytest.mark.gpu


@pytest.mark.filterwarnings("ignore:Input #")
def test_gradcheck_small():
    """The kernels are float32, so finite differences use a large step and loose tolerances."""
    import torch
    from paper_1611_03226_b300.dpd import dpd
    rng = np.random.default_rng(3)
    n, K, M = 64, 3, 5
    x = torch.tensor((rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64),
                     device="cuda", requires_grad=True)
    h = torch.tensor((rng.normal(0, .2, (K, M)) + 1j * rng.normal(0, .2, (K, M))).astype(np.complex64),
                     device="cuda", requires_grad=True)
    f = lambda a, b: dpd(a, b, (1, 3, 5))
    assert torch.autograd.gradcheck(f, (x, h), eps=2e-3, atol=2e-2, rtol=2e-2, nondet_tol=0.0)


@pytest.mark.parametrize("n,K,M,orders", [(64, 3, 5, (1, 3, 5)), (1500, 4, 10, (1, 3, 5, 7)),
                                          (300, 2, 32, (1, 9))])
def test_gradcheck_float64_default_tolerances(n, K, M, orders):
    """The same kernels instantiated in float64 (complex128 tensors) pass
    torch.autograd.gradcheck at its default step and tolerances, for the
    input and the taps, across one and several tiles (1024 samples each),
    and for the two-chunk tap path (M = 32)."""
    import torch
    from paper_1611_03226_b300.dpd import dpd
    rng = np.random.default_rng(n + K)
    x = torch.tensor(rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n), dtype=torch.complex128,
                     device="cuda", requires_grad=True)
    h = torch.tensor(rng.normal(0, .2, (K, M)) + 1j * rng.normal(0, .2, (K, M)), dtype=torch.complex128,
                     device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: dpd(a, b, orders), (x, h), nondet_tol=0.0)


def test_float64_forward_and_adjoint_match_the_oracle():
    """The float64 kernels against the float64 oracle at 1e-12."""
    import torch
    from oracle import dpd as D
    from paper_1611_03226_b300 import dpd as G
    rng = np.random.default_rng(21)
    n, K, M, orders = 5000, 4, 10, (1, 3, 5, 7)
    x = rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)
    h = rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))
    g = rng.normal(size=n) + 1j * rng.normal(size=n)
    xt, ht, gt = (torch.tensor(a, dtype=torch.complex128, device="cuda") for a in (x, h, g))
    y = G.dpd_forward(xt, ht, orders).cpu().numpy()
    assert D.rel_l2(y, D.dpd_stream(x, h, orders)) <= 1e-12
    gx, gh = G.dpd_backward(xt, ht, orders, gt)
    rx, rh = D.dpd_stream_backward(x, h, orders, g)
    assert D.rel_l2(gx.cpu().numpy(), rx) <= 1e-12
    assert D.rel_l2(gh.cpu().numpy(), rh) <= 1e-12


def test_pa_model_matches_oracle():
    import torch
    from paper_1611_03226_b300 import fit as F
    w = synth.dpd_fit(n=4096)
    y = F.saleh_pa(torch.from_numpy(w.x).cuda()).cpu().numpy()
    ref = OPA.pa(w.x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("graph", [True, False])
def test_ila_fit_tracks_float64_oracle(graph):
    """40 Adam steps on 2^14 samples, as one CUDA graph per step or eagerly: the
    engine's loss curve follows the float64 oracle's within 1e-3 relative, and
    the fit improves the PA."""
    import torch
    from paper_1611_03226_b300 import fit as F
    w = synth.dpd_fit(n=1 << 14)
    steps = 40
    h, losses = F.ila_fit(torch.from_numpy(w.x).cuda(), steps=steps, lr=1e-3, graph=graph)
    h64, losses64 = OF.ila_fit(w.x, steps=steps, lr=1e-3)
    assert losses.shape == (steps,)
    assert np.max(np.abs(losses - losses64) / losses64) < 1e-3
    assert losses[-1] < 0.9 * losses[0]
    assert np.linalg.norm(h.cpu().numpy() - h64) / np.linalg.norm(h64) < 1e-3


def test_graphed_and_eager_fits_agree():
    """The captured training step replays the eager one: same loss curve and taps
    up to float32 rounding of the update (the capturable Adam keeps its step
    count on the device)."""
    import torch
    from paper_1611_03226_b300 import fit as F
    w = synth.dpd_fit(n=1 << 15)
    x = torch.from_numpy(w.x).cuda()
    hg, lg = F.ila_fit(x, steps=30, graph=True)
    he, le = F.ila_fit(x, steps=30, graph=False)
    assert np.max(np.abs(lg - le) / le) < 1e-5
    assert torch.linalg.norm(hg - he) / torch.linalg.norm(he) < 1e-5


def test_iterative_ila_tracks_float64_oracle():
    """Two iterations of indirect learning with the predistorter in the loop
    (20 Adam steps each on 2^14 samples): every loss curve and the NMSE after
    each iteration follow the float64 oracle."""
    import torch
    from paper_1611_03226_b300 import fit as F
    w = synth.dpd_fit(n=1 << 14)
    h, curves, nmse = F.ila_fit_iterative(torch.from_numpy(w.x).cuda(), iterations=2, steps=20)
    h64, curves64, nmse64 = OF.ila_fit_iterative(w.x, iterations=2, steps=20)
    for c, c64 in zip(curves, curves64):
        assert np.max(np.abs(c - c64) / c64) < 1e-3
    assert np.max(np.abs(np.array(nmse) - nmse64)) < 1e-3
    assert np.linalg.norm(h.cpu().numpy() - h64) / np.linalg.norm(h64) < 1e-3


def test_fused_mse_matches_plain_torch_loss():
    """dpd_mse's value and tap gradient equal those of the plain composition
    mean |dpd(u, h) - t|^2 through autograd."""
    import torch
    from paper_1611_03226_b300.dpd import dpd, dpd_mse
    rng = np.random.default_rng(9)
    n, K, M = 5000, 4, 10
    u = torch.tensor((rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64), device="cuda")
    t = torch.tensor((rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64), device="cuda")
    h0 = torch.tensor((rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64),
                      device="cuda")
    h1 = h0.clone().requires_grad_(True)
    l1 = dpd_mse(u, h1, t, (1, 3, 5, 7))
    l1.backward()
    h2 = h0.clone().requires_grad_(True)
    l2 = (dpd(u, h2, (1, 3, 5, 7)) - t).abs().pow(2).mean()
    l2.backward()
    assert abs(l1.item() - l2.item()) <= 1e-5 * l2.item()
    assert torch.linalg.norm(h1.grad - h2.grad) <= 1e-4 * torch.linalg.norm(h2.grad)


@pytest.mark.parametrize("n,K,M", [(700, 3, 5), (3000, 4, 10)])
def test_fused_mse_float64_gradcheck_and_upstream_scale(n, K, M):
    """The fused loss in float64: gradcheck of the taps at default tolerances
    (one and several tiles of 1024, a ragged last tile), and an upstream
    gradient other than 1 (3 * loss) scales the taps' gradient by 3."""
    import torch
    from paper_1611_03226_b300.dpd import dpd_mse
    rng = np.random.default_rng(n + 7)
    orders = (1, 3, 5, 7)[:K]
    u = torch.tensor(rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n), dtype=torch.complex128, device="cuda")
    t = torch.tensor(rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n), dtype=torch.complex128, device="cuda")
    h = torch.tensor(rng.normal(0, .2, (K, M)) + 1j * rng.normal(0, .2, (K, M)), dtype=torch.complex128,
                     device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda b: dpd_mse(u, b, t, orders), (h,), nondet_tol=0.0)
    l1 = dpd_mse(u, h, t, orders)
    g1, = torch.autograd.grad(l1, h)
    g3, = torch.autograd.grad(3 * dpd_mse(u, h, t, orders), h)
    assert torch.linalg.norm(g3 - 3 * g1) <= 1e-12 * torch.linalg.norm(g1)
    # the loss itself against its definition on the float64 forward
    from paper_1611_03226_b300.dpd import dpd
    want = (dpd(u, h.detach(), orders) - t).abs().pow(2).mean()
    assert abs(l1.item() - want.item()) <= 1e-12 * want.item()
