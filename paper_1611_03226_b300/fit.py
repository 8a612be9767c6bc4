"""Indirect-learning fit of a predistorter to a power amplifier (torch plumbing
around the CUDA predistorter and its adjoint).

The amplifier is a Saleh model (AM/AM alpha_a r / (1 + beta_a r^2), AM/PM
alpha_p r^2 / (1 + beta_p r^2)) followed by a 3-tap memory FIR.  Indirect
learning: the postdistorter P is trained so that P(y / G) ~ x, where y is the
amplifier output for input x and G = alpha_a * sum(memory taps) its
small-signal gain; the trained P is then used as the predistorter.  The loss
is mean |P(y/G) - x|^2 over the whole signal, minimised with Adam starting
from the identity (h[0,0] = 1).  P's forward and gradient run in the
engine's kernels (DPDFunction); everything else is plain torch.
ila_fit_iterative repeats the procedure with the predistorter in the loop.
"""
from __future__ import annotations

import torch

from .dpd import dpd, dpd_mse


def saleh_pa(x: torch.Tensor, saleh=(2.1587, 1.1517, 4.0033, 9.1040),
             memory=(1.0, 0.1, -0.05)) -> torch.Tensor:
    aa, ba, ap, bp = saleh
    r = x.abs()
    r2 = r * r
    amp = aa * r / (1 + ba * r2)
    phase = torch.angle(x) + ap * r2 / (1 + bp * r2)
    v = torch.polar(amp, phase)
    y = torch.zeros_like(v)
    for i, c in enumerate(memory):
        if i == 0:
            y += c * v
        else:
            y[i:] += c * v[:-i]
    return y


def small_signal_gain(saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05)) -> float:
    return saleh[0] * float(sum(memory))


def nmse_db(a: torch.Tensor, ref: torch.Tensor) -> float:
    num = (a - ref).abs().pow(2).sum()
    den = ref.abs().pow(2).sum()
    return float(10 * torch.log10(num / den))


def adam_fit(u: torch.Tensor, target: torch.Tensor, h0: torch.Tensor, orders, steps=200, lr=1e-3,
             graph=True):
    """Adam on the predistorter taps so that P(u) ~ target (loss mean |P(u) - target|^2);
    P's forward and gradient run in the engine's kernels.  Returns (h, losses).

    graph=True records one whole training step (forward, loss, adjoint, Adam update)
    as a CUDA graph and replays it `steps` times, so the host issues one launch
    per step instead of a few dozen; graph=False runs the same step eagerly.
    The captured step's update is torch's fused Adam (one kernel) on the real
    view of the taps."""
    # the taps as a real (K, M, 2) leaf: Adam's moments are then per real and
    # imaginary part (the oracle's update), and in the captured step torch's
    # fused Adam (one kernel) does the update
    hr = torch.view_as_real(h0.detach()).clone().requires_grad_(True)
    if not graph:
        opt = torch.optim.Adam([hr], lr=lr)
        losses = []
        for _ in range(steps):
            opt.zero_grad(set_to_none=True)
            loss = dpd_mse(u, torch.view_as_complex(hr), target, orders)
            loss.backward()
            opt.step()
            losses.append(loss.detach())
        return torch.view_as_complex(hr.detach()).clone(), torch.stack(losses).cpu().numpy()
    opt = torch.optim.Adam([hr], lr=lr, capturable=True, fused=True)

    def train_step():
        loss = dpd_mse(u, torch.view_as_complex(hr), target, orders)
        loss.backward()
        opt.step()
        return loss.detach()

    # two eager steps on a side stream create the optimizer state, the gradient
    # and the adjoint's scratch before capture; then taps and state are reset
    side = torch.cuda.Stream(device=u.device)
    side.wait_stream(torch.cuda.current_stream(u.device))
    with torch.cuda.stream(side):
        for _ in range(2):
            opt.zero_grad(set_to_none=True)
            train_step()
        with torch.no_grad():
            hr.copy_(torch.view_as_real(h0))
            for st in opt.state[hr].values():
                st.zero_()
    torch.cuda.current_stream(u.device).wait_stream(side)
    g = torch.cuda.CUDAGraph()
    opt.zero_grad(set_to_none=True)
    with torch.cuda.graph(g):
        static_loss = train_step()
    losses = torch.empty(steps, dtype=static_loss.dtype, device=u.device)
    for i in range(steps):
        g.replay()
        losses[i].copy_(static_loss)
    return torch.view_as_complex(hr.detach()).clone(), losses.cpu().numpy()


def ila_fit(x: torch.Tensor, K=4, M=10, orders=(1, 3, 5, 7), steps=200, lr=1e-3,
            saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05), graph=True):
    """Returns (h, losses) for complex64 CUDA input x."""
    G = small_signal_gain(saleh, memory)
    u = (saleh_pa(x, saleh, memory) / G).to(torch.complex64).contiguous()
    h = torch.zeros((K, M), dtype=torch.complex64, device=x.device)
    h[0, 0] = 1
    return adam_fit(u, x, h, orders, steps, lr, graph)


def ila_fit_iterative(x: torch.Tensor, iterations=3, K=4, M=10, orders=(1, 3, 5, 7), steps=200,
                      lr=1e-3, saleh=(2.1587, 1.1517, 4.0033, 9.1040), memory=(1.0, 0.1, -0.05),
                      graph=True):
    """Iterative indirect learning: in iteration i the current predistorter P_i
    drives the amplifier with z = P_i(x) (forward kernel); a postdistorter started
    from P_i's taps is trained so that P(PA(z)/G) ~ z and becomes P_{i+1}; P_0 is
    the identity.  Returns (h, loss curves per iteration, NMSE in dB of
    PA(P_{i+1}(x))/G against x after each iteration)."""
    G = small_signal_gain(saleh, memory)
    h = torch.zeros((K, M), dtype=torch.complex64, device=x.device)
    h[0, 0] = 1
    curves, nmse = [], []
    for _ in range(iterations):
        with torch.no_grad():
            z = dpd(x, h, orders).contiguous()
            u = (saleh_pa(z, saleh, memory) / G).to(torch.complex64).contiguous()
        h, losses = adam_fit(u, z, h, orders, steps, lr, graph)
        curves.append(losses)
        with torch.no_grad():
            nmse.append(nmse_db(saleh_pa(dpd(x, h, orders), saleh, memory) / G, x))
    return h, curves, nmse
