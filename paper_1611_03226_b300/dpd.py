"""Differentiable predistorter on torch CUDA tensors (marshalling only).

``dpd(x, h, orders)`` evaluates y[t] = sum_k sum_m h[k,m] z_k[t-m] with
z_k = |x|^(orders[k]-1) x (every branch active, zero history) through
df_dpd_forward; its gradient goes through the hand-written adjoint
df_dpd_backward, which recomputes z_k from x instead of storing it.
Gradients follow PyTorch's convention for complex tensors
(dL/dRe + i dL/dIm).  complex64 tensors run the float32 kernels, complex128
tensors the float64 instantiation of the same kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def _orders(orders):
    arr = (C.c_int32 * len(orders))(*[int(o) for o in orders])
    return arr


def _check_inputs(x, h):
    if x.dtype not in (torch.complex64, torch.complex128) or h.dtype != x.dtype:
        raise TypeError("x and h must both be complex64 (float32 kernels) or both complex128 (float64)")
    if not (x.is_cuda and h.is_cuda):
        raise ValueError("x and h must be CUDA tensors")
    if x.dim() != 1 or h.dim() != 2:
        raise ValueError("x is (n,), h is (K, M)")


def dpd_forward(x: torch.Tensor, h: torch.Tensor, orders) -> torch.Tensor:
    _check_inputs(x, h)
    x = x.contiguous()
    h = h.contiguous()
    K, M = h.shape
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    fn = L.lib.df_dpd_forward if x.dtype == torch.complex64 else L.lib.df_dpd_forward_f64
    L.check(fn(C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(h.data_ptr()), K, M, _orders(orders),
               C.c_void_p(y.data_ptr()), C.c_void_p(stream)), "df_dpd_forward")
    return y


def dpd_backward(x: torch.Tensor, h: torch.Tensor, orders, grad_y: torch.Tensor,
                 need_x: bool = True):
    _check_inputs(x, h)
    x = x.contiguous()
    h = h.contiguous()
    grad_y = grad_y.contiguous().to(x.dtype)
    K, M = h.shape
    gx = torch.empty_like(x) if need_x else None
    gh = torch.empty_like(h)
    # the adjoint's tap-gradient partial sums come from torch's allocator, which
    # orders them on this stream and keeps them valid inside CUDA graph capture
    n_scratch = L.lib.df_dpd_backward_scratch_elems(x.numel(), K, M)
    scratch = torch.empty(n_scratch, dtype=x.dtype, device=x.device)
    stream = torch.cuda.current_stream(x.device).cuda_stream
    fn = L.lib.df_dpd_backward_scratch if x.dtype == torch.complex64 else L.lib.df_dpd_backward_f64
    L.check(fn(C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(h.data_ptr()), K, M, _orders(orders),
               C.c_void_p(grad_y.data_ptr()), C.c_void_p(gx.data_ptr()) if need_x else None,
               C.c_void_p(gh.data_ptr()), C.c_void_p(scratch.data_ptr()), n_scratch, C.c_void_p(stream)),
            "df_dpd_backward")
    return gx, gh


class DPDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, h, orders):
        ctx.save_for_backward(x, h)
        ctx.orders = tuple(orders)
        return dpd_forward(x, h, orders)

    @staticmethod
    def backward(ctx, grad_y):
        x, h = ctx.saved_tensors
        gx, gh = dpd_backward(x, h, ctx.orders, grad_y, need_x=ctx.needs_input_grad[0])
        return gx, gh, None


def dpd(x, h, orders):
    return DPDFunction.apply(x, h, tuple(orders))


class DPDMSEFunction(torch.autograd.Function):
    """loss = mean |P_h(u) - target|^2 in the engine's kernels: the forward
    writes the residual and the loss (df_dpd_mse_forward), the backward gives
    grad_h with dL/dy = 2 (y - target) g / n formed inside the adjoint
    (df_dpd_mse_backward), g the upstream gradient of the loss."""

    @staticmethod
    def forward(ctx, u, h, target, orders):
        if u.requires_grad or target.requires_grad:
            raise ValueError("dpd_mse is differentiable in h only: u and target must not require grad")
        _check_inputs(u, h)
        if target.dtype != u.dtype or not target.is_cuda or target.shape != u.shape:
            raise ValueError("target must be a CUDA tensor of u's dtype and shape")
        u = u.contiguous()
        h = h.contiguous()
        target = target.contiguous()
        K, M = h.shape
        f64 = u.dtype == torch.complex128
        real = torch.float64 if f64 else torch.float32
        resid = torch.empty_like(u)
        loss = torch.empty((), dtype=real, device=u.device)
        n_part = L.lib.df_dpd_mse_partial_elems(u.numel())
        partial = torch.empty(n_part, dtype=real, device=u.device)
        stream = torch.cuda.current_stream(u.device).cuda_stream
        fn = L.lib.df_dpd_mse_forward_f64 if f64 else L.lib.df_dpd_mse_forward
        L.check(fn(C.c_void_p(u.data_ptr()), u.numel(), C.c_void_p(h.data_ptr()), K, M, _orders(orders),
                   C.c_void_p(target.data_ptr()), C.c_void_p(resid.data_ptr()), C.c_void_p(loss.data_ptr()),
                   C.c_void_p(partial.data_ptr()), n_part, C.c_void_p(stream)), "df_dpd_mse_forward")
        ctx.save_for_backward(u, h, resid)
        ctx.orders = tuple(orders)
        return loss

    @staticmethod
    def backward(ctx, g):
        u, h, resid = ctx.saved_tensors
        K, M = h.shape
        f64 = u.dtype == torch.complex128
        g = g.reshape(()).to(torch.float64 if f64 else torch.float32).contiguous()
        gh = torch.empty_like(h)
        n_scratch = L.lib.df_dpd_backward_scratch_elems(u.numel(), K, M)
        scratch = torch.empty(n_scratch, dtype=u.dtype, device=u.device)
        stream = torch.cuda.current_stream(u.device).cuda_stream
        fn = L.lib.df_dpd_mse_backward_f64 if f64 else L.lib.df_dpd_mse_backward
        L.check(fn(C.c_void_p(u.data_ptr()), u.numel(), C.c_void_p(h.data_ptr()), K, M, _orders(ctx.orders),
                   C.c_void_p(resid.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(gh.data_ptr()),
                   C.c_void_p(scratch.data_ptr()), n_scratch, C.c_void_p(stream)), "df_dpd_mse_backward")
        return None, gh, None, None


def dpd_mse(u, h, target, orders):
    """mean |P_h(u) - target|^2, differentiable in h (u and target are data)."""
    return DPDMSEFunction.apply(u, h, target, tuple(orders))
