"""df_dpd_backward_noalloc: the adjoint for callers that may not allocate device
memory (its tap-gradient partial sums sit in a fixed array in the library).

It must give the same gradients as df_dpd_backward, call after call (the fixed
array is reused by every call), and refuse sizes beyond that array.  This file
is collected last so a failure here cannot hide the other tests' results."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _proto(lib):
    fn = lib.df_dpd_backward_noalloc
    fn.restype = C.c_int32
    fn.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int32, C.c_int32,
                   C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_noalloc_matches_allocating_adjoint_twice():
    import torch
    from paper_1611_03226_b300 import _lib as L
    noalloc = _proto(L.lib)
    rng = np.random.default_rng(2024)
    n, K, M = 50000, 4, 10
    orders = (C.c_int32 * K)(1, 3, 5, 7)
    x = torch.from_numpy((rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64)).cuda()
    h = torch.from_numpy((rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    p = lambda t: C.c_void_p(t.data_ptr())
    for call in range(2):
        g = torch.from_numpy((rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)).cuda()
        gx_ref, gh_ref = torch.empty_like(x), torch.empty_like(h)
        assert L.lib.df_dpd_backward(p(x), n, p(h), K, M, orders, p(g), p(gx_ref), p(gh_ref),
                                     C.c_void_p(stream)) == L.DF_OK
        gx, gh = torch.empty_like(x), torch.empty_like(h)
        assert noalloc(p(x), n, p(h), K, M, orders, p(g), p(gx), p(gh), C.c_void_p(stream)) == L.DF_OK
        torch.cuda.synchronize()
        assert _rel(gx.cpu().numpy(), gx_ref.cpu().numpy()) <= TOL, call
        assert _rel(gh.cpu().numpy(), gh_ref.cpu().numpy()) <= TOL, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1611_03226_b300 import _lib as L
    noalloc = _proto(L.lib)
    K, M = 16, 32                        # 512 partial sums per 1024-sample tile
    n = 1024 * 300                       # 153600 > 131072
    orders = (C.c_int32 * K)(*range(1, 2 * K, 2))
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    h = torch.zeros((K, M), dtype=torch.complex64, device="cuda")
    gh = torch.empty_like(h)
    st = noalloc(C.c_void_p(x.data_ptr()), n, C.c_void_p(h.data_ptr()), K, M, orders,
                 C.c_void_p(x.data_ptr()), None, C.c_void_p(gh.data_ptr()), None)
    assert st == L.DF_ENOTSUP
