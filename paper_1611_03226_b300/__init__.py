"""Dynamic-data-rate dataflow engine for one B300 (sm_103a).

Executes actor networks whose token consumption and production depend on the
data (Boutellier & Hautala, SiPS 2016): control tokens, device-side scans of
per-firing token counts, ring-buffer FIFOs with delay tokens, a fused
predistortion actor and a fused motion-detection actor, all in CUDA kernels
behind the C ABI of ``include/dfgpu.h``.
"""
from ._lib import DfError, lib  # noqa: F401  (raises ImportError when the library is missing)
from .net import Net  # noqa: F401
