"""Dynamic-data-rate dataflow engine for one B300 (sm_103a).

Executes actor networks whose token consumption and production depend on the
data (Boutellier & Hautala, SiPS 2016): control tokens, device-side scans of
per-firing token counts, ring-buffer FIFOs with delay tokens, a fused
predistortion actor and a fused motion-detection actor, all in CUDA kernels
behind the C ABI of ``include/dfgpu.h``.

``Net``, ``DfError`` and ``lib`` load ``libdfgpu.so`` on first use and raise
ImportError when it has not been built; the build step itself
(``python -m paper_1611_03226_b300.build``) does not need the library.
"""


def __getattr__(name):
    if name in ("Net",):
        from .net import Net
        return Net
    if name in ("DfError", "lib"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
