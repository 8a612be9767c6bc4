"""CPU oracle for dynamic-data-rate actor networks (test infrastructure).

This package is test infrastructure, not product code.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import or run it.  It shares no code with the CUDA engine and never imports it.

It is a plain, slow, sequential restatement of the paper (Boutellier & Hautala,
"Executing Dynamic Data Rate Actor Networks on OpenCL Platforms", SiPS 2016):

* :mod:`oracle.network`  the network model of Sec. 2.2: actors, order-preserving
  bounded FIFO channels with a token rate, static and dynamic actors with a
  control port, initial (delay) tokens; a sweep interpreter that fires one
  actor at a time, a random-order scheduler, a thread-per-actor runner
  (Sec. 3.3) and brute-force interleaving enumeration for tiny networks.
* :mod:`oracle.actors`   actor bodies: the predistortion network of Sec. 4.2
  (Poly, FIR, Adder and their fused composition), the motion-detection stages
  (frame difference, threshold, 3x3 erosion/dilation, tile emission), copy.
* :mod:`oracle.dpd`      predistortion arithmetic in float64 and its adjoint.
* :mod:`oracle.motion`   motion-detection arithmetic on exact integers.
* :mod:`oracle.pa`       the synthetic power amplifier used by the fit.
* :mod:`oracle.paper_layout` Eq. 1 channel capacities and the Fig. 2
  triple-buffer access pattern.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
except where its docstring says "parity unpinned".
"""
