"""GB300-native positivity-preserving fifth-order FV compact-WENO Euler solver.

The compute path is the C-ABI library ``libppcweno.so`` (hand-written CUDA for
sm_103a, declared in ``include/pp_cweno.h``); :mod:`.binding` is a thin ctypes
layer over it.  :mod:`.workloads` builds seeded initial data.  Importing this
package loads nothing; the library is loaded on first use of the binding and
fails loudly if it has not been built.
"""

__all__ = ["binding", "workloads"]
