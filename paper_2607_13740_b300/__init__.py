"""B300-native GRACE-DG hot path: batched DG coagulation-fragmentation RHS.

The compute path is the C-ABI library ``libgrace.so`` (hand-written sm_103a
CUDA kernels); :mod:`.grace` is a thin ctypes binding over it.  Importing the
package does not load the library; :func:`grace.load` does, and raises if it
is missing.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads"]
