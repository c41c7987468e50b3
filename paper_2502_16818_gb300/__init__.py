"""GB300-native central-moment discrete Boltzmann method (CDBM).

The compute path is the CUDA library ``_build/libcdbm.so`` (C ABI in
``include/cdbm.h``); ``cdbm`` is its ctypes binding and ``Solver`` a convenience
wrapper that takes device memory and streams from PyTorch.  ``workloads`` holds
the seeded initial conditions of the paper's test problems.
"""
from .cdbm import (BatchSolver, CdbmError, Solver, CDBM_BC_PERIODIC, CDBM_BC_ZEROGRAD, CDBM_FP64,  # noqa: F401
                   CDBM_FP32_BULK, CDBM_FP32_DF64, CDBM_FP32_DEV, CDBM_RK2_MIDPOINT, CDBM_RK2_TVD)
from . import workloads  # noqa: F401


def build(force: bool = False) -> str:
    """Compiles libcdbm.so for sm_103a in-tree and returns its path."""
    from . import _build
    return _build.build(force=force)
