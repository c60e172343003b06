"""GB300-native (sm_103a) D3V15 finite-difference lattice Boltzmann solver for
the 3D compressible Euler equations (Chen, Xu, Zhang & Li, arXiv:1010.4135).

The compute path is the C-ABI library liblbm.so built from ``csrc/`` (see
include/lbm.h); ``_abi`` binds it with ctypes under the same names, and
``Sim`` owns one grid with a torch-allocated workspace and stream.
"""
from . import _abi
from ._abi import LbmError

__all__ = ["_abi", "LbmError", "Sim", "from_workload"]


def __getattr__(name):
    # torch is imported lazily so that the ABI layer loads without it
    if name in ("Sim", "from_workload"):
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
