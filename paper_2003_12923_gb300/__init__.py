"""GB300-native ESMP2-TOP(1): the Krylov solve of the first-order equation and its sigma build.

The compute path is libesmp2 (CUDA, sm_103a) behind the C ABI of include/esmp2.h;
`esmp2.Handle` is its Python binding.
"""
from . import esmp2
from .esmp2 import FP64, MIXED_BF16, Esmp2Error, Handle

__all__ = ["esmp2", "Handle", "Esmp2Error", "FP64", "MIXED_BF16"]
