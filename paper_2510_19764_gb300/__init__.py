"""GB300-native structural plasticity on ragged sparse spiking networks.

The compute path is libsnnsp.so (CUDA for sm_103a, C ABI in include/snnsp.h); `abi`
binds it with ctypes and `net` allocates device memory with torch and fills the
descriptors.  Nothing here computes the method on the CPU.
"""
from . import abi  # noqa: F401

__all__ = ["abi"]
