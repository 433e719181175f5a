"""GB300-native tetrahedral FEM maps of Ebb's relational model.

The compute path is the CUDA library ``libebb_gb300.so`` (C ABI in
``include/ebb.h``); ``abi`` is its thin ctypes binding and ``device_mesh``
binds torch-owned device storage to it.  Importing ``abi`` without the built
library raises ImportError: there is no CPU fallback.
"""
__all__ = ["abi", "device_mesh", "build"]
