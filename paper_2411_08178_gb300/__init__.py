"""GB300-native randomized Nystrom-preconditioned image reconstruction.

The computation lives in the CUDA library lib/libnys.so (C ABI: include/nys.h);
`paper_2411_08178_gb300.api` is a thin ctypes binding with the same names.
Importing this package does not load the library; the first call that needs
it does, and fails loudly if it has not been built.
"""
from ._abi import LIB_PATH, NysError, load  # noqa: F401

__all__ = ["LIB_PATH", "NysError", "load"]
