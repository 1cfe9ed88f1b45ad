"""GB300 shifted-COCG Green's-function library (arXiv:0802.0748, Sec. III.C).

The compute path is the CUDA library ``_build/libscocg.so`` behind the C ABI
of ``include/scocg.h``; ``scocg`` is its thin ctypes binding (argument
marshalling only, PyTorch tensors for device memory and streams).  Importing
the package does not load the library; the first call does, and fails loudly
when the library has not been built.
"""

__all__ = ["scocg", "inputs"]
