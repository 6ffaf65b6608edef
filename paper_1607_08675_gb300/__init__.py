"""GB300-native filtered lattice Boltzmann MHD (arXiv:1607.08675).

The compute path is the CUDA library ``liblbmhd.so`` (sm_103a) behind the C
ABI declared in ``include/lbmhd.h``; ``paper_1607_08675_gb300.lbmhd`` is the
thin ctypes binding with the same names.  Nothing is loaded at import time,
so the seeded input generators in ``paper_1607_08675_gb300.inputs`` can be
used without a GPU; the first library call raises if the library was not
built.
"""
__all__ = ["inputs", "lbmhd"]
