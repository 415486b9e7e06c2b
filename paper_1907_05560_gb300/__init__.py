"""GB300-native multi-angle neutrino flavor evolution (bulb model, XFLAT,
arXiv 1907.05560).

The product is the C-ABI library libxf.so (include/xf.h, sources in csrc/);
``xf`` is its thin ctypes binding and ``inputs`` the seeded workload
parameters.  Importing this package does not load the CUDA library; the
first use of ``xf`` does, and fails loudly when it is missing.
"""

__all__ = ["inputs", "xf", "build"]
