"""Kalman-filter track building and fitting on GB300 (sm_103a): the data-parallel hot path
of Cerati et al., "Kalman filter tracking on parallel architectures" (arXiv:1702.06359).

The compute path is libtkf.so (CUDA kernels behind the C ABI in include/tkf.h); `tkf` is
its Python binding (argument marshalling only).  Importing this package does not load the
library; `tkf.lib()` does, and fails loudly when it has not been built.
"""
