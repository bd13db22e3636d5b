"""GB300-native even-odd preconditioned Moebius domain-wall solver (arXiv:1701.07559).

The compute path is the CUDA library libmdwf.so (sources in csrc/, C ABI in
include/mdwf.h); ``mdwf`` is its ctypes binding and ``serving`` the request
loop built on it.  Build with ``paper_1701_07559_gb300.build.build()``.
"""
__all__ = ['build', 'mdwf', 'serving']
