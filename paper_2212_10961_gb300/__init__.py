"""GB300-native spectral Gaussian-random-field synthesis.

Direct evaluation of the spectral (Fourier) sum of a Gaussian random field at
arbitrary cell centres, with lognormal / thresholded (facies) property maps,
its adjoint, and batched ensembles -- the random-field generator of Icardi et
al., "Computational framework for complex flow and transport in heterogeneous
porous media" (arXiv 2212.10961), Sec. 3, Sec. 4.1 and Appendices A-B.

The computation runs in libgrf.so (C ABI in include/grf.h): host C++ for the
O(N) mode drawing and table packing, hand-written sm_103a CUDA kernels for
every per-cell step.  This package is the Python binding.
"""
__all__ = ["field", "workloads"]
