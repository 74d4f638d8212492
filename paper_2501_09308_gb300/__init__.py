"""xrdvi: GB300-native variational sparse Bayesian crystalline-phase search.

The Monte-Carlo ELBO step of arXiv 2501.09308 as hand-written CUDA kernels
for sm_103a behind the C ABI of ``include/xrdvi.h``.  ``xrdvi`` is the ctypes
binding, ``autograd`` the torch.autograd.Function wrapper, ``serving`` the
continuous-batching request loop and ``synth`` the seeded synthetic inputs.
The library is loaded lazily, on first use.
"""
__all__ = ["xrdvi", "synth", "build"]
