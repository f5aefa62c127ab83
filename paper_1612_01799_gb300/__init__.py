"""GB300-native free-space Poisson solver: Gaussian-sum FFT convolution (Exl,
arXiv:1612.01799) as hand-written CUDA kernels for sm_103a behind a C ABI
(include/poisson.h).  The solver classes load libgspoisson.so on first use and raise if
it is missing; there is no CPU fallback."""

_API = ("Plan", "solve_batched", "supported_n")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
