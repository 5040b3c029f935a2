"""GB300-native stochastic-deterministic domain decomposition (SDD) mesh
generator: Monte Carlo evaluation of the Feynman-Kac representation of the
linear Winslow generator at subdomain-interface nodes, then independent
Dirichlet solves of the subdomains (Bihlo & Haynes, arXiv 1310.3435).

The compute path is libsdd.so (CUDA kernels for sm_103a behind the C ABI of
include/sdd.h); ``native`` is its ctypes binding.
"""
from . import build  # noqa: F401
from . import native  # noqa: F401

__all__ = ["build", "native"]
