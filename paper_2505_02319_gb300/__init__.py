"""GB300 (sm_103a) inexact-Krylov linear-response solver (arXiv:2505.02319 hot path).

``ikr`` is the ctypes binding of libikr.so (include/ikr.h); ``groundstate``
assembles the ground-state input from the library's H_k; ``autograd`` makes
drho(dV) differentiable through the adjoint solve; ``build`` compiles the
CUDA library.
"""
__all__ = ["ikr", "groundstate", "build", "autograd"]
