"""GB300-native (sm_103a) DOCH Ising solver.

Hot path of "A Continuous Energy Ising Machine Leveraging Difference-of-Convex
Programming" (arXiv 2509.01928): the fixed-point iteration
x <- cbrt(((J + alpha I) x + h) / beta) (Eq. FPE, Algorithm 1) fused with the
coupling product J x, then sign rounding and an exact Ising-energy / Max-Cut
reduction. The arithmetic runs in hand-written CUDA kernels behind the C ABI
of include/ising.h (libising_doch.so); ``_native`` is its ctypes binding and
``autograd`` wraps the adjoint for PyTorch. Importing this package loads
nothing native; the first call into ``_native`` does, and fails loudly when
the library has not been built.
"""
from . import inputs  # noqa: F401  (seeded synthetic inputs, numpy only)

__all__ = ["inputs"]
