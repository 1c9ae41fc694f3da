"""GB300-native NSFR-EC residual hot path (Cicchino & Nadarajah, arXiv 2312.07725).

The compute runs in ``libnsfr.so`` (hand-written sm_103a CUDA kernels behind the
C ABI of include/nsfr.h); ``nsfr.Solver`` is its ctypes binding and
``autograd`` its torch.autograd wrapper.
"""
from .nsfr import NSFRError, Solver, load_library  # noqa: F401
