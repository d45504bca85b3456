"""GB300-native HyRes (arXiv 2204.06979, Sec. 2.1): the data-parallel path of
the automatic wavelet-domain low-rank hyperspectral denoiser, as hand-written
sm_103a CUDA kernels behind the C ABI of ``include/hyde.h``.

``api`` holds the PyTorch-facing binding; ``build`` compiles libhyde.so.
"""

__all__ = ["api", "build"]
