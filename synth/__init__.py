"""Seeded synthetic hyperspectral inputs shared by the tests, the benchmark and
the oracle checks.

This package draws random numbers and builds clean cubes, noisy cubes,
window tables and the mixed-noise kinds of ``synth.noise``. It holds none of the denoiser's arithmetic (no regression, no
Gram, no wavelet, no threshold), so both the CUDA path and the FP64 oracle can
consume its output without sharing any of the method's code.
"""

from .cube import make_cube, make_scene, cube_config, CONFIGS  # noqa: F401
from .windows import make_window_table  # noqa: F401
