"""GB300-native visibility stacking in the Fourier domain (ViSta hot path).

The CUDA library libvista.so (include/vista.h) does the work; `vista` is its
thin Python binding and `synth` makes seeded synthetic inputs.
"""
from . import build  # noqa: F401
