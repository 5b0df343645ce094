"""GB300-native dual-layer lossless Radiance (RGBE) coder with the simple
linear regressive mantissa estimator (SLRME) of arXiv 2309.11072.

The codec runs in hand-written CUDA kernels (``csrc/``) behind a C ABI
(``include/slrme.h``); ``native`` loads that library and ``codec`` is the
Python API.  ``synth`` makes seeded synthetic RGBE images.  Importing the
package loads nothing native: the library is loaded on first use and the
call fails loudly if it is missing.
"""
__all__ = ["synth", "native", "codec"]
