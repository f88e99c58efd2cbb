"""GB300-native FFT-based continuous wavelet transform of multichannel EEG.

Implements the method of arXiv 2506.07793 (forward FFT per channel, product
with the analytic Fourier-domain Morlet wavelet of each scale, inverse FFT,
reduction to complex / power / phase) as hand-written sm_103a CUDA kernels
behind a C ABI (include/cwt.h).  This package is the thin ctypes binding;
importing it fails if the CUDA library has not been built.
"""
from .cwt import *  # noqa: F401,F403
from .cwt import CWT, CWTError, LIB_PATH  # noqa: F401
