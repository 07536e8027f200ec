"""GB300-native wavelet-reduced hyperspectral anomaly detection (LRX, DWRX, DWEST).

The compute path is libwdad.so (hand-written CUDA for sm_103a behind a C ABI,
include/wdad.h); `wdad` is its ctypes binding and `synth` the seeded scene
generator.  Importing the package loads nothing; `wdad` loads the library on
first use and raises if it is missing.
"""
