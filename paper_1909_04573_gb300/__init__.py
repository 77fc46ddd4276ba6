"""GB300 (sm_103a) PRNU camera-fingerprint extraction with Spatial Domain
Averaged frames: hand-written CUDA kernels behind the C ABI in include/prnu.h
(libprnu.so), with a thin Python binding (prnu.py) and a seeded synthetic
camera generator (synth.py)."""
