"""FP64 CPU oracle for PRNU camera-fingerprint extraction with SDA frames.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  It shares
no code with the CUDA product path (paper_1909_04573_gb300), and the product
path never imports it.

Contents:
  wavelet.py       Daubechies lowpass derived by spectral factorisation; the
                   explicit-matrix DWT used by the Parseval pin
  prnu_oracle.c    literal FP64 loops: SDA mean, mirror pad, periodised DWT /
                   IDWT, local-variance Wiener shrink, residual, MLE
  pipeline.py      the Python API over the C core, finalize and PCE (numpy FFT)
  grad.py          FP64 vector-Jacobian products of weighted SDA, residual,
                   MLE and PCE, and of the whole chain (mean PCE of queries)

Pins: tests/test_oracle_*.py hold every function to textbook values, closed
forms, invariants or brute force; the exact denoiser output on natural-looking
content is held to an independent computation of the definition (explicit
orthogonal level matrices from the published taps, a library periodic box
filter, the transposed matrices as the inverse).
"""
from .pipeline import (DEFAULT, TO_GRAY, WIENER_DFT, ZERO_MEAN, Params, PCEResult,  # noqa: F401
                       cross_correlation, denoise_plane, dwt2_level, fingerprint_accumulate,
                       fingerprint_finalize, idwt2_level, mle_accumulate, pad_mirror, padded_size, pce_match,
                       residual, residual_noise_form, sda_average, shrink_subband, to_gray,
                       wavedec2, waverec2, wiener_dft, zero_mean)
from .wavelet import daubechies_lowpass, dwt_matrix_1d, highpass  # noqa: F401
from .native import build, set_threads, threads  # noqa: F401
from . import grad  # noqa: F401
