"""Error bounds of the parity tests for products with G = M_perp^T M_perp.

A product with G is two FFTs over the grid (inverse, mask, forward) plus the
beta <-> v maps.  For an FFT of total length n computed in a precision of unit
round-off u with accurate twiddles, Higham ("Accuracy and Stability of Numerical
Algorithms", Sec. 24.1) bounds the norm-wise forward error by
log2(n) eta / (1 - log2(n) eta) with eta ~ 6u per radix-2 stage; two transforms and
the scalings of the maps give
    ||G_computed p - G p||_2 <= c u (log2 n + 2) ||p||_2,   c = 12,
with u = 2^-53 (FP64) or 2^-24 (the FP32 products of the mixed mode; rounding the
FP64 operand to FP32 is one more u).  Element by element we require
    |G_computed p - G p|_i <= c u (log2 n + 2) ||G p||_inf,
the same constant against the largest entry: FFT rounding errors spread over all
outputs (their typical size is u sqrt(log2 n) times the rms of the output), so a
localised error -- one wrong pencil, a twiddle wrong in its last bits, a ghost
slot handled slightly wrong -- shows up here long before the norm moves.
"""

import numpy as np

from paper_2502_04217_gb300 import binding

C_FFT = 12.0
UNIT_ROUNDOFF = {binding.IPM_FP64: 2.0 ** -53, binding.IPM_MIXED: 2.0 ** -24}


def fft_bound(dims, precision):
    """c u (log2 n + 2): the relative error allowed for one product with G (module docstring)."""
    n = int(np.prod(dims))
    return C_FFT * UNIT_ROUNDOFF[precision] * (np.log2(max(n, 2)) + 2.0)


def assert_g_close(got, ref, p, dims, precision):
    """got = the library's G p, ref = the oracle's, both on the half spectrum; p the
    operand (beta order).  Norm-wise and element-wise bounds of the module docstring."""
    b = fft_bound(dims, precision)
    err = np.abs(got - ref)
    assert np.linalg.norm(err) <= b * np.linalg.norm(p), ("norm-wise", np.linalg.norm(err) / np.linalg.norm(p), b)
    scale = np.abs(ref).max()
    assert np.all(err <= b * scale), ("element-wise", float(err.max() / scale), b)


