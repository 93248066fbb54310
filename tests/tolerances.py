"""Tolerances of the GPU parity tests, each derived from the arithmetic."""

import math

# FP64 filter (DMMA products in FP64): the filtered block must match the
# oracle to 1e-11 relative per column; measured errors are about 3e-15.
FP64_FILTER_RTOL = 1e-11

# One product entry of the 7-slice split-BF16 product (Ozaki-style 7-bit
# slices, pairs s + t <= 6) carries a truncation error of about 2^-49 of
# max|row of H| x max|column| per term of its K-term sum.
SPLIT_UNIT = 2.0 ** -49


def split_filter_rtol(n, max_degree, real=False):
    """Bar for the relative error per column of a degree <= max_degree filter
    on the 7-slice split product: the FP64 filter's bar (1e-11), raised where
    the split product's error model exceeds it.  Model: the K per-term
    truncation errors of a product (K = 2n complex, n real) have no common
    sign and add like sqrt(K), and the m products of the recurrence add
    theirs, so a column's error is about m sqrt(K) 2^-49; the factor 4
    covers the model's constants at large K.  Measured: 1.7e-12 to 5.1e-12
    for n <= 1000 (where the model is not the binding term), 7.3e-12 at
    n = 8000 and 1.04e-11 at n = 22500 (bars 3.2e-11 and 5.4e-11), all with
    degrees up to 36."""
    k = n if real else 2 * n
    return max(FP64_FILTER_RTOL, 4.0 * max_degree * math.sqrt(k) * SPLIT_UNIT)


def reduced_slice_rtol(nslices):
    """Per-column bound of a filter on the leading 3 or 4 slices (about
    2^-21 or 2^-28 relative per product), with the same 4000x allowance
    for degree, K and constants as the reduced-slice tests."""
    return 4000 * 2.0 ** (-7 * nslices)
