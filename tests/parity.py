"""Shared parity helpers for the GPU-vs-oracle tests."""
import numpy as np

# FP32 paths: per-pixel relative error |s - s_ref| / max(|s_ref|, 1e-6 median|s_ref|) <= 1e-4;
# DWT coefficients 1e-5; indices and census bit-exact.
TOL_SCORE = 1e-4
TOL_DWT = 1e-5


def relerr(got, want):
    """LRX/DWRX error |s - s_ref| / max(|s_ref|, sqrt(|s_ref| * median|s_ref|)).

    FP32 rounding of the centred difference vector d is a fixed fraction of the
    data scale, so a Mahalanobis score s = d^T C^-1 d carries an error that grows
    like sqrt(s): at and above the median score this is the plain relative error,
    below it the bar follows the sqrt(s) error model instead of blowing up at s -> 0."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    fin = np.isfinite(want)
    med = np.median(np.abs(want[fin])) if fin.any() else 0.0
    aw = np.abs(np.where(fin, want, 0.0))
    den = np.maximum(np.maximum(aw, np.sqrt(aw * med)), 1e-300)
    e = np.abs(got - want) / den
    both_nan = np.isnan(got) & np.isnan(want)
    e[both_nan] = 0.0
    e[np.isnan(got) ^ np.isnan(want)] = np.inf
    return e


def dwest_relerr(got, want, aux):
    """DWEST error against max(|s_ref|, ||m_diff||): Eq. 4 adds signed projections of
    m_diff, so a near-cancelling sum is far smaller than the terms the FP32 path
    rounds; the error is measured on the scale of those terms."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.maximum(np.abs(want), np.asarray(aux)[..., 4])
    e = np.abs(got - want) / np.maximum(den, 1e-300)
    e[np.isnan(got) & np.isnan(want)] = 0.0
    e[np.isnan(got) ^ np.isnan(want)] = np.inf
    return e


def dwest_ok_mask(aux, sel_margin=1e-4, sign_margin=1e-3, gap=1e-2):
    """Pixels whose DWEST score is well determined in FP32: no eigenvalue within
    sel_margin * max|lambda| of the threshold, the two largest entries of every
    selected eigenvector apart by sign_margin, and selected eigenvalues separated
    by gap * max|lambda|.  The others are counted, not compared."""
    a = np.asarray(aux)
    return (a[..., 0] >= sel_margin) & (a[..., 1] >= sign_margin) & (a[..., 2] >= gap)
