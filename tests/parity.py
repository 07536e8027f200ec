"""Shared parity helpers for the GPU-vs-oracle tests."""
import numpy as np

import oracle

# FP32 paths: per-pixel relative error <= 1e-4; DWT coefficients 1e-5; indices and census
# bit-exact.
#
# Departure from the plain relative error |s - s_ref| / max(|s_ref|, 1e-6 median|s_ref|):
# relerr() below divides by max(|s_ref|, sqrt(|s_ref| median|s_ref|)).  The two agree at and
# above the median score; below it this floor is larger than 1e-6 median, so the bar is looser
# for small scores.  The reason is the error model of a Mahalanobis score s = d^T C^-1 d: the
# FP32 rounding of d is a fixed fraction of the data scale, so the absolute error of s grows
# like sqrt(s), not like s, and a plain relative bar would blow up as s -> 0 (low-band cubes
# put many pixels near s = 0).
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


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _window(cube, y, x, wi, wo, inner):
    H, W, _ = cube.shape
    ri, ro = wi // 2, wo // 2
    r = ri if inner else ro
    return np.array([cube[oracle.reflect(y + dy, H), oracle.reflect(x + dx, W)]
                     for dy in range(-r, r + 1) for dx in range(-r, r + 1)
                     if inner or max(abs(dy), abs(dx)) > ri])


def bf16_data_score(cube, p, det, wi, wo, loading=1e-3):
    """LRX (det 0) or DWRX (det 1) of Eq. 1 / Eq. 5 evaluated in FP64 on the background samples
    centred on their FP32 mean and rounded to BF16: the quantity the MIXED path's BF16 Gram
    represents exactly."""
    H, W, L = cube.shape
    y, x = divmod(int(p), W)
    X = _window(cube, y, x, wi, wo, inner=False)
    mu = X.astype(np.float64).mean(0).astype(np.float32)
    Xc = bf16_round(X - mu[None]).astype(np.float64)
    C = Xc.T @ Xc / X.shape[0]
    delta = loading * np.trace(C) / L
    if det == 0:
        d = cube[y, x].astype(np.float64) - mu
    else:
        d = _window(cube, y, x, wi, wo, inner=True).astype(np.float64).mean(0) - mu
    s = d @ np.linalg.solve(C + delta * np.eye(L), d)
    return s if det == 0 else abs(s)
