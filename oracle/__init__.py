"""FP64 CPU oracle (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark may use it; the product path never imports it.  Every function
follows the paper's definitions (Sec. 2 Eq. 1-5 for the detectors, Sec. 3 Eq. 6-9
and Fig. 1 for the transform, Sec. 5.3.1 for the ROC AUC) in plain double
precision, see oracle.c for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "cnn_oracle.c")]
_lib = None

LRX, DWRX, DWEST = 0, 1, 2
NAUX = 6  # per-pixel diagnostics of detect(), see oracle.c


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP, no FMA contraction, portable flags)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", _SO + ".tmp", *srcs, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.or_daub_filter.argtypes = [ctypes.c_int, dp]
        L.or_highpass.argtypes = [dp, ctypes.c_int, dp]
        L.or_dwt_step.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, dp]
        L.or_dwt_levels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_dwt_full.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.or_dwt_inverse.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.or_dwt_approx.argtypes = [fp, ctypes.c_long, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
        L.or_reflect.argtypes = [ctypes.c_int, ctypes.c_int]
        L.or_detect.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, i64p,
                                ctypes.c_int64, dp, dp, ctypes.c_int, ctypes.c_int]
        L.or_window_census.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       i64p, ctypes.c_int64, i64p]
        L.or_window_moments.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        i64p, ctypes.c_int64, dp, dp, ctypes.c_int]
        L.or_auc.argtypes = [dp, u8p, ctypes.c_int64]
        L.or_adaptive_threshold.argtypes = [dp, ctypes.c_int64, ctypes.c_double, dp, dp, dp, u8p]
        L.or_adaptive_threshold.restype = ctypes.c_int64
        L.or_scene_whiten.argtypes = [ctypes.c_int, dp, ctypes.c_long, dp, dp]
        L.or_cnn_forward_bf16act.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.or_bf16_round.argtypes = [ctypes.c_double]
        L.or_bf16_round.restype = ctypes.c_double
        L.or_cnn_nparam.argtypes = [ctypes.c_int]
        L.or_cnn_nparam.restype = ctypes.c_long
        L.or_cnn_forward.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.or_cnn_grad.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  dp, dp]
        L.or_auc.restype = ctypes.c_double
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def num_threads() -> int:
    return int(lib().or_num_threads())


def daub_filter(taps: int = 8) -> np.ndarray:
    h = np.zeros(taps)
    if lib().or_daub_filter(taps, _ptr(h, ctypes.c_double)) != 0:
        raise ValueError("taps must be even, 2..20")
    return h


def highpass(h: np.ndarray) -> np.ndarray:
    h = np.ascontiguousarray(h, dtype=np.float64)
    g = np.zeros_like(h)
    lib().or_highpass(_ptr(h, ctypes.c_double), len(h), _ptr(g, ctypes.c_double))
    return g


def dwt_step(x: np.ndarray, f: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((len(x) + 1) // 2)
    lib().or_dwt_step(_ptr(x, ctypes.c_double), len(x), _ptr(f, ctypes.c_double), len(f),
                      _ptr(out, ctypes.c_double))
    return out


def dwt_levels(L: int, level: int = -1):
    K = ctypes.c_int(0)
    J = lib().or_dwt_levels(L, level, ctypes.byref(K))
    return J, K.value


def dwt_full(x: np.ndarray, taps: int = 8, level: int = -1) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2 * len(x) + 64)
    n = lib().or_dwt_full(_ptr(x, ctypes.c_double), len(x), taps, level, _ptr(out, ctypes.c_double))
    return out[:n].copy()


def dwt_inverse(coef: np.ndarray, L: int, taps: int = 8, level: int = -1) -> np.ndarray:
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    x = np.zeros(L)
    lib().or_dwt_inverse(_ptr(coef, ctypes.c_double), L, taps, level, _ptr(x, ctypes.c_double))
    return x


def dwt_approx(cube: np.ndarray, taps: int = 8, level: int = -1, nthreads: int = 0) -> np.ndarray:
    """cube [..., L] float32 -> approximation matrix [..., K] float64 (Sec. 4)."""
    c = np.ascontiguousarray(cube, dtype=np.float32)
    L = c.shape[-1]
    P = c.size // L
    _, K = dwt_levels(L, level)
    out = np.zeros(P * K)
    lib().or_dwt_approx(_ptr(c, ctypes.c_float), P, L, taps, level, _ptr(out, ctypes.c_double), nthreads)
    return out.reshape(c.shape[:-1] + (K,))


def reflect(i: int, n: int) -> int:
    return int(lib().or_reflect(i, n))


def detect(cube: np.ndarray, detector: int, inner: int, outer: int, loading: float = 1e-3,
           border: int = 0, dwest_mode: int = 0, pixels=None, want_aux: bool = False,
           want_cond: bool = False, nthreads: int = 0):
    """Scores of LRX (0), DWRX (1) or DWEST (2) on cube [H][W][D] (any float dtype).

    pixels: None for the whole map, else an array of linear pixel indices.
    Returns the [H][W] map (pixels=None) or a vector; with want_aux also the
    per-pixel aux array (see oracle.c)."""
    c = np.ascontiguousarray(cube, dtype=np.float64)
    H, W, D = c.shape
    full = pixels is None
    pix = np.arange(H * W, dtype=np.int64) if full else np.ascontiguousarray(pixels, dtype=np.int64)
    score = np.zeros(len(pix))
    aux = np.zeros((len(pix), NAUX)) if want_aux else None
    rc = lib().or_detect(_ptr(c, ctypes.c_double), H, W, D, detector, inner, outer, loading, border,
                         dwest_mode, _ptr(pix, ctypes.c_int64), len(pix), _ptr(score, ctypes.c_double),
                         _ptr(aux, ctypes.c_double) if want_aux else None, int(want_cond), nthreads)
    if rc != 0:
        raise ValueError("bad detector arguments")
    if full:
        score = score.reshape(H, W)
        if want_aux:
            aux = aux.reshape(H, W, NAUX)
    return (score, aux) if want_aux else score


def window_moments(cube: np.ndarray, inner: int, outer: int, pixels, nthreads: int = 0):
    """Background mean [n, D] and covariance [n, D, D] (1/N) of the listed pixels (Sec. 2.1)."""
    c = np.ascontiguousarray(cube, dtype=np.float64)
    H, W, D = c.shape
    pix = np.ascontiguousarray(pixels, dtype=np.int64)
    mu = np.zeros((len(pix), D))
    cov = np.zeros((len(pix), D, D))
    if lib().or_window_moments(_ptr(c, ctypes.c_double), H, W, D, inner, outer, _ptr(pix, ctypes.c_int64), len(pix),
                               _ptr(mu, ctypes.c_double), _ptr(cov, ctypes.c_double), nthreads) != 0:
        raise ValueError("bad window")
    return mu, cov


def window_census(H: int, W: int, inner: int, outer: int, border: int = 0, pixels=None) -> np.ndarray:
    pix = np.arange(H * W, dtype=np.int64) if pixels is None else np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros((len(pix), 6), dtype=np.int64)
    if lib().or_window_census(H, W, inner, outer, border, _ptr(pix, ctypes.c_int64), len(pix),
                              _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("bad window")
    return out


def scene_whiten(x: np.ndarray):
    """Whitening of the network input: x [..., K] -> (mu [K], M [K][K]) with z = M (x - mu)."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    K = xx.shape[-1]
    P = xx.size // K
    mu = np.zeros(K)
    M = np.zeros((K, K))
    if lib().or_scene_whiten(K, _ptr(xx, ctypes.c_double), P, _ptr(mu, ctypes.c_double), _ptr(M, ctypes.c_double)):
        raise ValueError("scene_whiten: K in 1..8 and at least one pixel")
    return mu, M


def cnn_nparam(K: int = 4) -> int:
    return int(lib().or_cnn_nparam(K))


def cnn_forward(params: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Screening CNN forward (FP64): x [B][H][W][K] (normalised) -> [B][H][W]."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    B, H, W, K = xx.shape
    out = np.zeros((B, H, W))
    lib().or_cnn_forward(K, _ptr(p, ctypes.c_double), _ptr(xx, ctypes.c_double), B, H, W, _ptr(out, ctypes.c_double))
    return out


def cnn_forward_bf16act(params: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Screening CNN forward (FP64) with the inputs of the two 32 -> 32 layers rounded to
    bfloat16 (the tensor-core inference form)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    B, H, W, K = xx.shape
    out = np.zeros((B, H, W))
    lib().or_cnn_forward_bf16act(K, _ptr(p, ctypes.c_double), _ptr(xx, ctypes.c_double), B, H, W,
                                 _ptr(out, ctypes.c_double))
    return out


def bf16_round(v: float) -> float:
    return float(lib().or_bf16_round(float(v)))


def cnn_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray, edge: int = 7):
    """Loss (interior MSE) and its gradient with respect to every parameter (FP64)."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    B, H, W, K = xx.shape
    g = np.zeros_like(p)
    loss = ctypes.c_double(0.0)
    lib().or_cnn_grad(K, _ptr(p, ctypes.c_double), _ptr(xx, ctypes.c_double), _ptr(tt, ctypes.c_double), B, H, W, edge,
                      _ptr(g, ctypes.c_double), ctypes.byref(loss))
    return loss.value, g


def adaptive_threshold(score: np.ndarray, z: float):
    """Eq. 12 cut-off: (mu_d, sigma_d, tau, mask) over the finite entries of a score map."""
    s = np.ascontiguousarray(score, dtype=np.float64)
    mask = np.zeros(s.shape, dtype=np.uint8)
    mu, sd, tau = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_adaptive_threshold(_ptr(s, ctypes.c_double), s.size, float(z), ctypes.byref(mu), ctypes.byref(sd),
                                ctypes.byref(tau), _ptr(mask, ctypes.c_uint8))
    return mu.value, sd.value, tau.value, mask


def auc(score: np.ndarray, mask: np.ndarray) -> float:
    s = np.ascontiguousarray(score, dtype=np.float64).ravel()
    m = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    return float(lib().or_auc(_ptr(s, ctypes.c_double), _ptr(m, ctypes.c_uint8), len(s)))


def global_rx(cube: np.ndarray, loading: float = 1e-3, want_cond: bool = False):
    """Global RX, Eq. 1 (Sec. 2.1): s(r) = (r - mu)^T (C + delta I)^-1 (r - mu), with mu and
    C = (1/P) sum (x - mu)(x - mu)^T taken over all P pixels of the image (one background for
    the whole scene) and delta = loading * trace(C) / L, the loading rule of the local
    detectors.  cube [H][W][L] -> scores [H][W] float64; with want_cond also cond(C + delta I)."""
    c = np.asarray(cube, dtype=np.float64)
    L = c.shape[-1]
    X = c.reshape(-1, L)
    mu = X.mean(axis=0)
    Xc = X - mu
    C = Xc.T @ Xc / X.shape[0]
    delta = loading * np.trace(C) / L
    M = C + delta * np.eye(L)
    Z = np.linalg.solve(M, Xc.T)          # M^-1 (x - mu) for every pixel
    s = np.einsum("pl,lp->p", Xc, Z).reshape(c.shape[:-1])
    if want_cond:
        ev = np.linalg.eigvalsh(M)
        return s, float(ev[-1] / ev[0])
    return s
