"""Python binding of libwdad (include/wdad.h): argument marshalling only.

Functions carry the C entry points' names.  Tensors are torch CUDA tensors
(contiguous float32 cubes [H, W, L]); calls run on torch's current stream of the
tensor's device.  Every computation happens in the library's CUDA kernels: if
libwdad.so is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libwdad.so")

WDAD_OK, WDAD_ERR_ARG, WDAD_ERR_CUDA, WDAD_ERR_NOMEM, WDAD_ERR_NUMERIC, WDAD_ERR_TIMEOUT, WDAD_ERR_UNSUPPORTED = range(7)
WDAD_LRX, WDAD_DWRX, WDAD_DWEST = 0, 1, 2
WDAD_PREC_FP32, WDAD_PREC_MIXED, WDAD_PREC_FP64 = 0, 1, 2
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOMEM", 4: "ERR_NUMERIC", 5: "ERR_TIMEOUT",
           6: "ERR_UNSUPPORTED"}


class WdadError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"wdad {_STATUS.get(status, status)}: {detail}")
        self.status = status


class wdad_params(ctypes.Structure):
    _fields_ = [("wavelet_taps", ctypes.c_int), ("level", ctypes.c_int), ("inner", ctypes.c_int),
                ("outer", ctypes.c_int), ("loading", ctypes.c_float), ("cond_gate", ctypes.c_float),
                ("border", ctypes.c_int), ("dwest_mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("dwest_tau", ctypes.c_float)]


class wdad_job(ctypes.Structure):
    _fields_ = [("cube", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("L", ctypes.c_int),
                ("detector", ctypes.c_int), ("params", wdad_params), ("scores", ctypes.c_void_p),
                ("flags", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_handles: dict = {}


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise RuntimeError(f"{_SO} is missing: build it with paper_1201_2025_gb300.build.build()")
    L = ctypes.CDLL(_SO)
    vp, i32, i64, f32p = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    pp = ctypes.POINTER(wdad_params)
    L.wdad_default_params.argtypes = [pp]
    L.wdad_default_params.restype = None
    L.wdad_create.argtypes = [ctypes.POINTER(vp), i32]
    L.wdad_destroy.argtypes = [vp]
    L.wdad_last_error_detail.argtypes = [vp, ctypes.c_char_p, i32]
    L.wdad_query_K.argtypes = [i32, i32, i32]
    L.wdad_dwt_approx.argtypes = [vp, f32p, i32, i32, i32, pp, f32p, ctypes.POINTER(i32), vp]
    L.wdad_detect.argtypes = [vp, f32p, i32, i32, i32, i32, i32, pp, f32p, vp, vp]
    L.wdad_detect_all.argtypes = [vp, f32p, i32, i32, i32, i32, pp, f32p, vp, vp]
    L.wdad_detect_all_host.argtypes = [vp, vp, i32, i32, i32, i32, i32, pp, vp, vp]
    L.wdad_window_census.argtypes = [vp, i32, i32, pp, vp, vp]
    L.wdad_window_moments.argtypes = [vp, f32p, i32, i32, i32, vp, i64, pp, f32p, f32p, vp]
    jp = ctypes.POINTER(wdad_job)
    L.wdad_autotune.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32), vp]
    L.wdad_batch_create.argtypes = [vp, i32, jp, i32, i32, ctypes.POINTER(vp), vp]
    L.wdad_batch_launch.argtypes = [vp, vp]
    L.wdad_batch_status.argtypes = [vp, ctypes.POINTER(i32)]
    L.wdad_batch_destroy.argtypes = [vp]
    L.wdad_batch_run.argtypes = [vp, i32, jp, vp]
    L.wdad_detect_all_noalloc.argtypes = [f32p, i32, i32, i32, pp, f32p, vp, vp]
    L.wdad_auc.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_double)]
    for name in ("wdad_create", "wdad_destroy", "wdad_last_error_detail", "wdad_dwt_approx", "wdad_detect",
                 "wdad_detect_all", "wdad_detect_all_host", "wdad_window_census", "wdad_auc",
                 "wdad_detect_all_noalloc", "wdad_window_moments", "wdad_autotune", "wdad_batch_create",
                 "wdad_batch_launch", "wdad_batch_status", "wdad_batch_destroy", "wdad_batch_run"):
        getattr(L, name).restype = i32
    L.wdad_query_K.restype = i32
    _lib = L
    return L


def wdad_default_params(**over) -> wdad_params:
    p = wdad_params()
    lib().wdad_default_params(ctypes.byref(p))
    for k, v in over.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def handle(device: int = 0) -> int:
    """Per-process, per-device handle (created on first use)."""
    with _lock:
        h = _handles.get(device)
        if h is None:
            hv = ctypes.c_void_p()
            st = lib().wdad_create(ctypes.byref(hv), device)
            if st != WDAD_OK:
                raise WdadError(st, f"wdad_create(device={device})")
            h = _handles[device] = hv.value
        return h


def _check(st: int, h) -> None:
    if st != WDAD_OK:
        buf = ctypes.create_string_buffer(512)
        if h:
            lib().wdad_last_error_detail(h, buf, 512)
        raise WdadError(st, buf.value.decode(errors="replace"))


def _stream(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _cube(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 3):
        raise TypeError("cube must be a CUDA float32 tensor [H, W, L]")
    return t.contiguous()


def _params(params, over):
    if params is None:
        return wdad_default_params(**over)
    if over:
        p = wdad_params.from_buffer_copy(params)
        for k, v in over.items():
            setattr(p, k, v)
        return p
    return params


def wdad_query_K(L: int, taps: int = 8, level: int = -1) -> int:
    return int(lib().wdad_query_K(L, taps, level))


def wdad_dwt_approx(cube, params: wdad_params | None = None, out=None, **over):
    """A1: approximation matrix [H, W, K] of a CUDA cube [H, W, L]."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    K = wdad_query_K(L, p.wavelet_taps, p.level)
    if K < 1:
        raise WdadError(WDAD_ERR_ARG, "bad L/taps/level")
    if out is None:
        out = torch.empty((H, W, K), device=cube.device, dtype=torch.float32)
    h = handle(cube.device.index or 0)
    k = ctypes.c_int(0)
    _check(lib().wdad_dwt_approx(h, cube.data_ptr(), H, W, L, ctypes.byref(p), out.data_ptr(), ctypes.byref(k),
                                 _stream(cube)), h)
    return out


def wdad_detect(cube, detector: int, reduce: bool = True, params: wdad_params | None = None, out=None,
                flags=None, **over):
    """One detector on every pixel: [H, W] float32 score map (and the flags map if given)."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((H, W), device=cube.device, dtype=torch.float32)
    h = handle(cube.device.index or 0)
    _check(lib().wdad_detect(h, cube.data_ptr(), H, W, L, int(detector), int(bool(reduce)), ctypes.byref(p),
                             out.data_ptr(), flags.data_ptr() if flags is not None else None, _stream(cube)), h)
    return out


def wdad_detect_all(cube, reduce: bool = True, params: wdad_params | None = None, out=None, flags=None, **over):
    """LRX, DWRX, DWEST in one pass: [3, H, W] float32."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((3, H, W), device=cube.device, dtype=torch.float32)
    h = handle(cube.device.index or 0)
    _check(lib().wdad_detect_all(h, cube.data_ptr(), H, W, L, int(bool(reduce)), ctypes.byref(p), out.data_ptr(),
                                 flags.data_ptr() if flags is not None else None, _stream(cube)), h)
    return out


def wdad_detect_all_host(cube, reduce: bool = True, params=None, out=None, device: int = 0, **over):
    """Host-memory variant: cube is a CPU float32 tensor (pinned for asynchronous copies)
    [H, W, L]; params a list of wdad_params (one per window pair).  Returns the host
    tensor [nwin, 3, H, W].  Runs on torch's current stream of `device`; the call
    returns once the work is enqueued, synchronise before reading the result."""
    import torch
    if not (isinstance(cube, torch.Tensor) and not cube.is_cuda and cube.dtype == torch.float32 and cube.dim() == 3):
        raise TypeError("cube must be a CPU float32 tensor [H, W, L]")
    cube = cube.contiguous()
    plist = list(params) if params is not None else [_params(None, over)]
    n = len(plist)
    arr = (wdad_params * n)(*plist)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((n, 3, H, W), dtype=torch.float32).pin_memory()
    h = handle(device)
    st = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    _check(lib().wdad_detect_all_host(h, cube.data_ptr(), H, W, L, int(bool(reduce)), n, arr, out.data_ptr(), st), h)
    return out


def wdad_detect_all_noalloc(cube, params: wdad_params | None = None, out=None, flags=None, **over):
    """Reduced LRX, DWRX, DWEST pass [3, H, W] with no device allocation inside the
    library (for callers that cannot call cudaMalloc; limits and sharing rules in
    include/wdad.h).  `out` may be given to avoid the allocation of the result here."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((3, H, W), device=cube.device, dtype=torch.float32)
    with torch.cuda.device(cube.device):
        st = lib().wdad_detect_all_noalloc(cube.data_ptr(), H, W, L, ctypes.byref(p), out.data_ptr(),
                                           flags.data_ptr() if flags is not None else None, _stream(cube))
    if st != WDAD_OK:
        raise WdadError(st, "wdad_detect_all_noalloc")
    return out


def wdad_window_moments(cube, pixels, params: wdad_params | None = None, **over):
    """A3: background mean [npix, L] and covariance [npix, L, L] of the listed pixels."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    pix = torch.as_tensor(pixels, dtype=torch.int64).to(cube.device).contiguous()
    n = pix.numel()
    mu = torch.empty((n, L), device=cube.device, dtype=torch.float32)
    cov = torch.empty((n, L, L), device=cube.device, dtype=torch.float32)
    h = handle(cube.device.index or 0)
    _check(lib().wdad_window_moments(h, cube.data_ptr(), H, W, L, pix.data_ptr(), n, ctypes.byref(p), mu.data_ptr(),
                                     cov.data_ptr(), _stream(cube)), h)
    return mu, cov


def wdad_autotune(D: int, inner: int, outer: int, device: int = 0) -> int:
    """Tile height the autotuner picks for D bands and an (inner, outer) window."""
    import torch
    h = handle(device)
    th = ctypes.c_int(0)
    _check(lib().wdad_autotune(h, D, inner, outer, ctypes.byref(th),
                               ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)), h)
    return th.value


def _jobs(jobs):
    arr = (wdad_job * len(jobs))()
    for i, j in enumerate(jobs):
        cube = _cube(j["cube"])
        H, W, L = cube.shape
        p = j.get("params") or wdad_default_params(**j.get("over", {}))
        arr[i] = wdad_job(cube.data_ptr(), H, W, L, int(j["detector"]), p, j["scores"].data_ptr(),
                          j["flags"].data_ptr() if j.get("flags") is not None else None)
    return arr


class wdad_batch:
    """A8: many reduced-path jobs in one persistent launch (optionally one CUDA graph).
    jobs: list of dicts {cube: CUDA [H,W,L], detector: 0..3, scores: CUDA [H,W] or [3,H,W],
    params or over: wdad_params fields, flags: optional CUDA uint8 [H,W]}."""

    def __init__(self, jobs, autotune: bool = True, use_graph: bool = True, device: int = 0):
        import torch
        self.device = device
        self._keep = list(jobs)
        self._arr = _jobs(jobs)
        self._h = handle(device)
        b = ctypes.c_void_p()
        st = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        _check(lib().wdad_batch_create(self._h, len(jobs), self._arr, int(autotune), int(use_graph), ctypes.byref(b),
                                       st), self._h)
        self._b = b.value
        self.n = len(jobs)

    def launch(self):
        import torch
        _check(lib().wdad_batch_launch(self._b, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)),
               self._h)

    def status(self):
        """Synchronise; returns (wdad status code, per-job tile heights)."""
        ths = (ctypes.c_int * self.n)()
        st = lib().wdad_batch_status(self._b, ths)
        return st, list(ths)

    def close(self):
        if self._b:
            lib().wdad_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wdad_batch_run(jobs, device: int = 0):
    import torch
    arr = _jobs(jobs)
    h = handle(device)
    _check(lib().wdad_batch_run(h, len(jobs), arr, ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)), h)


def wdad_window_census(H: int, W: int, params: wdad_params | None = None, device: int = 0, **over):
    """A2 integer census [H, W, 6] int64 from the detectors' own tile loader and box sums."""
    import torch
    p = _params(params, over)
    out = torch.empty((H, W, 6), device=f"cuda:{device}", dtype=torch.int64)
    h = handle(device)
    _check(lib().wdad_window_census(h, H, W, ctypes.byref(p), out.data_ptr(), _stream(out)), h)
    return out


def wdad_auc(score, mask) -> float:
    """Pixel-level ROC AUC (host arrays)."""
    s = np.ascontiguousarray(np.asarray(score, dtype=np.float32)).ravel()
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8)).ravel()
    out = ctypes.c_double(0.0)
    _check(lib().wdad_auc(s.ctypes.data, m.ctypes.data, s.size, ctypes.byref(out)), None)
    return float(out.value)
