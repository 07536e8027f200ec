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
    L.wdad_cnn_create.argtypes = [vp, i32, i32, ctypes.c_uint64, i64, ctypes.POINTER(vp)]
    L.wdad_cnn_destroy.argtypes = [vp]
    L.wdad_cnn_set_norm.argtypes = [vp, vp]
    L.wdad_cnn_params.argtypes = [vp, vp, ctypes.POINTER(i64)]
    L.wdad_cnn_set_params.argtypes = [vp, vp, i64]
    L.wdad_cnn_forward.argtypes = [vp, f32p, i32, i32, i32, f32p, vp]
    L.wdad_cnn_grad.argtypes = [vp, f32p, f32p, i32, i32, i32, vp, vp, vp]
    L.wdad_cnn_train.argtypes = [vp, f32p, f32p, i32, i32, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]
    L.wdad_cnn_save.argtypes = [vp, ctypes.c_char_p]
    L.wdad_cnn_load.argtypes = [vp, ctypes.c_char_p, i64, ctypes.POINTER(vp)]
    L.wdad_screen_run.argtypes = [vp, vp, f32p, i32, i32, i32, pp, ctypes.c_float, ctypes.c_float, ctypes.c_uint64,
                                  i32, i32, f32p, vp, vp, ctypes.POINTER(i64), vp]
    L.wdad_detect_all_noalloc.argtypes = [f32p, i32, i32, i32, pp, f32p, vp, vp]
    L.wdad_auc.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_double)]
    L.wdad_scene_whitening.argtypes = [vp, f32p, i64, i32, f32p, vp]
    L.wdad_adaptive_threshold.argtypes = [vp, f32p, i64, ctypes.c_double, vp, vp, vp]
    L.wdad_wavelet_filter.argtypes = [i32, vp]
    L.wdad_global_rx.argtypes = [vp, f32p, i32, i32, i32, i32, pp, f32p, vp]
    L.wdad_detect_windows.argtypes = [vp, f32p, i32, i32, i32, i32, i32, pp, f32p, vp, vp]
    L.wdad_detect_sequence.argtypes = [vp, i32, vp, i32, i32, i32, i32, pp, vp, vp, vp]
    for name in ("wdad_create", "wdad_destroy", "wdad_last_error_detail", "wdad_dwt_approx", "wdad_detect",
                 "wdad_detect_all", "wdad_detect_all_host", "wdad_window_census", "wdad_auc",
                 "wdad_detect_all_noalloc", "wdad_window_moments", "wdad_autotune", "wdad_batch_create",
                 "wdad_batch_launch", "wdad_batch_status", "wdad_batch_destroy", "wdad_batch_run",
                 "wdad_cnn_create", "wdad_cnn_destroy", "wdad_cnn_set_norm", "wdad_cnn_params",
                 "wdad_cnn_set_params", "wdad_cnn_forward", "wdad_cnn_grad", "wdad_cnn_train", "wdad_cnn_save",
                 "wdad_cnn_load", "wdad_screen_run", "wdad_scene_whitening", "wdad_adaptive_threshold",
                 "wdad_wavelet_filter", "wdad_global_rx", "wdad_detect_windows", "wdad_detect_sequence"):
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


def _check_out(t, shape, dtype, device, name="out"):
    """A caller-supplied buffer must be a contiguous CUDA tensor of exactly this shape and
    dtype on the cube's device: the kernels write shape's element count through its pointer."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == device and t.dtype == dtype
            and tuple(t.shape) == tuple(shape) and t.is_contiguous()):
        got = (tuple(t.shape), t.dtype, str(t.device), t.is_contiguous()) if isinstance(t, torch.Tensor) else type(t)
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)} on {device}; got {got}")
    return t


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


def wdad_wavelet_filter(taps: int = 8) -> np.ndarray:
    """The DWT's scaling filter (host computation, no GPU): float64 [taps]."""
    h = np.zeros(taps if taps > 0 else 1, dtype=np.float64)
    _check(lib().wdad_wavelet_filter(int(taps), h.ctypes.data), None)
    return h[:taps]


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
    _check_out(out, (H, W, K), torch.float32, cube.device)
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
    _check_out(out, (H, W), torch.float32, cube.device)
    if flags is not None:
        _check_out(flags, (H, W), torch.uint8, cube.device, "flags")
    h = handle(cube.device.index or 0)
    _check(lib().wdad_detect(h, cube.data_ptr(), H, W, L, int(detector), int(bool(reduce)), ctypes.byref(p),
                             out.data_ptr(), flags.data_ptr() if flags is not None else None, _stream(cube)), h)
    return out


def wdad_detect_windows(cube, params, reduce: bool = True, out=None, flags=None):
    """LRX, DWRX, DWEST at several windows in one call: [nwin, 3, H, W] float32.
    params: a list of wdad_params (same wavelet and level)."""
    import torch
    cube = _cube(cube)
    H, W, L = cube.shape
    n = len(params)
    arr = (wdad_params * n)(*params)
    if out is None:
        out = torch.empty((n, 3, H, W), device=cube.device, dtype=torch.float32)
    _check_out(out, (n, 3, H, W), torch.float32, cube.device)
    if flags is not None:
        _check_out(flags, (n, H, W), torch.uint8, cube.device, "flags")
    h = handle(cube.device.index or 0)
    _check(lib().wdad_detect_windows(h, cube.data_ptr(), H, W, L, int(bool(reduce)), n, arr, out.data_ptr(),
                                     flags.data_ptr() if flags is not None else None, _stream(cube)), h)
    return out


def wdad_global_rx(cube, reduce: bool = True, params: wdad_params | None = None, out=None, **over):
    """Global RX (Eq. 1, image-wide mean and covariance) on every pixel: [H, W] float32."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((H, W), device=cube.device, dtype=torch.float32)
    _check_out(out, (H, W), torch.float32, cube.device)
    h = handle(cube.device.index or 0)
    _check(lib().wdad_global_rx(h, cube.data_ptr(), H, W, L, int(bool(reduce)), ctypes.byref(p), out.data_ptr(),
                                _stream(cube)), h)
    return out


def wdad_detect_all(cube, reduce: bool = True, params: wdad_params | None = None, out=None, flags=None, **over):
    """LRX, DWRX, DWEST in one pass: [3, H, W] float32."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    if out is None:
        out = torch.empty((3, H, W), device=cube.device, dtype=torch.float32)
    _check_out(out, (3, H, W), torch.float32, cube.device)
    if flags is not None:
        _check_out(flags, (H, W), torch.uint8, cube.device, "flags")
    h = handle(cube.device.index or 0)
    _check(lib().wdad_detect_all(h, cube.data_ptr(), H, W, L, int(bool(reduce)), ctypes.byref(p), out.data_ptr(),
                                 flags.data_ptr() if flags is not None else None, _stream(cube)), h)
    return out


def wdad_detect_sequence(cubes, params, outs=None, events=None):
    """All three detectors at several windows on each cube of a sequence (reduced path), the
    DWT of each cube overlapping the previous cube's detectors: a list of [nwin, 3, H, W]
    float32 tensors, one per cube, equal to wdad_detect_windows(cube, params) bit for bit.
    cubes: device tensors [H, W, L] of one shape; outs: optional list of result tensors
    (entries may repeat); events: optional list of 4 n torch.cuda.Event or None (per cube:
    DWT start, DWT end on the library's stream; detector start, end on torch's current
    stream)."""
    import torch
    cubes = [_cube(c) for c in cubes]
    n = len(cubes)
    plist = list(params)
    nwin = len(plist)
    arr = (wdad_params * nwin)(*plist)
    if n == 0:
        return []
    H, W, L = cubes[0].shape
    dev = cubes[0].device
    for c in cubes:
        if tuple(c.shape) != (H, W, L) or c.device != dev:
            raise ValueError("all cubes of a sequence share one shape and device")
    if outs is None:
        outs = [torch.empty((nwin, 3, H, W), device=dev, dtype=torch.float32) for _ in range(n)]
    if len(outs) != n:
        raise ValueError(f"outs must hold {n} tensors")
    for o in outs:
        _check_out(o, (nwin, 3, H, W), torch.float32, dev)
    cp = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cubes])
    op = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    ep = None
    if events is not None:
        if len(events) != 4 * n:
            raise ValueError(f"events must hold {4 * n} torch.cuda.Event")
        stream = torch.cuda.current_stream(dev)
        for e in events:
            if e is not None and not e.cuda_event:  # torch creates the CUDA event on its first record
                e.record(stream)
        ep = (ctypes.c_void_p * (4 * n))(*[e.cuda_event if e is not None else None for e in events])
    h = handle(dev.index or 0)
    _check(lib().wdad_detect_sequence(h, n, cp, H, W, L, nwin, arr, op, ep, _stream(cubes[0])), h)
    return outs


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
    if not (isinstance(out, torch.Tensor) and not out.is_cuda and out.dtype == torch.float32
            and tuple(out.shape) == (n, 3, H, W) and out.is_contiguous()):
        raise ValueError(f"out must be a contiguous CPU float32 tensor of shape {(n, 3, H, W)}")
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
    _check_out(out, (3, H, W), torch.float32, cube.device)
    if flags is not None:
        _check_out(flags, (H, W), torch.uint8, cube.device, "flags")
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
        import torch
        _check_out(j["scores"], (3, H, W) if int(j["detector"]) == 3 else (H, W), torch.float32, cube.device, "scores")
        if j.get("flags") is not None:
            _check_out(j["flags"], (H, W), torch.uint8, cube.device, "flags")
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


class wdad_cnn:
    """A9 screening network (K -> 32 -> 32 -> 32 -> 1, receptive field 15)."""

    def __init__(self, K: int = 4, bf16_weights: bool = True, seed: int = 0, max_batch_pixels: int = 1 << 16,
                 device: int = 0, _ptr=None):
        self.device = device
        self._h = handle(device)
        if _ptr is None:
            c = ctypes.c_void_p()
            _check(lib().wdad_cnn_create(self._h, K, int(bool(bf16_weights)), seed, max_batch_pixels, ctypes.byref(c)),
                   self._h)
            self._c = c.value
        else:
            self._c = _ptr
        self.K = K

    @classmethod
    def load(cls, path: str, max_batch_pixels: int = 1 << 16, device: int = 0):
        h = handle(device)
        c = ctypes.c_void_p()
        _check(lib().wdad_cnn_load(h, path.encode(), max_batch_pixels, ctypes.byref(c)), h)
        obj = cls.__new__(cls)
        obj.device, obj._h, obj._c = device, h, c.value
        obj.K = 0
        return obj

    def _stream(self):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def set_norm(self, mu_M=None):
        """Fixed input map [mu (K), M (K x K)] with z = M (x - mu); None: whiten each scene."""
        if mu_M is None:
            _check(lib().wdad_cnn_set_norm(self._c, None), self._h)
            return
        a = np.ascontiguousarray(mu_M, dtype=np.float32).ravel()
        _check(lib().wdad_cnn_set_norm(self._c, a.ctypes.data), self._h)

    def params(self) -> np.ndarray:
        n = ctypes.c_int64(0)
        _check(lib().wdad_cnn_params(self._c, None, ctypes.byref(n)), self._h)
        out = np.zeros(n.value, dtype=np.float32)
        _check(lib().wdad_cnn_params(self._c, out.ctypes.data, ctypes.byref(n)), self._h)
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().wdad_cnn_set_params(self._c, a.ctypes.data, a.size), self._h)

    def forward(self, x, out=None):
        """x: CUDA [B, H, W, K] raw approximation values -> [B, H, W]."""
        import torch
        x = x.contiguous()
        B, H, W, _ = x.shape
        if out is None:
            out = torch.empty((B, H, W), device=x.device, dtype=torch.float32)
        _check_out(out, (B, H, W), torch.float32, x.device)
        _check(lib().wdad_cnn_forward(self._c, x.data_ptr(), B, H, W, out.data_ptr(), self._stream()), self._h)
        return out

    def grad(self, x, t):
        """Interior-MSE loss and gradient (host) for mapped input z [B, H, W, K], targets [B, H, W]."""
        x = x.contiguous()
        t = t.contiguous()
        B, H, W, _ = x.shape
        n = ctypes.c_int64(0)
        lib().wdad_cnn_params(self._c, None, ctypes.byref(n))
        g = np.zeros(n.value, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().wdad_cnn_grad(self._c, x.data_ptr(), t.data_ptr(), B, H, W, g.ctypes.data, ctypes.byref(loss),
                                   self._stream()), self._h)
        return loss.value, g

    def train(self, approx, score, steps: int, batch: int = 8, crop: int = 32, lr: float = 1e-3, seed: int = 0):
        """`steps` Adam steps on random crops of one reduced cube approx [H, W, K] and its score map [H, W]."""
        approx = approx.contiguous()
        score = score.contiguous()
        H, W, _ = approx.shape
        loss = ctypes.c_float(0.0)
        _check(lib().wdad_cnn_train(self._c, approx.data_ptr(), score.data_ptr(), H, W, steps, batch, crop, lr, seed,
                                    ctypes.byref(loss), self._stream()), self._h)
        return loss.value

    def save(self, path: str):
        _check(lib().wdad_cnn_save(self._c, path.encode()), self._h)

    def close(self):
        if getattr(self, "_c", None):
            lib().wdad_cnn_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wdad_screen_run(net: "wdad_cnn", cube, top_frac: float = 0.02, audit_frac: float = 0.005, seed: int = 0,
                    tile_rows: int = 256, exact_reduce: bool = False, params: wdad_params | None = None,
                    want_pred: bool = True, **over):
    """A9 screened LRX: (score [H, W] with -inf where not evaluated, pred, selected, n_selected)."""
    import torch
    cube = _cube(cube)
    p = _params(params, over)
    H, W, L = cube.shape
    score = torch.empty((H, W), device=cube.device, dtype=torch.float32)
    pred = torch.empty((H, W), device=cube.device, dtype=torch.float32) if want_pred else None
    sel = torch.empty((H, W), device=cube.device, dtype=torch.uint8)
    n = ctypes.c_int64(0)
    h = handle(cube.device.index or 0)
    _check(lib().wdad_screen_run(h, net._c, cube.data_ptr(), H, W, L, ctypes.byref(p), top_frac, audit_frac, seed,
                                 tile_rows, int(bool(exact_reduce)), score.data_ptr(),
                                 pred.data_ptr() if pred is not None else None, sel.data_ptr(), ctypes.byref(n),
                                 _stream(cube)), h)
    return score, pred, sel, n.value


def wdad_scene_whitening(x):
    """[mu (K), M (K x K) row-major] of the scene whitening of x [..., K] (CUDA tensor)."""
    import torch
    x = x.contiguous()
    K = x.shape[-1]
    P = x.numel() // K
    out = torch.empty(K + K * K, device=x.device, dtype=torch.float32)
    h = handle(x.device.index or 0)
    _check(lib().wdad_scene_whitening(h, x.data_ptr(), P, K, out.data_ptr(), _stream(x)), h)
    return out


def wdad_window_census(H: int, W: int, params: wdad_params | None = None, device: int = 0, **over):
    """A2 integer census [H, W, 6] int64 from the detectors' own tile loader and box sums."""
    import torch
    p = _params(params, over)
    out = torch.empty((H, W, 6), device=f"cuda:{device}", dtype=torch.int64)
    h = handle(device)
    _check(lib().wdad_window_census(h, H, W, ctypes.byref(p), out.data_ptr(), _stream(out)), h)
    return out


def wdad_adaptive_threshold(score, z_alpha: float, mask=None, want_mask: bool = True, want_stats: bool = True):
    """Eq. 12 cut-off of a CUDA score map: (mu_d, sigma_d, tau, count, mask uint8 or None).
    want_stats=False leaves the call asynchronous (no host statistics; the four are NaN, -1)."""
    import torch
    score = score.contiguous()
    n = score.numel()
    if want_mask and mask is None:
        mask = torch.empty(score.shape, device=score.device, dtype=torch.uint8)
    if mask is not None:
        _check_out(mask, score.shape, torch.uint8, score.device, "mask")
    stats = np.zeros(4, dtype=np.float64)
    h = handle(score.device.index or 0)
    _check(lib().wdad_adaptive_threshold(h, score.data_ptr() if n else None, n, float(z_alpha),
                                         mask.data_ptr() if (mask is not None and n) else None,
                                         stats.ctypes.data if want_stats else None, _stream(score)), h)
    if not want_stats:
        return float("nan"), float("nan"), float("nan"), -1, mask
    return float(stats[0]), float(stats[1]), float(stats[2]), int(stats[3]), mask


def wdad_auc(score, mask) -> float:
    """Pixel-level ROC AUC (host arrays)."""
    s = np.ascontiguousarray(np.asarray(score, dtype=np.float32)).ravel()
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8)).ravel()
    out = ctypes.c_double(0.0)
    _check(lib().wdad_auc(s.ctypes.data, m.ctypes.data, s.size, ctypes.byref(out)), None)
    return float(out.value)
