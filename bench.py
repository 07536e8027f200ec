"""Benchmark of the DWT-reduced anomaly-detection path on GB300.

Workload: one 512x512x224 float32 AVIRIS-shaped synthetic cube (200 implanted
targets of 1-3 px at abundance 0.1-0.5), windows (3,9), (5,15) and (7,21).
A step = one db4 DWT of the cube (approximation matrix, K = 4) followed by the
fused LRX + DWRX + DWEST pass at the three window pairs (one launch whose grid holds
the tiles of all three windows): 9 score maps.
The timed steps are one wdad_detect_sequence call over the cube K times: the DWT of
the next step (HBM-bound, on the library's own stream and part of the SMs) overlaps the
issue-bound detector launch of the current one, through two approximation buffers.
value = 3 * H * W / step time (pixel-window evaluations per second, each with all
three detectors; the DWT is counted once per cube).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (each rank its own cube; no collective
on the data path), so scaling is weak and value sums over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 512
L = 224
WINDOWS = [(3, 9), (5, 15), (7, 21)]
WORKLOAD = "512x512x224 f32 cube, db4 DWT to K=4, LRX+DWRX+DWEST at windows (3,9),(5,15),(7,21)"
METRIC = "Mpixel/s per detector: full-band vs DWT-reduced vs mixed/learned; % roofline"
UNIT = "Mpixel/s"
BYTES_DWT_PER_PX = L * 4 + 4 * 4  # algorithmic: read the spectrum, write K=4 coefficients
# Algorithmic FP32 operations per pixel of the fused three-detector pass on K=4 bands:
# 10 channel products, 112 box-sum updates (14 channels x outer/inner x horizontal/vertical x
# enter/leave), 62 for the moments, 80 for LRX+DWRX (loading, 4x4 Cholesky, two solves),
# 780 for DWEST (C_diff, three Jacobi sweeps of six rotations, selection and projection).
FLOPS_DETECT_PER_PX = 10 + 112 + 62 + 80 + 780
# FP32 peak: 152 SMs x 128 lanes x 2 flops (FMA) at the clock sampled during the run
FP32_LANES = 152 * 128 * 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Sustained dense BF16 tensor rate (TFLOP/s) for kernels timed inside a longer run."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


def fullband_ceiling_flops(L: int, inner: int, outer: int, detectors: str):
    """Definitional work per pixel of the full-band detectors (the window Gram on the tensor
    cores, the factorisations on FP32 SIMT): (tensor flops, SIMT flops).
    LRX/DWRX: background Gram 2 N L^2, Cholesky L^3 / 3 and two triangular solves 2 L^2.
    DWEST adds the inner Gram 2 n_i L^2 and a symmetric eigen-decomposition, about 9 L^3."""
    N = outer * outer - inner * inner
    ni = inner * inner
    tc = 2.0 * N * L * L
    simt = L ** 3 / 3.0 + 2.0 * L * L
    if detectors == "all3":
        tc += 2.0 * ni * L * L
        simt += 9.0 * L ** 3
    return tc, simt


def fullband_roofline(L, inner, outer, detectors, mpx_s, tc_peak_tflops, fp32_peak_tflops):
    """Fraction of the full-band ceiling: ceiling time per pixel (Gram at the tensor rate plus
    the factorisation at the FP32 SIMT rate) over the measured time per pixel."""
    tc, simt = fullband_ceiling_flops(L, inner, outer, detectors)
    t_ceiling = tc / (tc_peak_tflops * 1e12) + simt / (fp32_peak_tflops * 1e12)
    t_meas = 1.0 / (mpx_s * 1e6)
    return {"ceiling_Mpixel_s": 1e-6 / t_ceiling, "achieved_Mpixel_s": mpx_s, "frac": t_ceiling / t_meas,
            "tensor_flops_per_px": tc, "simt_flops_per_px": simt}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        self.start_n = len(self.lines)

    def __exit__(self, *a):
        time.sleep(0.1)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [l.split(", ") for l in self.lines[getattr(self, "start_n", 0):] if l.count(",") >= 8]
        if not rows:
            rows = [l.split(", ") for l in self.lines if l.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _config(ws: int) -> dict:
    """The workload both arms report (the reference arm times a row sample of it, stated in its
    cpu_baseline)."""
    return {"workload": WORKLOAD, "H": H, "W": W, "L": L, "windows": WINDOWS, "path": "DWT-reduced",
            "l2": "inputs larger than L2 (235 MB cube vs 129 MB L2)", "parallelism": f"replicas x{ws}"}


def max_over_ranks(v: float, ws: int, device=None) -> float:
    """The largest of one float per rank (the slowest rank's time); v itself for one rank.
    device: where the collective's tensor lives (the rank's GPU under NCCL, CPU under gloo)."""
    if ws <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes its own cube, 3 windows per step."""
    return ws * 3 * H * W / (ms_per_step * 1e-3) / 1e6


def cpu_oracle_sample(cube: np.ndarray, rows: int, min_seconds: float = 0.0):
    """Time the FP64 oracle (as it stands) on the first `rows` rows of the cube: DWT
    plus the three detectors at the three windows, repeated until min_seconds have
    passed.  Returns (pixel-windows/s, seconds, repetitions)."""
    import oracle
    sub = np.ascontiguousarray(cube[:rows])
    t0 = time.perf_counter()
    reps = 0
    while True:
        a = oracle.dwt_approx(sub)
        for wi, wo in WINDOWS:
            for det in range(3):
                oracle.detect(a, det, wi, wo)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_seconds:
            break
    return reps * 3 * sub.shape[0] * sub.shape[1] / dt, dt, reps


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1201_2025_gb300 import synth
    sc = synth.scene_512x512(0)
    rows = args.ref_rows
    for _ in range(args.warmup):
        cpu_oracle_sample(sc.cube, rows)
    times = []
    for _ in range(args.steps):
        _, dt, _ = cpu_oracle_sample(sc.cube, rows)
        times.append(dt)
    per_step = sum(times) / len(times)
    v = 3 * rows * W / per_step / 1e6
    cores = oracle.num_threads()
    sample = f"rows 0..{rows - 1} of the 512x512 cube ({rows * W} px) per step, all 3 windows x 3 detectors"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(1),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _timer(stream):
    import torch

    def _time(fn, n=10, warm=2):
        for _ in range(warm):
            fn()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / n
    return _time


def bench_batching(dev, stream, peak, side_lo=128, side_hi=1024):
    """64 cubes of uneven size (side U{side_lo..side_hi}), band count (128/188/224), window and
    detector in one persistent graph-captured launch, against the same jobs run one after
    another through the single-cube entry points (DWT + detector each)."""
    import torch
    from paper_1201_2025_gb300 import synth, wdad
    _time = _timer(stream)
    specs = synth.batch_specs(64, seed=0, side_lo=side_lo, side_hi=side_hi)
    jobs, nbytes, npx = [], 0, 0
    for sp in specs:
        Hh, Ww, Ll = sp["H"], sp["W"], sp["L"]
        cube, _ = synth.make_scene_device(Hh, Ww, Ll, seed=sp["seed"], n_anom=max(1, Hh * Ww // 1300),
                                          anom_side=(1, 3), abundance=(0.1, 0.5), margin=10, device=dev)
        K = wdad.wdad_query_K(Ll)
        jobs.append(dict(cube=cube, detector=sp["detector"], scores=torch.empty((Hh, Ww), device=dev),
                         over=dict(inner=sp["inner"], outer=sp["outer"])))
        npx += Hh * Ww
        nbytes += Hh * Ww * (4 * Ll + 4 * K + 4 * K + 4)  # DWT read + write, detector read + score write
    torch.cuda.synchronize()
    res = {"jobs": len(jobs), "pixels": npx, "cube_GB": sum(j["cube"].numel() * 4 for j in jobs) / 1e9,
           "workload": f"64 cubes, side U{{{side_lo}..{side_hi}}}, L in {{128,188,224}}, windows (3,9)/(5,15)/(7,21), "
                       "one detector each (LRX/DWRX/DWEST), f32, device-generated (same recipe)"}
    batched = None
    for name, tuned in (("default_plans", False), ("autotuned", True)):
        b = wdad.wdad_batch(jobs, autotune=tuned, use_graph=True)
        ms = _time(b.launch, n=5)
        st, ths = b.status()
        if not tuned:
            batched = [j["scores"].clone() for j in jobs]
        res[name] = {"graph_ms": ms, "Mpixel_s": npx / (ms * 1e-3) / 1e6, "status": st,
                     "algorithmic_GBps": nbytes / (ms * 1e-3) / 1e9, "frac_of_hbm": nbytes / (ms * 1e-3) / 1e9 / peak,
                     "tile_heights": {str(t): ths.count(t) for t in sorted(set(ths))}}
        b.close()

    def seq():
        for j in jobs:
            wdad.wdad_detect(j["cube"], j["detector"], reduce=True, out=j["scores"], **j["over"])
    ms = _time(seq, n=2)
    res["sequential"] = {"ms": ms, "Mpixel_s": npx / (ms * 1e-3) / 1e6,
                         "algorithmic_GBps": nbytes / (ms * 1e-3) / 1e9}
    res["speedup_graph_vs_sequential"] = ms / res["default_plans"]["graph_ms"]
    # the default-plan batch must give the single-cube entry points' scores bit for bit
    res["default_plans"]["bit_identical_to_sequential"] = all(torch.equal(a, j["scores"]) for a, j in zip(batched, jobs))
    del jobs, batched
    torch.cuda.empty_cache()
    return res


def bench_screening(dev, stream, n_train: int, train_steps: int):
    """Learned screening on a 2048x2048x224 cube in 256-row tiles; exact LRX on the top 2% +
    0.5% audit; recall of implanted anomalies against the exact full-map LRX.  Two networks,
    each trained on the DWT-LRX (5,15) scores of n_train seeded 256x256 cubes: one on the db4
    approximation at the automatic level (K = 4) screening for the exact DWT-LRX, one on the
    approximation at level 5 (K = 7) screening for the exact full-band LRX (the four-coefficient
    input cannot see part of what the full band separates)."""
    import torch
    from paper_1201_2025_gb300 import synth, wdad
    _time = _timer(stream)
    levels = {"dwt_lrx": -1, "fullband_lrx": 5}
    t0 = time.perf_counter()
    data = {k: [] for k in levels}
    for s in range(n_train):
        c, _ = synth.make_scene_device(256, 256, L, seed=10000 + s, n_anom=50, anom_side=(1, 3),
                                       abundance=(0.1, 0.5), margin=4, device=dev)
        for name, lev in levels.items():
            ap = wdad.wdad_dwt_approx(c, level=lev)
            data[name].append((ap, wdad.wdad_detect(ap, 0, reduce=False, inner=5, outer=15)))
        del c
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    per_call = 5
    calls = max(1, train_steps // per_call)
    nets, train_s = {}, {}
    for name in levels:
        K = data[name][0][0].shape[-1]
        net = wdad.wdad_cnn(K=K, bf16_weights=True, seed=11, max_batch_pixels=8 * 32 * 32)
        t0 = time.perf_counter()
        for it in range(calls):
            ap, lrx = data[name][it % len(data[name])]
            net.train(ap, lrx, steps=per_call, batch=8, crop=32, lr=2e-3 if it < 0.7 * calls else 1e-3, seed=100 + it)
        torch.cuda.synchronize()
        train_s[name] = time.perf_counter() - t0
        nets[name] = net
    del data
    HS = 2048
    cube, mask = synth.make_scene_device(HS, HS, L, seed=4242, n_anom=3200, anom_side=(1, 3), abundance=(0.1, 0.5),
                                         margin=10, device=dev)
    P = HS * HS
    out = {"workload": f"{HS}x{HS}x{L} f32 cube, 3200 targets (1-3 px, f 0.1-0.5), 256-row tiles, window (5,15), "
                       f"top 2% + 0.5% audit; CNNs trained on {n_train} seeded 256x256 cubes, {calls * per_call} Adam "
                       f"steps each (batch 8, 32x32 crops); network input: db4 approximation, K = 4 (automatic level) "
                       f"for the DWT-LRX entry, K = 7 (level 5) for the full-band entry",
           "train_data_s": gen_s, "train_s": train_s,
           "train_steps_per_s": {k: calls * per_call / v for k, v in train_s.items()}}
    full = torch.empty((HS, HS), device=dev)
    ms_full = _time(lambda: wdad.wdad_detect(cube, 0, reduce=False, inner=5, outer=15, out=full), n=1, warm=0)
    red = torch.empty((HS, HS), device=dev)
    ms_red = _time(lambda: wdad.wdad_detect(cube, 0, reduce=True, inner=5, outer=15, out=red), n=5)
    full_h, red_h = full.cpu().numpy(), red.cpu().numpy()
    for name, exact_reduce, ref, ms_ref in (("fullband_lrx", False, full_h, ms_full), ("dwt_lrx", True, red_h, ms_red)):
        box = {}
        net, lev = nets[name], levels[name]

        def run():
            box["r"] = wdad.wdad_screen_run(net, cube, top_frac=0.02, audit_frac=0.005, seed=1, tile_rows=256,
                                            exact_reduce=exact_reduce, inner=5, outer=15, level=lev, want_pred=False)
        ms = _time(run, n=3, warm=1)
        score, _, sel, nsel = box["r"]
        s = score.cpu().numpy()
        selm = sel.cpu().numpy() > 0
        truth = (mask > 0) & (ref >= np.quantile(ref, 0.98))
        out[name] = {
            "screened_ms": ms, "exact_map_ms": ms_ref, "speedup": ms_ref / ms,
            "screened_Mpixel_s": P / (ms * 1e-3) / 1e6, "exact_Mpixel_s": P / (ms_ref * 1e-3) / 1e6,
            "fraction_evaluated": nsel / P, "implanted_in_exact_top2pct": int(truth.sum()),
            "recall": float((selm & truth).sum() / max(1, truth.sum())),
            "auc_exact": wdad.wdad_auc(ref, mask), "auc_screened": wdad.wdad_auc(s, mask),
            "exact_values_identical": bool(np.array_equal(s[selm], ref[selm])),
        }
        out[name]["dauc"] = out[name]["auc_screened"] - out[name]["auc_exact"]
        # second convention: unevaluated pixels ranked below every evaluated one but among
        # themselves by the network's prediction (the timed run skips the prediction map)
        _, pred, sel2, _ = wdad.wdad_screen_run(net, cube, top_frac=0.02, audit_frac=0.005, seed=1, tile_rows=256,
                                                exact_reduce=exact_reduce, inner=5, outer=15, level=lev,
                                                want_pred=True)
        pr = pred.cpu().numpy().ravel()
        sel2 = sel2.cpu().numpy().ravel() > 0
        key = np.empty(P, dtype=np.float64)
        ex = s.ravel()[sel2]
        key[sel2] = 2.0 + np.argsort(np.argsort(ex, kind="stable"), kind="stable") / max(1, ex.size)
        un = pr[~sel2]
        key[~sel2] = np.argsort(np.argsort(un, kind="stable"), kind="stable") / max(1, un.size)
        out[name]["auc_screened_pred_below_cut"] = wdad.wdad_auc(key.reshape(s.shape).astype(np.float32), mask)
        out[name]["dauc_pred_below_cut"] = out[name]["auc_screened_pred_below_cut"] - out[name]["auc_exact"]
    for net in nets.values():
        net.close()
    del cube, full, red
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1201_2025_gb300 import synth, wdad

    sc = synth.scene_512x512(rank)
    x = torch.from_numpy(sc.cube).to(dev)
    K = wdad.wdad_query_K(L)
    approx = torch.empty((H, W, K), device=dev)
    out = torch.empty((len(WINDOWS), 3, H, W), device=dev)
    params = [wdad.wdad_default_params(inner=a, outer=b) for a, b in WINDOWS]
    pdwt = wdad.wdad_default_params()
    stream = torch.cuda.current_stream(dev)
    nsteps = args.steps
    # The timed steps are one wdad_detect_sequence call over the same cube K times: the DWT of
    # step k (HBM-bound) runs on the library's own stream, on part of the SMs, beside the
    # detector launch of step k - 1 (issue-bound) on the caller's stream, through two
    # approximation buffers.  Every step still runs the whole path (one DWT of the cube, nine
    # score maps).  Launch durations are timed with CUDA events on every EV_EVERY-th step only:
    # a timing event on every step costs a few microseconds of overlap per step.
    EV_EVERY = 8

    def make_events(n, timing):
        if not timing:
            return None
        evs = [torch.cuda.Event(enable_timing=True) if k % EV_EVERY == 0 else None
               for k in range(n) for _ in range(4)]
        for e in evs:  # create the CUDA events now, outside the timed region
            if e is not None:
                e.record(stream)
        return evs

    def run_steps(evs, n):
        wdad.wdad_detect_sequence([x] * n, params, outs=[out] * n, events=evs)

    run_steps(None, max(3, args.warmup))
    torch.cuda.synchronize()
    ev = make_events(nsteps, True)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        clk.mark()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        run_steps(ev, nsteps)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms_total = max_over_ranks(t0.elapsed_time(t1), ws, dev)
    ms_step = ms_total / nsteps
    value = job_value(ws, ms_step)

    # launch durations inside the timed region, on each kernel's own stream (they overlap)
    sampled = [k for k in range(nsteps) if ev[4 * k] is not None]
    dwt_ms = sum(ev[4 * k].elapsed_time(ev[4 * k + 1]) for k in sampled) / len(sampled)
    det_launch_ms = sum(ev[4 * k + 2].elapsed_time(ev[4 * k + 3]) for k in sampled) / len(sampled)

    wdad.wdad_dwt_approx(x, pdwt, out=approx)  # the approximation matrix the launches below read

    def _time_serial(fn, n=20):
        for _ in range(3):
            fn()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / n

    # the same kernels alone (serial): the three-window launch, and each window on its own
    windows_ms = _time_serial(lambda: wdad.wdad_detect_windows(approx, params, reduce=False, out=out))
    det_ms = [_time_serial(lambda p=p, i=i: wdad.wdad_detect_all(approx, reduce=False, params=p, out=out[i]))
              for i, p in enumerate(params)]
    dwt_alone_ms = _time_serial(lambda: wdad.wdad_dwt_approx(x, pdwt, out=approx))
    peak, peak_kind = _peaks()
    dwt_gbs = H * W * BYTES_DWT_PER_PX / (dwt_ms * 1e-3) / 1e9
    def _traffic(name):  # dram read + write bytes of one launch, from the committed ncu summary
        try:
            with open(os.path.join(ROOT, "profiles", name)) as f:
                for line in f:
                    if line.startswith("dram_bytes_per_launch:"):
                        return int(line.split(":")[1])
        except Exception:
            pass
        return None

    traffic = _traffic("dwt_apply_kernel_512x512x224.md")
    roofline_dwt = {"kernel": "dwt_apply_kernel", "bound": "hbm", "achieved": dwt_gbs, "peak": peak, "unit": "GB/s",
                    "frac": dwt_gbs / peak, "traffic": traffic, "peak_source": peak_kind,
                    "algorithmic_bytes_per_launch": H * W * BYTES_DWT_PER_PX}
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    det_flops = len(WINDOWS) * H * W * FLOPS_DETECT_PER_PX  # one launch covers the three windows
    det_tflops = det_flops / (det_launch_ms * 1e-3) / 1e12
    alu_peak = FP32_LANES * sm_mhz * 1e6 / 1e12
    roofline_det = {"kernel": "detect_multi_kernel<4>", "bound": "alu", "achieved": det_tflops, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": det_tflops / alu_peak,
                    "traffic": _traffic("detect_multi_kernel_512x512_K4_3windows.md"),
                    "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 at {sm_mhz:.0f} MHz",
                    "algorithmic_flops_per_launch": det_flops}
    # the dominant kernel of the step is the one with the larger share of the step time
    if dwt_ms >= det_launch_ms:
        roofline, roofline_other = roofline_dwt, roofline_det
    else:
        roofline, roofline_other = roofline_det, roofline_dwt
    # per-detector reduced timings and full-band throughput on a strip (outside the timed step)
    def _time(fn, n=10):
        for _ in range(2):
            fn()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / n

    one = torch.empty((H, W), device=dev)
    per_det = {}
    for (wi, wo), p in zip(WINDOWS, params):
        for det, name in enumerate(("lrx", "dwrx", "dwest")):
            ms = _time(lambda: wdad.wdad_detect(approx, det, reduce=False, params=p, out=one))
            dwt_plus = dwt_alone_ms + ms
            per_det[f"{name}@{wi}/{wo}"] = {"detector_ms": ms, "Mpixel_s_with_dwt": H * W / (dwt_plus * 1e-3) / 1e6}
    # adaptive cut-off of Eq. 12 (z = 2.33, alpha = 0.01) on the three maps of window (5,15)
    thr = {}
    maps5 = out[WINDOWS.index((5, 15))]
    for d, dn in enumerate(("lrx", "dwrx", "dwest")):
        mk = torch.empty((H, W), dtype=torch.uint8, device=dev)
        ms = _time(lambda: wdad.wdad_adaptive_threshold(maps5[d], 2.33, mask=mk, want_stats=False), n=10)
        ms_host = _time(lambda: wdad.wdad_adaptive_threshold(maps5[d], 2.33, mask=mk), n=10)
        mu_d, sd_d, tau, cnt, mk = wdad.wdad_adaptive_threshold(maps5[d], 2.33, mask=mk)
        m = mk.cpu().numpy() > 0
        thr[dn] = {"us_per_map": ms * 1e3, "us_per_map_with_host_stats": ms_host * 1e3, "tau": tau,
                   "declared_fraction": float(m.mean()),
                   "implanted_recall": float((m & (sc.mask > 0)).sum() / max(1, (sc.mask > 0).sum()))}
    thr["workload"] = "DWT-reduced maps of the 512x512x224 cube at window (5,15), z_alpha = 2.33"
    # global RX (Eq. 1): image-wide mean and covariance, on the full band and on the reduced cube
    grx = {}
    gout = torch.empty((H, W), device=dev)
    for name, red in (("full_band", False), ("dwt_reduced", True)):
        ms = _time(lambda: wdad.wdad_global_rx(x, reduce=red, out=gout), n=5)
        g = wdad.wdad_global_rx(x, reduce=red, out=gout).cpu().numpy()
        grx[name] = {"ms": ms, "Mpixel_s": H * W / (ms * 1e-3) / 1e6, "auc": wdad.wdad_auc(g, sc.mask)}
    grx["workload"] = "512x512x224 cube, loading 1e-3 (the reduced entry includes its DWT)"
    full = {}
    if not args.no_full:
        rows = args.full_rows
        strip = x[:rows].contiguous()
        sout = torch.empty((3, rows, W), device=dev)
        sone = torch.empty((rows, W), device=dev)
        tc_peak, tc_kind = _bf16_peak()
        for (wi, wo), p in zip(WINDOWS, params):
            ms_all = _time(lambda: wdad.wdad_detect_all(strip, reduce=False, params=p, out=sout), n=2)
            ms_lrx = _time(lambda: wdad.wdad_detect(strip, 0, reduce=False, params=p, out=sone), n=2)
            pm = wdad.wdad_default_params(inner=wi, outer=wo, precision=1)
            ms_lrx_mixed = _time(lambda: wdad.wdad_detect(strip, 0, reduce=False, params=pm, out=sone), n=2)
            ent = {"all3_Mpixel_s": rows * W / (ms_all * 1e-3) / 1e6,
                   "lrx_Mpixel_s": rows * W / (ms_lrx * 1e-3) / 1e6,
                   "lrx_mixed_Mpixel_s": rows * W / (ms_lrx_mixed * 1e-3) / 1e6,
                   "reduced_speedup_all3": (ms_all / (rows * W)) / ((dwt_alone_ms + det_ms[WINDOWS.index((wi, wo))]) / (H * W))}
            ent["roofline_lrx_fp32"] = fullband_roofline(L, wi, wo, "lrx", ent["lrx_Mpixel_s"], tc_peak, alu_peak)
            ent["roofline_lrx_mixed"] = fullband_roofline(L, wi, wo, "lrx", ent["lrx_mixed_Mpixel_s"], tc_peak, alu_peak)
            ent["roofline_all3_fp32"] = fullband_roofline(L, wi, wo, "all3", ent["all3_Mpixel_s"], tc_peak, alu_peak)
            full[f"{wi}/{wo}"] = ent
        full["sample"] = f"{rows} x {W} x {L} strip of the cube, all pixels of the strip"
        full["roofline_peaks"] = {"tensor_TFLOP_s": tc_peak, "tensor_source": tc_kind, "fp32_simt_TFLOP_s": alu_peak,
                                  "fp32_source": f"derived: 152 SMs x 128 FP32 lanes x 2 at {sm_mhz:.0f} MHz"}
    # mixed precision against the FP32 and FP64 full-band forms on an ill-conditioned AR(1) scene.
    # Window 3/11 (N = 112 < L): LRX/DWRX take the FP32 sample-Gram (Woodbury) form in every
    # precision, DWEST the BF16 tensor-core Gram in MIXED; window 7/21 (N = 392 >= L): all three
    # detectors use the BF16 tensor-core Gram in MIXED.
    mixed = {}
    if not args.no_full:
        ar = synth.make_scene(64, 64, L, seed=7, n_anom=10, anom_side=(1, 3), abundance=(0.1, 0.5), margin=6,
                              ar_rho=0.98)
        xa = torch.from_numpy(ar.cube).to(dev)
        # loading 1e-6 as well: at 1e-3 the loading bounds cond(C_o + delta I) by 1 + 1e3 L < 1e6,
        # so only a lighter loading lets the 1e6 gate fire
        for wi, wo, ld in ((3, 11, 1e-3), (7, 21, 1e-3), (3, 11, 1e-6)):
            res = {}
            for name, prec, gate in (("fp64", 2, 1e6), ("fp32", 0, 1e6), ("mixed_gate1e6", 1, 1e6),
                                     ("mixed_gate1e3", 1, 1e3)):
                maps, ms_det, frac_det = [], [], []
                for d in range(3):
                    fl = torch.zeros((64, 64), dtype=torch.uint8, device=dev)
                    pp = wdad.wdad_default_params(inner=wi, outer=wo, precision=prec, cond_gate=gate, loading=ld)
                    ms_det.append(_time(lambda: wdad.wdad_detect(xa, d, reduce=False, params=pp, flags=fl), n=1))
                    fl.zero_()
                    maps.append(wdad.wdad_detect(xa, d, reduce=False, params=pp, flags=fl).cpu().numpy())
                    frac_det.append(float((fl.cpu().numpy() & 1).mean()))
                res[name] = (maps, ms_det, frac_det)
            ref = res["fp64"][0]
            mw = {}
            for name, (maps, ms_det, frac_det) in res.items():
                ent = {}
                for d, dn in enumerate(("lrx", "dwrx", "dwest")):
                    ent[f"{dn}_Mpixel_s"] = 64 * 64 / (ms_det[d] * 1e-3) / 1e6
                    ent[f"{dn}_fp64_resolved_fraction"] = frac_det[d]
                    ent[f"{dn}_auc"] = wdad.wdad_auc(maps[d], ar.mask)
                    ent[f"{dn}_dauc_vs_fp64"] = ent[f"{dn}_auc"] - wdad.wdad_auc(ref[d], ar.mask)
                    rel = np.abs(maps[d] - ref[d]) / np.maximum(np.abs(ref[d]), 1e-6 * np.median(np.abs(ref[d])))
                    ent[f"{dn}_median_rel_err_vs_fp64"] = float(np.median(rel))
                    ent[f"{dn}_max_rel_err_vs_fp64"] = float(np.max(rel))
                mw[name] = ent
            mixed[f"{wi}/{wo}" + ("" if ld == 1e-3 else f"_loading{ld:g}")] = mw
        mixed["workload"] = ("64x64x224 AR(1) rho=0.98 scene, 10 targets, windows 3/11 and 7/21 at loading 1e-3, "
                             "3/11 at loading 1e-6")
    batching = None
    if not args.no_batch:
        batching = bench_batching(dev, stream, peak)
        batching["small_cubes"] = bench_batching(dev, stream, peak, side_lo=32, side_hi=160)
    screening = bench_screening(dev, stream, args.screen_train_cubes, args.screen_train_steps) \
        if not args.no_screen else None
    step_bytes = H * W * (BYTES_DWT_PER_PX + 3 * 3 * 4)
    breakdown = {"pipeline": "wdad_detect_sequence: the DWT of step k on the library's high-priority stream (3/4 of "
                             "the SMs, a shared-memory reservation leaving room for one detector CTA per SM) beside "
                             "the detector launch of step k-1; launch times from events on every "
                             f"{EV_EVERY}th step",
                 "dwt_ms_in_step": dwt_ms, "detect_launch_ms_in_step": det_launch_ms, "dwt_ms_alone": dwt_alone_ms,
                 "detect_ms_alone": dict(zip([f"{a}/{b}" for a, b in WINDOWS], det_ms)),
                 "detect_three_windows_one_launch_ms_alone": windows_ms,
                 "step_algorithmic_GBps": step_bytes / (ms_step * 1e-3) / 1e9,
                 "step_frac_of_hbm": step_bytes / (ms_step * 1e-3) / 1e9 / peak, "per_detector": per_det,
                 "adaptive_threshold": thr, "global_rx": grx, "fullband_fp32": full, "mixed_precision": mixed, "batching": batching,
                 "screening": screening}

    # end to end through the host-buffer entry point: H2D cube, DWT, 3 windows, D2H 9 maps
    hc = torch.from_numpy(sc.cube).pin_memory()
    hs = torch.empty((len(WINDOWS), 3, H, W), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(nsteps, args.e2e_steps))
    for _ in range(3):
        wdad.wdad_detect_all_host(hc, params=params, out=hs)
    torch.cuda.synchronize()
    barrier()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(e2e_steps):
        wdad.wdad_detect_all_host(hc, params=params, out=hs)
        stream.synchronize()  # the host reads its scores each step
    s1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(s0.elapsed_time(s1) / e2e_steps, ws, dev)
    # the host link on its own: plain pinned copies of the same bytes, H2D and D2H
    dcube = torch.empty((H, W, L), device=dev)
    dmaps = torch.empty((len(WINDOWS), 3, H, W), device=dev)
    h2d_ms = _time(lambda: dcube.copy_(hc, non_blocking=True), n=10)
    d2h_ms = _time(lambda: hs.copy_(dmaps, non_blocking=True), n=10)
    del dcube, dmaps
    h2d_b, d2h_b = H * W * L * 4, len(WINDOWS) * 3 * H * W * 4
    e2e = {"value": job_value(ws, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b, "ms_per_step": e2e_ms,
           "link_GBps_achieved": (h2d_b + d2h_b) / (e2e_ms * 1e-3) / 1e9,
           "plain_pinned_copy_GBps": {"h2d": h2d_b / (h2d_ms * 1e-3) / 1e9, "d2h": d2h_b / (d2h_ms * 1e-3) / 1e9},
           "link_bound_ms": h2d_ms + d2h_ms,
           "pipeline": "row bands over three streams: a copy engine moves band b to the device while the DWT "
                       "of band b - 1 and the detector tiles of band b - 2 run, and each band's score rows go "
                       "back in one strided copy behind its tiles"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        v, dt, reps = cpu_oracle_sample(sc.cube, args.cpu_rows, args.cpu_seconds)
        cpu = {"value": v / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"rows 0..{args.cpu_rows - 1} of the cube ({args.cpu_rows * W} px) x {reps} repetitions, "
                         f"DWT + 3 windows x 3 detectors, FP64, {dt:.1f} s"}
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": nsteps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded AVIRIS-shaped linear-mixing cube)",
        "config": _config(ws),
        "per_detector": {"value": 3 * value, "unit": "Mpixel/s per detector",
                         "note": "pixel-window-detector evaluations per second: value x 3 detectors"},
        "step_frac_of_hbm": breakdown["step_algorithmic_GBps"] / peak,
        "roofline": roofline, "roofline_other_kernel": roofline_other,
        "roofline_fullband": {k: {f: full[k][f]["frac"] for f in ("roofline_lrx_fp32", "roofline_lrx_mixed",
                                                                   "roofline_all3_fp32")}
                              for k in full if isinstance(full.get(k), dict) and "roofline_lrx_fp32" in full[k]},
        "breakdown": breakdown, "e2e": e2e,
        "cpu_baseline": cpu, "gpu_launches": nsteps * 2, "clocks": clocks,
    }), flush=True)


def run_c3_table():
    """The precision workload at its own size: a 1024x1024x224 cube with band-to-band AR(1)
    noise (rho 0.98).  LRX and DWRX on every pixel, DWEST on a 128-row strip (its FP64 path takes
    minutes on the whole map), windows (3,11) and (7,21), loading 1e-3, gate 1e6.  The GPU FP64
    path (held to 1e-6 of the oracle by the tests) is the yardstick: per detector and precision the
    median and 99th-percentile relative error against it, the AUC change against it, the
    throughput and the FP64 re-solved fraction of MIXED.  Prints one JSON object."""
    import torch
    from paper_1201_2025_gb300 import synth, wdad
    dev = torch.device("cuda", 0)
    sc = synth.scene_ar1(1024, 1024, L, seed=0)
    x = torch.from_numpy(sc.cube).to(dev)
    strip_rows = 128
    xs = x[:strip_rows].contiguous()
    mask_s = sc.mask[:strip_rows]
    res = {"workload": "1024x1024x224 f32, AR(1) rho 0.98, 209 targets (1-3 px, f 0.1-0.5); LRX/DWRX whole map, "
                       f"DWEST on rows 0..{strip_rows - 1}; errors against the GPU FP64 path", "windows": {}}
    for wi, wo in ((3, 11), (7, 21)):
        ent = {}
        for det, dn in enumerate(("lrx", "dwrx", "dwest")):
            cube, mask = (xs, mask_s) if det == 2 else (x, sc.mask)
            Hh, Ww = cube.shape[0], cube.shape[1]
            maps, ms, frac = {}, {}, {}
            for name, prec in (("fp64", 2), ("fp32", 0), ("mixed", 1)):
                fl = torch.zeros((Hh, Ww), dtype=torch.uint8, device=dev)
                pp = wdad.wdad_default_params(inner=wi, outer=wo, precision=prec)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m = wdad.wdad_detect(cube, det, reduce=False, params=pp, flags=fl)
                torch.cuda.synchronize()
                ms[name] = (time.perf_counter() - t0) * 1e3
                maps[name] = m.cpu().numpy().astype(np.float64)
                frac[name] = float((fl.cpu().numpy() & 1).mean())
            ref = maps["fp64"]
            auc_ref = wdad.wdad_auc(ref, mask)
            out = {"pixels": int(Hh * Ww), "auc_fp64": auc_ref}
            for name in ("fp32", "mixed"):
                den = np.maximum(np.abs(ref), 1e-6 * np.median(np.abs(ref)))
                rel = np.abs(maps[name] - ref) / den
                out[name] = {"Mpixel_s": Hh * Ww / (ms[name] * 1e-3) / 1e6, "median_rel_err": float(np.median(rel)),
                             "p99_rel_err": float(np.quantile(rel, 0.99)),
                             "dauc_vs_fp64": wdad.wdad_auc(maps[name], mask) - auc_ref}
            out["mixed"]["fp64_resolved_fraction"] = frac["mixed"]
            out["fp64_Mpixel_s"] = Hh * Ww / (ms["fp64"] * 1e-3) / 1e6
            ent[dn] = out
        res["windows"][f"{wi}/{wo}"] = ent
    print(json.dumps({"c3_table": res}), flush=True)


def run_profile_case(case: str):
    """Small workloads for ncu captures of kernels outside the timed step (a few GB at most):
    batch (8 cubes, side <= 512), screen (1024x1024x224 screening pass), mixed (64x64x224 AR(1)
    full-band LRX, MIXED and FP32 at window 7/21, then FP32 at 3/11), grx (global RX on a 512x512x224 cube).  Each runs its workload twice and exits."""
    import torch
    from paper_1201_2025_gb300 import synth, wdad
    dev = torch.device("cuda", 0)
    if case == "batch":
        jobs = []
        for sp in synth.batch_specs(8, seed=0):
            S = min(sp["H"], 512)
            cube, _ = synth.make_scene_device(S, S, sp["L"], seed=sp["seed"], n_anom=20, anom_side=(1, 3),
                                              abundance=(0.1, 0.5), margin=10, device=dev)
            jobs.append(dict(cube=cube, detector=sp["detector"], scores=torch.empty((S, S), device=dev),
                             over=dict(inner=sp["inner"], outer=sp["outer"])))
        b = wdad.wdad_batch(jobs, autotune=False, use_graph=True)
        for _ in range(2):
            b.launch()
        st, _ = b.status()
        b.close()
        if st != 0:
            raise SystemExit(f"batch status {st}")
    elif case == "screen":
        net = wdad.wdad_cnn(K=4, seed=1)
        cube, _ = synth.make_scene_device(1024, 1024, L, seed=5, n_anom=800, anom_side=(1, 3), abundance=(0.1, 0.5),
                                          margin=10, device=dev)
        for _ in range(2):
            wdad.wdad_screen_run(net, cube, top_frac=0.02, audit_frac=0.005, seed=1, tile_rows=256, exact_reduce=True,
                                 inner=5, outer=15)
        net.close()
    elif case == "mixed":
        sc = synth.make_scene(64, 64, L, seed=7, n_anom=10, anom_side=(1, 3), abundance=(0.1, 0.5), margin=6,
                              ar_rho=0.98)
        x = torch.from_numpy(sc.cube).to(dev)
        for _ in range(2):  # MIXED and FP32 at 7/21 (BF16 / split tensor-core Gram), FP32 at 3/11 (sample Gram)
            wdad.wdad_detect(x, 0, reduce=False, inner=7, outer=21, precision=1, cond_gate=1e6)
            wdad.wdad_detect(x, 0, reduce=False, inner=7, outer=21, precision=0)
            wdad.wdad_detect(x, 0, reduce=False, inner=3, outer=11, precision=0)
    elif case == "grx":
        sc = synth.make_scene(512, 512, L, seed=0, n_anom=200, anom_side=(1, 3), abundance=(0.1, 0.5), margin=10)
        x = torch.from_numpy(sc.cube).to(dev)
        for _ in range(2):
            wdad.wdad_global_rx(x, reduce=False)
    torch.cuda.synchronize()
    print("profile case", case, "ok")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-rows", type=int, default=512)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-full", action="store_true")
    ap.add_argument("--full-rows", type=int, default=16)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-screen", action="store_true")
    ap.add_argument("--screen-train-cubes", type=int, default=200)
    ap.add_argument("--screen-train-steps", type=int, default=2000)
    ap.add_argument("--c3-table", action="store_true",
                    help="precision workload at full size (1024x1024x224 AR(1)): errors and AUC changes per detector")
    ap.add_argument("--profile-case", choices=["batch", "screen", "mixed", "grx"], default=None,
                    help="run one small workload for an ncu capture and exit")
    args = ap.parse_args()
    if args.c3_table:
        run_c3_table()
    elif args.profile_case:
        run_profile_case(args.profile_case)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
