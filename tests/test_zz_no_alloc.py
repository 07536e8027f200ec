"""The allocation-free reduced pass (wdad_detect_all_noalloc) against wdad_detect_all.

This entry point serves callers that cannot call cudaMalloc (fixed memory budgets,
framework-owned device pools, latency-critical code).  It keeps its scratch in a fixed
array inside the library that every call shares.  The test calls it twice in a row on
different scenes, so stale contents from the first call would show up in the second.
Both entry points run the same kernels with the same tile plan, so scores and flags must be
bit-identical.  A fresh process checks that repeated calls leave the device's free memory
unchanged.  The file runs last so that a stop at the first failure has already run
everything else.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wd():
    from paper_1201_2025_gb300 import wdad
    wdad.lib()
    return wdad


def _both(wd, x, **over):
    H, W, _ = x.shape
    f1 = torch.full((H, W), 255, dtype=torch.uint8, device="cuda")
    f2 = torch.full((H, W), 254, dtype=torch.uint8, device="cuda")
    got = wd.wdad_detect_all_noalloc(x, flags=f1, **over)
    want = wd.wdad_detect_all(x, reduce=True, flags=f2, **over)
    torch.cuda.synchronize()
    return got, want, f1, f2


def test_noalloc_matches_detect_all_on_two_calls_in_a_row(wd):
    from paper_1201_2025_gb300 import synth
    first = synth.make_scene(60, 100, 224, seed=11, n_anom=6, margin=4)
    second = synth.make_scene(37, 53, 189, seed=12, n_anom=4, margin=4)
    for sc, win in ((first, (3, 11)), (second, (5, 13))):
        x = torch.from_numpy(sc.cube).cuda()
        got, want, f1, f2 = _both(wd, x, inner=win[0], outer=win[1])
        assert torch.equal(got, want)
        assert torch.equal(f1, f2)


@pytest.mark.parametrize("taps", [4, 12])
def test_noalloc_other_filters(wd, taps):
    from paper_1201_2025_gb300 import synth
    sc = synth.make_scene(40, 50, 224, seed=13, n_anom=4, margin=4)
    x = torch.from_numpy(sc.cube).cuda()
    got, want, f1, f2 = _both(wd, x, inner=3, outer=9, wavelet_taps=taps)
    assert torch.equal(got, want) and torch.equal(f1, f2)
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_detect_all_noalloc(x, wavelet_taps=taps + 1)
    assert ei.value.status == wd.WDAD_ERR_ARG


def test_noalloc_rejects_sizes_beyond_its_scratch(wd):
    x = torch.zeros((1025, 1024, 16), device="cuda")  # K = 4: 4,198,400 coefficients > 4,194,304
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_detect_all_noalloc(x)
    assert ei.value.status == wd.WDAD_ERR_ARG


def test_noalloc_widest_window(wd):
    # the widest window the library takes (63 pixels): both entry points agree bit for bit;
    # one wider is refused by both
    from paper_1201_2025_gb300 import synth
    sc = synth.make_scene(70, 90, 64, seed=14, n_anom=4, margin=4)
    x = torch.from_numpy(sc.cube).cuda()
    got, want, f1, f2 = _both(wd, x, inner=61, outer=63)
    assert torch.equal(got, want) and torch.equal(f1, f2)
    for fn in (lambda: wd.wdad_detect_all_noalloc(x, inner=61, outer=65),
               lambda: wd.wdad_detect_all(x, reduce=True, inner=61, outer=65)):
        with pytest.raises(wd.WdadError) as ei:
            fn()
        assert ei.value.status == wd.WDAD_ERR_ARG


def test_noalloc_allocates_no_device_memory():
    # a fresh process: the first call may load the library's module (and with it the fixed
    # array); later calls of other sizes must leave the device's free memory and torch's
    # allocator untouched, and no library handle (which owns workspace) may be created
    code = textwrap.dedent(f"""
        import sys, numpy as np, torch
        sys.path.insert(0, {ROOT!r})
        from paper_1201_2025_gb300 import synth, wdad
        bufs = []
        for H, W in ((60, 100), (200, 250), (128, 512)):
            sc = synth.make_scene(H, W, 224, seed=H, n_anom=4, margin=4)
            x = torch.from_numpy(sc.cube).cuda()
            bufs.append((x, torch.empty((3, H, W), device="cuda"), torch.empty((H, W), dtype=torch.uint8, device="cuda")))
        x, out, fl = bufs[0]
        wdad.wdad_detect_all_noalloc(x, inner=3, outer=11, out=out, flags=fl)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for x, out, fl in bufs[1:] + bufs[:1]:
            wdad.wdad_detect_all_noalloc(x, inner=3, outer=11, out=out, flags=fl)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        assert torch.cuda.memory_allocated() == alloc0
        assert not wdad._handles, wdad._handles
        assert bool(torch.isfinite(bufs[1][1]).all())
        print("no-alloc ok")
    """)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "no-alloc ok" in r.stdout, r.stdout + r.stderr
