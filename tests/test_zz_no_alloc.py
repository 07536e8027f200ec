"""The allocation-free reduced pass (wdad_detect_all_noalloc) against wdad_detect_all.

This entry point serves callers that cannot call cudaMalloc (fixed memory budgets,
framework-owned device pools, latency-critical code).  It keeps its scratch in a fixed
array inside the library that every call shares.  The test calls it twice in a row on
different scenes, so stale contents from the first call would show up in the second.
It compares each result with the handle-based entry point under the score tolerance
of the other tests.  The file runs last so that a stop at the first failure has already
run everything else.
"""
import numpy as np
import pytest

from parity import TOL_SCORE

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    from paper_1201_2025_gb300 import wdad
    wdad.lib()
    return wdad


def _close(a, b):
    a = a.cpu().numpy().astype(np.float64)
    b = b.cpu().numpy().astype(np.float64)
    floor = 1e-6 * np.median(np.abs(b))
    err = np.abs(a - b) / np.maximum(np.abs(b), floor)
    return np.nanmax(err) <= TOL_SCORE and np.array_equal(np.isnan(a), np.isnan(b))


def test_noalloc_matches_detect_all_on_two_calls_in_a_row(wd):
    from paper_1201_2025_gb300 import synth
    first = synth.make_scene(60, 100, 224, seed=11, n_anom=6, margin=4)
    second = synth.make_scene(37, 53, 189, seed=12, n_anom=4, margin=4)
    for sc, win in ((first, (3, 11)), (second, (5, 13))):
        x = torch.from_numpy(sc.cube).cuda()
        got = wd.wdad_detect_all_noalloc(x, inner=win[0], outer=win[1])
        torch.cuda.synchronize()
        want = wd.wdad_detect_all(x, reduce=True, inner=win[0], outer=win[1])
        torch.cuda.synchronize()
        assert _close(got, want)


@pytest.mark.parametrize("taps", [4, 12])
def test_noalloc_other_filters(wd, taps):
    from paper_1201_2025_gb300 import synth
    sc = synth.make_scene(40, 50, 224, seed=13, n_anom=4, margin=4)
    x = torch.from_numpy(sc.cube).cuda()
    got = wd.wdad_detect_all_noalloc(x, inner=3, outer=9, wavelet_taps=taps)
    torch.cuda.synchronize()
    want = wd.wdad_detect_all(x, reduce=True, inner=3, outer=9, wavelet_taps=taps)
    torch.cuda.synchronize()
    assert _close(got, want)
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_detect_all_noalloc(x, wavelet_taps=taps + 1)
    assert ei.value.status == wd.WDAD_ERR_ARG


def test_noalloc_rejects_sizes_beyond_its_scratch(wd):
    x = torch.zeros((1025, 1024, 16), device="cuda")  # K = 4: 4,198,400 coefficients > 4,194,304
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_detect_all_noalloc(x)
    assert ei.value.status == wd.WDAD_ERR_ARG
