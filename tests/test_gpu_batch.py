"""A8 batching: uneven cubes in one persistent launch (optionally a CUDA graph), against
the same jobs run alone and against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle
from parity import TOL_SCORE, dwest_ok_mask, dwest_relerr, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(40, 50, 128, (3, 9), 3), (33, 70, 188, (5, 15), 0), (64, 64, 224, (7, 21), 2), (17, 100, 224, (3, 11), 1),
          (90, 31, 128, (1, 15), 3), (50, 50, 188, (3, 9), 2), (25, 25, 224, (5, 13), 3)]


@pytest.fixture(scope="module")
def wd():
    from paper_1201_2025_gb300 import wdad
    wdad.lib()
    return wdad


@pytest.fixture(scope="module")
def scenes():
    from paper_1201_2025_gb300 import synth
    return [synth.make_scene(H, W, L, seed=100 + i, n_anom=4, margin=3) for i, (H, W, L, _, _) in enumerate(SHAPES)]


def _jobs(wd, scenes):
    jobs = []
    for sc, (H, W, L, win, det) in zip(scenes, SHAPES):
        x = torch.from_numpy(sc.cube).cuda()
        out = torch.full((3, H, W) if det == 3 else (H, W), -1.0, device="cuda")
        jobs.append({"cube": x, "detector": det, "scores": out, "over": {"inner": win[0], "outer": win[1]}})
    return jobs


def _alone(wd, job):
    o = job["over"]
    if job["detector"] == 3:
        return wd.wdad_detect_all(job["cube"], reduce=True, inner=o["inner"], outer=o["outer"])
    return wd.wdad_detect(job["cube"], job["detector"], reduce=True, inner=o["inner"], outer=o["outer"])


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_default_plans_bit_identical_to_jobs_alone(wd, scenes, use_graph):
    jobs = _jobs(wd, scenes)
    b = wd.wdad_batch(jobs, autotune=False, use_graph=use_graph)
    for _ in range(2):  # replays reuse the same buffers
        b.launch()
        st, _ = b.status()
        assert st == wd.WDAD_OK
        for job in jobs:
            assert torch.equal(job["scores"], _alone(wd, job))
    b.close()


def test_graph_replay_sees_new_cube_contents(wd, scenes):
    jobs = _jobs(wd, scenes)
    b = wd.wdad_batch(jobs, autotune=False, use_graph=True)
    b.launch()
    assert b.status()[0] == wd.WDAD_OK
    first = jobs[2]["scores"].clone()
    jobs[2]["cube"].mul_(1.5).add_(0.01 * torch.sin(torch.arange(jobs[2]["cube"].numel(), device="cuda")
                                                   ).reshape(jobs[2]["cube"].shape))
    b.launch()
    assert b.status()[0] == wd.WDAD_OK
    assert not torch.equal(first, jobs[2]["scores"])
    assert torch.equal(jobs[2]["scores"], _alone(wd, jobs[2]))
    b.close()


def test_autotuned_batch_matches_oracle(wd, scenes):
    jobs = _jobs(wd, scenes)
    b = wd.wdad_batch(jobs, autotune=True, use_graph=True)
    b.launch()
    st, ths = b.status()
    assert st == wd.WDAD_OK and all(1 <= t <= 16 for t in ths)
    for sc, job, (H, W, L, win, det) in zip(scenes, jobs, SHAPES):
        a = oracle.dwt_approx(sc.cube)
        got = job["scores"].cpu().numpy()
        dets = [0, 1, 2] if det == 3 else [det]
        for i, d in enumerate(dets):
            g = got[i] if det == 3 else got
            if d < 2:
                assert relerr(g, oracle.detect(a, d, *win)).max() <= TOL_SCORE
            else:
                want, aux = oracle.detect(a, 2, *win, want_aux=True)
                ok = dwest_ok_mask(aux)
                assert dwest_relerr(g, want, aux)[ok].max() <= TOL_SCORE
    b.close()


def test_autotune_returns_a_feasible_tile_height(wd):
    th = wd.wdad_autotune(4, 7, 21)
    assert 1 <= th <= 16
    assert wd.wdad_autotune(4, 7, 21) == th  # cached


def test_dropped_dwt_item_times_out_without_hanging(wd, scenes, monkeypatch):
    # host-side fault injection: job 1 loses one DWT item, so its tiles' bounded wait runs out
    jobs = _jobs(wd, scenes)
    monkeypatch.setenv("WDAD_FAULT_DROP_DWT_ITEM", "1")
    b = wd.wdad_batch(jobs, autotune=False, use_graph=False)
    monkeypatch.delenv("WDAD_FAULT_DROP_DWT_ITEM")
    b.launch()
    st, _ = b.status()
    assert st == wd.WDAD_ERR_TIMEOUT
    assert bool((jobs[1]["scores"] == -1.0).all())  # the starved job wrote nothing
    for i, job in enumerate(jobs):
        if i != 1:
            assert torch.equal(job["scores"], _alone(wd, job))
    b.close()


def test_batch_rejects_unsupported_band_count(wd):
    x = torch.rand((8, 8, 189), device="cuda")
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_batch([{"cube": x, "detector": 0, "scores": torch.empty((8, 8), device="cuda")}])
    assert ei.value.status == wd.WDAD_ERR_UNSUPPORTED


@pytest.mark.parametrize("use_graph", [True, False])
def test_large_jobs_run_as_their_own_launches(wd, scenes, use_graph):
    # jobs of 512 x 512 pixels or more leave the persistent kernel (they fill the GPU alone) and
    # run as their own DWT and detector launches inside the batch: still the single-cube scores
    from paper_1201_2025_gb300 import synth
    jobs = _jobs(wd, scenes[:3])
    for i, (H, W, L, det) in enumerate(((512, 520, 224, 3), (600, 440, 128, 0))):
        sc = synth.make_scene(H, W, L, seed=300 + i, n_anom=10, margin=5)
        jobs.append({"cube": torch.from_numpy(sc.cube).cuda(), "detector": det,
                     "scores": torch.full((3, H, W) if det == 3 else (H, W), -1.0, device="cuda"),
                     "over": {"inner": 5, "outer": 15}})
    b = wd.wdad_batch(jobs, autotune=False, use_graph=use_graph)
    for _ in range(2):
        b.launch()
        st, ths = b.status()
        assert st == wd.WDAD_OK and len(ths) == len(jobs)
        for job in jobs:
            assert torch.equal(job["scores"], _alone(wd, job))
    b.close()
    only_large = jobs[3:]
    b = wd.wdad_batch(only_large, autotune=False, use_graph=use_graph)  # no persistent part at all
    b.launch()
    assert b.status()[0] == wd.WDAD_OK
    for job in only_large:
        assert torch.equal(job["scores"], _alone(wd, job))
    b.close()


def test_full_batching_workload_bit_identical(wd):
    # the batching workload at full size: 64 cubes, side U{128..1024}, L in {128, 188, 224},
    # mixed windows and detectors (device-generated, about 20 GB), one graph launch
    from paper_1201_2025_gb300 import synth
    jobs = []
    for sp in synth.batch_specs(64, seed=0):
        cube, _ = synth.make_scene_device(sp["H"], sp["W"], sp["L"], seed=sp["seed"], n_anom=4, anom_side=(1, 3),
                                          abundance=(0.1, 0.5), margin=10, device=torch.device("cuda", 0))
        jobs.append({"cube": cube, "detector": sp["detector"], "scores": torch.full((sp["H"], sp["W"]), -1.0,
                                                                                    device="cuda"),
                     "over": {"inner": sp["inner"], "outer": sp["outer"]}})
    b = wd.wdad_batch(jobs, autotune=False, use_graph=True)
    b.launch()
    assert b.status()[0] == wd.WDAD_OK
    for job in jobs:
        assert torch.equal(job["scores"], _alone(wd, job))
    b.close()
    del jobs
    torch.cuda.empty_cache()
