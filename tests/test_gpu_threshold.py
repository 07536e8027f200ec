"""Adaptive cut-off of Eq. 12 on the GPU against the FP64 oracle: statistics to FP64 rounding,
decisions identical except for scores within rounding distance of tau."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    from paper_1201_2025_gb300 import wdad
    wdad.lib()
    return wdad


def _check(wd, s, z):
    got_mu, got_sd, got_tau, got_n, mask = wd.wdad_adaptive_threshold(torch.from_numpy(s).cuda(), z)
    mu, sd, tau, want = oracle.adaptive_threshold(s.astype(np.float64), z)
    assert got_n == int(np.isfinite(s).sum())
    for g, w in ((got_mu, mu), (got_sd, sd), (got_tau, tau)):
        assert abs(g - w) <= 1e-12 * max(abs(w), 1.0), (g, w)
    m = mask.cpu().numpy().reshape(s.shape)
    near = np.abs(s.astype(np.float64) - tau) <= 1e-9 * max(abs(tau), 1.0)
    assert np.array_equal(m[~near], want[~near])


@pytest.mark.parametrize("n", [1, 7, 1000, 512 * 512, 1024 * 1024 + 13])
@pytest.mark.parametrize("z", [0.0, 1.5, 2.33, -1.0])
def test_threshold_matches_oracle(wd, n, z):
    rng = np.random.default_rng(7 * n + int(100 * (z + 2)))
    s = (rng.chisquare(4, n) * rng.uniform(0.5, 2.0)).astype(np.float32)
    s[rng.random(n) < 0.01] = np.nan  # border-style NaN entries
    _check(wd, s, z)


def test_threshold_on_a_detector_map(wd):
    from paper_1201_2025_gb300 import synth
    sc = synth.scene_48x48(0)
    x = torch.from_numpy(sc.cube).cuda()
    lrx = wd.wdad_detect(x, 0, reduce=True, inner=3, outer=11, border=1)  # NaN where the window leaves the image
    _check(wd, lrx.cpu().numpy(), 2.33)


def test_threshold_edge_cases(wd):
    mu, sd, tau, n, _ = wd.wdad_adaptive_threshold(torch.zeros(0, device="cuda"), 1.0)
    assert n == 0 and np.isnan(mu) and np.isnan(tau)
    s = np.full(100, np.nan, np.float32)  # no finite score: nothing declared
    mu, sd, tau, n, mask = wd.wdad_adaptive_threshold(torch.from_numpy(s).cuda(), 1.0)
    assert n == 0 and np.isnan(tau) and int(mask.sum()) == 0
    s = np.full(50, 3.0, np.float32)  # constant map: sigma 0, tau = mean, nothing above it
    mu, sd, tau, n, mask = wd.wdad_adaptive_threshold(torch.from_numpy(s).cuda(), 2.0)
    assert mu == 3.0 and sd == 0.0 and tau == 3.0 and int(mask.sum()) == 0
    with pytest.raises(RuntimeError):
        wd.wdad_adaptive_threshold(torch.ones(10, device="cuda"), float("nan"))


def test_threshold_without_host_stats_gives_the_same_mask(wd):
    rng = np.random.default_rng(11)
    s = torch.from_numpy(rng.chisquare(4, 300001).astype(np.float32)).cuda()
    *_, m_sync = wd.wdad_adaptive_threshold(s, 2.33)
    mu, sd, tau, n, m_async = wd.wdad_adaptive_threshold(s, 2.33, want_stats=False)
    torch.cuda.synchronize()
    assert n == -1 and np.isnan(tau)
    assert torch.equal(m_sync, m_async)
