"""Mixed precision (A7): the BF16 tensor-core window Gram, its FP32/FP64 siblings, and the
condition-gated full-band detectors, against the FP64 oracle through the C ABI."""
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


@pytest.fixture(scope="module")
def scene48():
    from paper_1201_2025_gb300 import synth
    return synth.scene_48x48(0)


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _annulus(cube, y, x, wi, wo):
    H, W, _ = cube.shape
    ri, ro = wi // 2, wo // 2
    return np.array([cube[oracle.reflect(y + dy, H), oracle.reflect(x + dx, W)]
                     for dy in range(-ro, ro + 1) for dx in range(-ro, ro + 1) if max(abs(dy), abs(dx)) > ri])


def _pixels(H, W, n=12, seed=0):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.choice(H * W, n, replace=False), [0, H * W - 1, W - 1]]))


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (2, 1e-6)])
def test_window_moments_simt_vs_oracle(wd, scene48, prec, tol):
    cube = scene48.cube
    pix = _pixels(48, 48)
    mu, cov = wd.wdad_window_moments(_gpu(cube), pix, inner=3, outer=11, precision=prec)
    mu_r, cov_r = oracle.window_moments(cube.astype(np.float64), 3, 11, pix)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_r, rtol=1e-6, atol=0)
    err = np.abs(cov.cpu().numpy() - cov_r).max(axis=(1, 2)) / np.abs(cov_r).max(axis=(1, 2))
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("D,win", [(224, (3, 11)), (100, (7, 21)), (256, (5, 15))])
def test_tensor_core_gram_is_the_bf16_gram(wd, D, win):
    """The MIXED Gram equals the FP64 Gram of the BF16-rounded centred samples (up to FP32
    accumulation), and is within the BF16 rounding level of the exact covariance."""
    rng = np.random.default_rng(D)
    H, W = 23, 29
    cube = (0.3 + 0.1 * rng.standard_normal((H, W, D)) @ (np.eye(D) + 0.05 * rng.standard_normal((D, D)))
            ).astype(np.float32)
    pix = _pixels(H, W, n=6, seed=D)
    mu, cov = wd.wdad_window_moments(_gpu(cube), pix, inner=win[0], outer=win[1], precision=1)
    mu, cov = mu.cpu().numpy(), cov.cpu().numpy()
    _, cov_exact = oracle.window_moments(cube.astype(np.float64), win[0], win[1], pix)
    for t, p in enumerate(pix):
        y, x = divmod(int(p), W)
        X = _annulus(cube, y, x, *win)  # [N][D] float32
        Xc = bf16_round(X - mu[t][None, :].astype(np.float32)).astype(np.float64)
        ref = Xc.T @ Xc / X.shape[0]
        scale = np.abs(ref).max()
        assert np.abs(cov[t] - ref).max() <= 2e-6 * scale, (t, np.abs(cov[t] - ref).max() / scale)
        assert np.abs(cov[t] - cov_exact[t]).max() <= 2.0 ** -7 * np.abs(cov_exact[t]).max()


def test_mixed_gate_everything_reproduces_fp64(wd, scene48):
    # cond_gate = 1: every pixel's estimate exceeds it -> FP64 re-solve from the data for all
    cube = scene48.cube[:20, :24]
    x = _gpu(cube)
    flags = torch.zeros(cube.shape[:2], dtype=torch.uint8, device="cuda")
    mixed = wd.wdad_detect_all(x, reduce=False, inner=3, outer=9, precision=1, cond_gate=1.0, flags=flags)
    fp64 = wd.wdad_detect_all(x, reduce=False, inner=3, outer=9, precision=2)
    assert torch.equal(mixed, fp64)
    assert bool(torch.all(flags & 1))


def test_mixed_without_gate_is_finite_and_unflagged(wd, scene48):
    # with the gate off, LRX and DWRX stay on the BF16 Gram + FP32 solve; DWEST decides its
    # selection in FP32 and re-solves in FP64 only the pixels with an eigenvalue within
    # 2^-17 max|lambda| of the threshold: the FP32 map elsewhere, the FP64 map there
    cube = scene48.cube[:20, :24]
    x = _gpu(cube)
    for det in (0, 1):
        flags = torch.zeros(cube.shape[:2], dtype=torch.uint8, device="cuda")
        s = wd.wdad_detect(x, det, reduce=False, inner=3, outer=9, precision=1, cond_gate=1e30, flags=flags)
        assert bool(torch.isfinite(s).all())
        assert not bool(torch.any(flags & 1))
    # n_i + N = 81 < L: C_i - C_o has exact zero eigenvalues, whose FP32 values lie within the
    # band around tau, so every pixel is re-solved.  At 7/21 (n_i + N = 441 >= L) FP32 decides
    # the selection of the interior pixels; near the border the reflected window repeats
    # samples, C_o loses rank and those pixels are re-solved.
    for win, sub in (((3, 9), x), ((7, 21), _gpu(scene48.cube))):
        Hh, Ww = sub.shape[:2]
        flags = torch.zeros((Hh, Ww), dtype=torch.uint8, device="cuda")
        mixed = wd.wdad_detect(sub, 2, reduce=False, inner=win[0], outer=win[1], precision=1, cond_gate=1e30,
                               flags=flags)
        fp32 = wd.wdad_detect(sub, 2, reduce=False, inner=win[0], outer=win[1], precision=0)
        fp64 = wd.wdad_detect(sub, 2, reduce=False, inner=win[0], outer=win[1], precision=2)
        re = (flags & 1).bool()
        assert torch.equal(mixed[~re], fp32[~re]) and torch.equal(mixed[re], fp64[re])
        if win == (3, 9):
            assert bool(re.all())
        else:
            ro = win[1] // 2
            frac = float(re[ro:Hh - ro, ro:Ww - ro].float().mean())
            assert frac < 0.5, frac


@pytest.mark.parametrize("win,gate,loading", [((3, 11), 1e6, 1e-3), ((5, 15), 1e6, 1e-3), ((3, 11), 3e4, 1e-3),
                                              ((3, 11), 1e6, 1e-6)])
def test_mixed_fewer_samples_than_bands_matches_oracle(wd, scene48, win, gate, loading):
    # N < L: mixed LRX/DWRX take the FP32 sample-Gram (Woodbury) solve; pixels below the gate
    # meet the FP32 bar max(1e-4, 1.5 u kappa) of the full-band tests (measured up to 0.31 u kappa
    # here), pixels above it are the FP64 re-solve (1e-6)
    from parity import TOL_SCORE, relerr
    cube = scene48.cube.astype(np.float64)
    x = _gpu(scene48.cube)
    pix = _pixels(48, 48, n=40, seed=win[1])
    _, aux = oracle.detect(cube, 0, win[0], win[1], loading=loading, pixels=pix, want_aux=True, want_cond=True)
    kappa = aux[..., 1] / aux[..., 0]
    for det in (0, 1):  # one detector per call: the flags then tell which pixels were re-solved
        flags = torch.zeros((48, 48), dtype=torch.uint8, device="cuda")
        got = wd.wdad_detect(x, det, reduce=False, inner=win[0], outer=win[1], precision=1, cond_gate=gate,
                             loading=loading, flags=flags).cpu().numpy()
        re = (flags.cpu().numpy().ravel()[pix] & 1).astype(bool)
        tol = np.where(re, 1e-6, np.maximum(TOL_SCORE, 1.5 * 2.0 ** -24 * kappa))
        want = oracle.detect(cube, det, win[0], win[1], loading=loading, pixels=pix)
        e = relerr(got.ravel()[pix], want)
        assert np.all(e <= tol), (det, e.max(), np.max(e / tol))
        # the gate bounds kappa from above by (|G|_F + delta) / delta: every pixel whose kappa is
        # above the gate is re-solved; at loading 1e-3 kappa here is ~1e5 and the bound stays
        # below 1 + 1e3 L, so a 1e6 gate re-solves nothing
        assert re[kappa > gate].all()
        if loading == 1e-3 and gate >= 1e6:
            assert not re.any()


@pytest.fixture(scope="module")
def ar1_1024(wd):
    # the precision workload at full size: 1024 x 1024 x 224 with band-to-band AR(1) noise
    # (rho 0.98); 160 sampled pixels, every eighth implanted one and three corners
    from paper_1201_2025_gb300 import synth
    sc = synth.make_scene(1024, 1024, 224, seed=3, n_anom=400, anom_side=(1, 3), abundance=(0.1, 0.5), margin=10,
                          ar_rho=0.98)
    rng = np.random.default_rng(1024)
    pix = np.unique(np.concatenate([rng.choice(1024 * 1024, 160, replace=False), np.flatnonzero(sc.mask)[::8],
                                    [0, 1023, 1024 * 1024 - 1]]))
    return sc, sc.cube.astype(np.float64), _gpu(sc.cube), pix


def test_mixed_full_size_ar1_sampled(wd, ar1_1024):
    # window (3,11), N = 112 < L: MIXED LRX and DWRX on every pixel take the FP32 sample-Gram
    # form (FP32 bar max(1e-4, 1.5 u kappa) as in the full-band tests, 1e-6 where re-solved)
    from parity import TOL_SCORE, relerr
    sc, c64, x, pix = ar1_1024
    _, aux = oracle.detect(c64, 0, 3, 11, pixels=pix, want_aux=True, want_cond=True)
    kappa = aux[..., 1] / aux[..., 0]
    for det in (0, 1):
        flags = torch.zeros((1024, 1024), dtype=torch.uint8, device="cuda")
        got = wd.wdad_detect(x, det, reduce=False, inner=3, outer=11, precision=1, flags=flags)
        got = got.cpu().numpy().ravel()[pix]
        re = (flags.cpu().numpy().ravel()[pix] & 1).astype(bool)
        tol = np.where(re, 1e-6, np.maximum(TOL_SCORE, 1.5 * 2.0 ** -24 * kappa))
        e = relerr(got, oracle.detect(c64, det, 3, 11, pixels=pix))
        assert np.all(e <= tol), (det, e.max(), np.max(e / tol))


def test_mixed_full_size_ar1_wide_window(wd, ar1_1024):
    # window (7,21), N = 392 >= L: the BF16 tensor-core Gram and the FP32 L x L solve on every
    # pixel.  Against the detector's definition on the BF16-rounded centred samples the FP32
    # bar max(1e-4, 0.25 u kappa) holds; against the oracle on the unrounded data, 4 u kappa
    # (the bars and their measurements are derived in test_gpu_fullband_wide.py)
    from parity import bf16_data_score, relerr
    sc, c64, x, pix = ar1_1024
    _, aux = oracle.detect(c64, 0, 7, 21, pixels=pix, want_aux=True, want_cond=True)
    kappa = aux[..., 1] / aux[..., 0]
    u = 2.0 ** -24
    sub = pix[::4]
    ksub = kappa[::4]
    for det in (0, 1):
        flags = torch.zeros((1024, 1024), dtype=torch.uint8, device="cuda")
        got = wd.wdad_detect(x, det, reduce=False, inner=7, outer=21, precision=1, flags=flags)
        got = got.cpu().numpy().ravel()
        assert not (flags.cpu().numpy().ravel()[pix] & 1).any()  # kappa <= 1 + 1e3 L < 1e6: nothing gated
        e0 = relerr(got[pix], oracle.detect(c64, det, 7, 21, pixels=pix))
        assert np.all(e0 <= 4.0 * u * kappa), (det, e0.max(), np.max(e0 / (u * kappa)))
        ref = np.array([bf16_data_score(sc.cube, p, det, 7, 21) for p in sub])
        e = relerr(got[sub], ref)
        assert np.all(e <= np.maximum(1e-4, 0.25 * u * ksub)), (det, e.max(), np.max(e / (u * ksub)))
