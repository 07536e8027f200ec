"""GPU parity of the full-band detectors (A3-A5 on the L-band cube) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from parity import TOL_SCORE, dwest_relerr, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24  # FP32 unit roundoff


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


def _sample(H, W, mask, n=96, seed=0):
    rng = np.random.default_rng(seed)
    pix = set(rng.choice(H * W, n, replace=False).tolist())
    pix |= {0, W - 1, (H - 1) * W, H * W - 1, (H // 2) * W + W // 2}
    pix |= set(np.flatnonzero(mask).tolist()[:8])
    return np.array(sorted(pix))


# FP32 full-band bar: max(1e-4, C_FP32 u kappa(C_o + delta I)) per pixel.  C_o (or the N x N
# sample Gram of the Woodbury form) is formed and factored in FP32, so the score carries a
# relative error of a multiple of u kappa.  Measured on GB300 over these tests' cases, the L x L
# form at 13-224 bands and the sample-Gram form at N = 8..200: at most 0.50 u kappa (37 bands,
# window 3/9), 0.45 (224 bands, 5/15 sample Gram), 0.30 (224 bands, 1/5, N = 24).  C_FP32 = 1.5
# leaves a factor of 3.
C_FP32 = 1.5


def _fp32_rx_tol(cube, det, win, pix):
    _, aux = oracle.detect(cube, det, win[0], win[1], pixels=pix, want_aux=True, want_cond=True)
    kappa = aux[..., 1] / aux[..., 0]
    return np.maximum(TOL_SCORE, C_FP32 * U32 * kappa)


@pytest.mark.parametrize("prec", [2, 0])
def test_fullband_scene48(wd, scene48, prec):
    cube = scene48.cube
    win = (3, 11)
    got = wd.wdad_detect_all(_gpu(cube), reduce=False, inner=win[0], outer=win[1], precision=prec).cpu().numpy()
    pix = _sample(48, 48, scene48.mask)
    c64 = cube.astype(np.float64)
    for det in (0, 1):
        want = oracle.detect(c64, det, win[0], win[1], pixels=pix)
        e = relerr(got[det].ravel()[pix], want)
        tol = 1e-6 if prec == 2 else _fp32_rx_tol(c64, det, win, pix)
        assert np.all(e <= tol), (det, e.max(), np.max(e / tol))
    want, aux = oracle.detect(c64, 2, win[0], win[1], pixels=pix, want_aux=True)
    e = dwest_relerr(got[2].ravel()[pix], want, aux)
    assert e.max() <= (1e-6 if prec == 2 else TOL_SCORE), e.max()


@pytest.mark.parametrize("D", [13, 37])
@pytest.mark.parametrize("prec", [2, 0])
def test_fullband_odd_band_counts(wd, D, prec):
    rng = np.random.default_rng(D)
    mix = np.eye(D) + 0.3 * rng.standard_normal((D, D))
    cube = (0.2 * rng.standard_normal((21, 26, D)) @ mix + 1.0).astype(np.float32)
    got = wd.wdad_detect_all(_gpu(cube), reduce=False, inner=3, outer=9, precision=prec).cpu().numpy()
    c64 = cube.astype(np.float64)
    for det in (0, 1):
        want = oracle.detect(c64, det, 3, 9)
        e = relerr(got[det], want)
        tol = 1e-6 if prec == 2 else _fp32_rx_tol(c64, det, (3, 9), None)
        assert np.all(e <= tol), (det, e.max())
    want, aux = oracle.detect(c64, 2, 3, 9, want_aux=True)
    e = dwest_relerr(got[2], want, aux)
    assert e.max() <= (1e-6 if prec == 2 else TOL_SCORE), e.max()


@pytest.mark.parametrize("prec", [2, 0])
def test_fullband_single_equals_fused(wd, prec):
    rng = np.random.default_rng(5)
    cube = (1.0 + 0.2 * rng.standard_normal((12, 17, 20))).astype(np.float32)
    x = _gpu(cube)
    allv = wd.wdad_detect_all(x, reduce=False, inner=3, outer=7, precision=prec).cpu().numpy()
    for det in range(3):
        one = wd.wdad_detect(x, det, reduce=False, inner=3, outer=7, precision=prec).cpu().numpy()
        assert np.array_equal(one, allv[det])


def test_fullband_valid_border_and_dwest_mode1(wd):
    rng = np.random.default_rng(6)
    cube = (1.0 + 0.2 * rng.standard_normal((15, 16, 11))).astype(np.float32)
    flags = torch.zeros((15, 16), dtype=torch.uint8, device="cuda")
    got = wd.wdad_detect_all(_gpu(cube), reduce=False, inner=1, outer=5, border=1, dwest_mode=1, precision=2,
                             flags=flags).cpu().numpy()
    f = flags.cpu().numpy()
    inv = np.ones((15, 16), bool)
    inv[2:-2, 2:-2] = False
    assert np.isnan(got[:, inv]).all() and np.all(f[inv] == 4) and np.isfinite(got[:, ~inv]).all()
    c64 = cube.astype(np.float64)
    for det in range(3):
        want, aux = oracle.detect(c64, det, 1, 5, border=1, dwest_mode=1, want_aux=True)
        if det < 2:
            assert relerr(got[det], want)[~inv].max() <= 1e-6
        else:
            assert dwest_relerr(got[det], want, aux)[~inv].max() <= 1e-6


@pytest.mark.parametrize("prec", [2, 0])
def test_fullband_singular_background_without_loading(wd, prec):
    # 8 background samples in 12 bands, no loading: C_o is singular -> NaN and flag bit 1
    rng = np.random.default_rng(7)
    cube = (1.0 + 0.2 * rng.standard_normal((10, 10, 12))).astype(np.float32)
    flags = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    got = wd.wdad_detect(_gpu(cube), 0, reduce=False, inner=1, outer=3, loading=0.0, precision=prec,
                         flags=flags).cpu().numpy()
    assert np.isnan(got).all() and np.all(flags.cpu().numpy() & 2)


def test_reduce_to_more_than_eight_coefficients_is_unsupported(wd, scene48):
    # the DWT kernel keeps at most 8 coefficients in registers; level 1 (K = 112) is refused
    x = _gpu(scene48.cube[:16, :16])
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_detect_all(x, reduce=True, level=1, inner=3, outer=7)
    assert ei.value.status == wd.WDAD_ERR_UNSUPPORTED


@pytest.mark.parametrize("D,win", [(37, (1, 3)), (61, (3, 7)), (130, (5, 11)), (224, (5, 15))])
@pytest.mark.parametrize("prec", [2, 0])
def test_fullband_fewer_samples_than_bands(wd, D, win, prec):
    # N = outer^2 - inner^2 < D: LRX and DWRX are solved at dimension N through the sample
    # Gram (Woodbury identity); the scores must match the oracle's D x D solve
    rng = np.random.default_rng(D + win[1])
    mix = np.eye(D) + 0.1 * rng.standard_normal((D, D))
    cube = (0.2 * rng.standard_normal((19, 23, D)) @ mix + 1.0).astype(np.float32)
    cube[9, 11] += 0.5 * rng.standard_normal(D).astype(np.float32)  # one outlier pixel
    got = wd.wdad_detect_all(_gpu(cube), reduce=False, inner=win[0], outer=win[1], precision=prec).cpu().numpy()
    c64 = cube.astype(np.float64)
    pix = _sample(19, 23, np.zeros((19, 23), bool), n=60, seed=D)
    for det in (0, 1):
        want = oracle.detect(c64, det, win[0], win[1], pixels=pix)
        e = relerr(got[det].ravel()[pix], want)
        tol = 1e-6 if prec == 2 else _fp32_rx_tol(c64, det, win, pix)
        assert np.all(e <= tol), (det, e.max(), np.max(e / tol))
    want, aux = oracle.detect(c64, 2, win[0], win[1], pixels=pix, want_aux=True)
    e = dwest_relerr(got[2].ravel()[pix], want, aux)
    assert e.max() <= (1e-6 if prec == 2 else TOL_SCORE), e.max()


def test_fullband_fewer_samples_valid_border_and_flags(wd):
    # the sample-Gram form with border = 1: NaN and flag bit 2 outside the valid region, the
    # oracle's scores inside
    rng = np.random.default_rng(12)
    cube = (0.2 * rng.standard_normal((18, 21, 64)) + 1.0).astype(np.float32)
    flags = torch.zeros((18, 21), dtype=torch.uint8, device="cuda")
    got = wd.wdad_detect_all(_gpu(cube), reduce=False, inner=3, outer=7, border=1, precision=0,
                             flags=flags).cpu().numpy()
    f = flags.cpu().numpy()
    inv = np.ones((18, 21), bool)
    inv[3:-3, 3:-3] = False
    assert np.isnan(got[:2, inv]).all() and np.all(f[inv] == 4)
    c64 = cube.astype(np.float64)
    for det in (0, 1):
        want = oracle.detect(c64, det, 3, 7, border=1)
        e = relerr(got[det], want)[~inv]
        tol = np.asarray(_fp32_rx_tol(c64, det, (3, 7), None)).reshape(18, 21)[~inv]
        assert np.all(e <= tol), (det, e.max())
