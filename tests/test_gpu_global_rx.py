"""Global RX (Eq. 1: one mean and covariance for the whole image) on the GPU against the FP64
oracle, on the full-band and the DWT-reduced cube, through the C ABI."""
import numpy as np
import pytest

import oracle
from parity import TOL_SCORE, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def wd():
    from paper_1201_2025_gb300 import wdad
    wdad.lib()
    return wdad


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _check(wd, cube, reduce, loading=1e-3, taps=8):
    got = wd.wdad_global_rx(_gpu(cube), reduce=reduce, loading=loading, wavelet_taps=taps).cpu().numpy()
    c = oracle.dwt_approx(cube, taps=taps) if reduce else cube.astype(np.float64)
    want, kappa = oracle.global_rx(c, loading=loading, want_cond=True)
    # FP32 bar of the arithmetic: the covariance and its inverse are held in FP32, so a score
    # carries a relative error up to ~ c u kappa (c = 32), and never less than the FP32 bar
    tol = max(TOL_SCORE, 32 * U32 * kappa)
    e = relerr(got, want)
    assert e.max() <= tol, (e.max(), tol, kappa)
    return got, want


def test_global_rx_scene48_full_band(wd):
    from paper_1201_2025_gb300 import synth
    sc = synth.scene_48x48(0)
    got, want = _check(wd, sc.cube, reduce=False)
    # the implanted targets stand out: the top 40 scores hold most of them
    top = np.argsort(-got.ravel())[:40]
    assert sc.mask.ravel()[top].mean() > 0.5


@pytest.mark.parametrize("taps", [8, 4, 12])
def test_global_rx_scene48_reduced(wd, taps):
    from paper_1201_2025_gb300 import synth
    sc = synth.scene_48x48(0)
    _check(wd, sc.cube, reduce=True, taps=taps)


@pytest.mark.parametrize("shape", [(21, 26, 13), (9, 40, 37), (30, 31, 97), (17, 19, 257), (33, 35, 300),
                                   (40, 40, 600), (1, 700, 5), (3, 3, 1)])
def test_global_rx_band_counts(wd, shape):
    # every score-kernel width (1-32 rows per lane), the inverse in shared and in global memory
    rng = np.random.default_rng(shape[2])
    L = shape[2]
    mix = np.eye(L) + 0.2 * rng.standard_normal((L, L)) / np.sqrt(L)
    cube = (0.3 * rng.standard_normal(shape) @ mix + 1.0).astype(np.float32)
    _check(wd, cube, reduce=False)


def test_global_rx_512_sampled(wd):
    from paper_1201_2025_gb300 import synth
    sc = synth.scene_512x512(0)
    got, want = _check(wd, sc.cube, reduce=False)
    again = wd.wdad_global_rx(_gpu(sc.cube), reduce=False).cpu().numpy()
    assert np.array_equal(got, again)  # fixed summation orders: run to run identical


def test_global_rx_degenerate(wd):
    # one pixel: zero covariance, zero loading -> not positive definite -> NaN
    one = wd.wdad_global_rx(_gpu(np.ones((1, 1, 6))), reduce=False).cpu().numpy()
    assert np.isnan(one).all()
    # fewer pixels than bands and no loading: singular covariance -> NaN everywhere
    rng = np.random.default_rng(0)
    few = wd.wdad_global_rx(_gpu(rng.standard_normal((2, 3, 12))), reduce=False, loading=0.0).cpu().numpy()
    assert np.isnan(few).all()
    # the same with loading is well posed and matches the oracle
    _check(wd, rng.standard_normal((2, 3, 12)).astype(np.float32), reduce=False, loading=1e-2)
    assert wd.wdad_global_rx(torch.empty((0, 4, 9), device="cuda"), reduce=False).shape == (0, 4)
    with pytest.raises(wd.WdadError) as ei:
        wd.wdad_global_rx(torch.ones((2, 2, 1025), device="cuda"), reduce=False)
    assert ei.value.status == wd.WDAD_ERR_UNSUPPORTED
