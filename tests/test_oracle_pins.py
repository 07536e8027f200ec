"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a published
table, a closed form, an invariance, an exact finite-sample distribution, a
library routine on a tiny case, or a hand-enumerated window.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(float(line))
    return np.array(vals)


# ---------------------------------------------------------------- filters (Sec. 3, Sec. 4)
def test_db4_matches_published_table():
    h = oracle.daub_filter(8)
    np.testing.assert_allclose(h, _table("db4_table.txt"), rtol=0, atol=2e-15)


def test_d4_closed_form():
    s3, r = math.sqrt(3.0), 4.0 * math.sqrt(2.0)
    want = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / r
    np.testing.assert_allclose(oracle.daub_filter(4), want, rtol=0, atol=1e-15)


def test_haar_closed_form():
    np.testing.assert_allclose(oracle.daub_filter(2), [1 / math.sqrt(2)] * 2, atol=1e-15)


@pytest.mark.parametrize("taps", [2, 4, 6, 8, 10, 12, 16, 20])
def test_filter_identities(taps):
    h = oracle.daub_filter(taps)
    n = np.arange(taps)
    assert abs(h.sum() - math.sqrt(2)) < 1e-13
    for m in range(taps // 2):  # double-shift orthonormality
        v = np.dot(h[: taps - 2 * m], h[2 * m:])
        assert abs(v - (1.0 if m == 0 else 0.0)) < 1e-12, (m, v)
    for p in range(taps // 2):  # vanishing moments of the wavelet filter
        assert abs(np.sum((-1.0) ** n * n ** p * h)) < 1e-9 * max(1, taps ** p), p
    g = oracle.highpass(h)
    assert abs(np.dot(h, g)) < 1e-14


# ---------------------------------------------------------------- transform (Eq. 9, Fig. 1)
def test_eq9_phase_with_haar():
    # Eq. 9 literally: a[k] = h0 x[2k] + h1 x[2k-1] (periodic), so a[0] pairs x[0] with x[M-1].
    x = np.arange(1.0, 9.0)
    a = oracle.dwt_step(x, oracle.daub_filter(2))
    want = np.array([x[0] + x[7], x[2] + x[1], x[4] + x[3], x[6] + x[5]]) / math.sqrt(2)
    np.testing.assert_allclose(a, want, atol=1e-14)


def test_odd_length_pads_last_sample():
    x = np.array([1.0, 2.0, 3.0])  # padded to [1,2,3,3]
    a = oracle.dwt_step(x, oracle.daub_filter(2))
    np.testing.assert_allclose(a, np.array([1 + 3, 3 + 2]) / math.sqrt(2), atol=1e-14)


@pytest.mark.parametrize("L", [64, 128, 256, 224, 188, 189, 7, 5])
@pytest.mark.parametrize("taps", [2, 4, 6, 8, 12, 20])
def test_perfect_reconstruction(L, taps):
    x = np.random.default_rng(L + taps).standard_normal(L)
    c = oracle.dwt_full(x, taps)
    np.testing.assert_allclose(oracle.dwt_inverse(c, L, taps), x, atol=1e-12)


@pytest.mark.parametrize("taps", [2, 4, 8, 12, 20])
def test_full_dwt_is_orthogonal_for_power_of_two(taps):
    L = 128
    Wm = np.stack([oracle.dwt_full(e, taps) for e in np.eye(L)], axis=1)
    assert Wm.shape == (L, L)
    np.testing.assert_allclose(Wm @ Wm.T, np.eye(L), atol=1e-13)
    x = np.random.default_rng(3).standard_normal(L)
    assert abs(np.sum(oracle.dwt_full(x, taps) ** 2) - np.sum(x ** 2)) < 1e-11  # Parseval


def test_levels_rule():
    # Sec. 4: decompose "until four samples are left"
    assert oracle.dwt_levels(224) == (6, 4)
    assert oracle.dwt_levels(128) == (5, 4)
    assert oracle.dwt_levels(188) == (6, 3)
    assert oracle.dwt_levels(189) == (6, 3)
    assert oracle.dwt_levels(4) == (0, 4)
    assert oracle.dwt_levels(224, 3) == (3, 28)


@pytest.mark.parametrize("L", [224, 188, 128, 97])
def test_constant_spectrum(L):
    # sum h = sqrt(2): a constant spectrum maps to constant * 2^(J/2) at every position
    J, K = oracle.dwt_levels(L)
    cube = np.full((2, 3, L), 0.3, np.float32)
    a = oracle.dwt_approx(cube)
    np.testing.assert_allclose(a, np.float64(np.float32(0.3)) * 2 ** (J / 2), rtol=1e-13)


def test_approximation_is_linear_map_with_orthonormal_rows():
    L = 128
    A = oracle.dwt_approx(np.eye(L, dtype=np.float32).reshape(L, 1, L)).reshape(L, -1).T
    np.testing.assert_allclose(A @ A.T, np.eye(A.shape[0]), atol=1e-13)
    x = np.random.default_rng(0).standard_normal((5, L)).astype(np.float32)
    np.testing.assert_allclose(oracle.dwt_approx(x[:, None, :])[:, 0, :], x.astype(np.float64) @ A.T, atol=1e-12)


def test_smooth_spectrum_has_no_first_level_detail():
    # 4 vanishing moments: the high-pass response falls like w^8 in energy, so a slow periodic
    # spectrum leaves (almost) nothing in d_1, the last L/2 coefficients of [a_J, d_J, ..., d_1]
    L = 128
    x = np.cos(2 * np.pi * np.arange(L) / L)
    c = oracle.dwt_full(x, 8)
    assert np.sum(c[-L // 2:] ** 2) < 1e-9 * np.sum(x ** 2)
    c4 = oracle.dwt_full(x, 4)  # two vanishing moments: w^4, a much weaker bound
    assert 1e-9 * np.sum(x ** 2) < np.sum(c4[-L // 2:] ** 2) < 1e-4 * np.sum(x ** 2)


# ---------------------------------------------------------------- windows (Sec. 2.2, Sec. 5.2)
def test_reflect101():
    assert [oracle.reflect(i, 5) for i in range(-4, 9)] == [4, 3, 2, 1, 0, 1, 2, 3, 4, 3, 2, 1, 0]
    assert oracle.reflect(-7, 1) == 0 and oracle.reflect(3, 2) == 1


def test_window_census_hand_enumerated_corner():
    # 4x4 image, pixel (0,0), inner 1, outer 3: reflected neighbours (1,1)x4, (1,0)x2, (0,1)x2
    c = oracle.window_census(4, 4, 1, 3, pixels=[0])[0]
    assert list(c) == [8, 4 * 5 + 2 * 4 + 2 * 1, 4 * 25 + 2 * 16 + 2 * 1, 1, 0, 0]


def test_window_census_interior_closed_form():
    H, W, wi, wo = 30, 40, 3, 9
    ri, ro = wi // 2, wo // 2
    pix = [15 * W + 20, 10 * W + 10]
    got = oracle.window_census(H, W, wi, wo, pixels=pix)
    dd = [(dy, dx) for dy in range(-ro, ro + 1) for dx in range(-ro, ro + 1)]
    bg = [(dy, dx) for dy, dx in dd if max(abs(dy), abs(dx)) > ri]
    inn = [(dy, dx) for dy, dx in dd if max(abs(dy), abs(dx)) <= ri]
    for row, p in zip(got, pix):
        for (n, s, ss), lst in ((row[:3], bg), (row[3:], inn)):
            assert n == len(lst) and s == len(lst) * p
            assert ss == len(lst) * p * p + sum((dy * W + dx) ** 2 for dy, dx in lst)
    assert got[0][0] == wo * wo - wi * wi


def test_window_moments_match_numpy_cov_on_explicit_windows():
    rng = np.random.default_rng(21)
    H, W, D = 9, 12, 5
    cube = rng.standard_normal((H, W, D))
    pix = [0, 13, 57, H * W - 1]
    mu, cov = oracle.window_moments(cube, 3, 7, pix)
    for t, p in enumerate(pix):
        y, x = divmod(p, W)
        bg = [cube[oracle.reflect(y + dy, H), oracle.reflect(x + dx, W)]
              for dy in range(-3, 4) for dx in range(-3, 4) if max(abs(dy), abs(dx)) > 1]
        bg = np.array(bg)
        np.testing.assert_allclose(mu[t], bg.mean(0), atol=1e-13)
        np.testing.assert_allclose(cov[t], np.cov(bg.T, bias=True), atol=1e-12)


def test_valid_border_mode_gives_nan():
    cube = np.random.default_rng(0).standard_normal((12, 12, 3))
    s = oracle.detect(cube, 0, 1, 5, border=1)
    assert np.isnan(s[:2]).all() and np.isnan(s[:, -2:]).all() and np.isfinite(s[2:-2, 2:-2]).all()


# ---------------------------------------------------------------- detectors (Eq. 1-5)
def _brute(cube, y, x, wi, wo, loading):
    """Brute force with library primitives: explicit window lists, np.cov, np.linalg.inv/eigh."""
    H, W, D = cube.shape
    ri, ro = wi // 2, wo // 2
    bg, inn = [], []
    for dy in range(-ro, ro + 1):
        for dx in range(-ro, ro + 1):
            v = cube[oracle.reflect(y + dy, H), oracle.reflect(x + dx, W)]
            (inn if max(abs(dy), abs(dx)) <= ri else bg).append(v)
    bg, inn = np.array(bg), np.array(inn)
    mo, mi = bg.mean(0), inn.mean(0)
    Co = np.atleast_2d(np.cov(bg.T, bias=True))
    Ci = np.atleast_2d(np.cov(inn.T, bias=True)) if len(inn) > 1 else np.zeros((D, D))
    Cl = Co + loading * np.trace(Co) / D * np.eye(D)
    inv = np.linalg.inv(Cl)
    lrx = (cube[y, x] - mo) @ inv @ (cube[y, x] - mo)
    dwrx = abs((mi - mo) @ inv @ (mi - mo))
    lam, V = np.linalg.eigh(Ci - Co)
    tau = 1e-6 * np.abs(lam).max()
    sel = lam > tau
    acc = 0.0
    for k in np.nonzero(sel)[0]:
        v = V[:, k]
        v = v if v[np.argmax(np.abs(v))] >= 0 else -v
        acc += v @ (mi - mo)
    dwest1 = np.linalg.norm(V[:, sel].T @ (mi - mo))
    return lrx, dwrx, abs(acc), dwest1


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("win", [(1, 5), (3, 5), (3, 7)])
def test_detectors_match_brute_force(D, win):
    rng = np.random.default_rng(D * 10 + win[0])
    H, W = 9, 11
    cube = rng.standard_normal((H, W, D)) @ rng.standard_normal((D, D)) + rng.standard_normal(D)
    wi, wo = win
    pix = [0, 5, W * 4 + 5, H * W - 1, W * 8 + 3]
    got = [oracle.detect(cube, det, wi, wo, loading=1e-3, pixels=pix, dwest_mode=m)
           for det, m in ((0, 0), (1, 0), (2, 0), (2, 1))]
    for t, p in enumerate(pix):
        want = _brute(cube, p // W, p % W, wi, wo, 1e-3)
        for g, w in zip(got, want):
            assert abs(g[t] - w) <= 1e-10 * max(1.0, abs(w)), (t, g[t], w)


def test_affine_invariance_without_loading():
    rng = np.random.default_rng(7)
    H, W, D = 16, 16, 4
    x = rng.standard_normal((H, W, D))
    B = rng.standard_normal((D, D)) + 3 * np.eye(D)
    y = x @ B.T + rng.standard_normal(D)
    for det in (0, 1):
        a = oracle.detect(x, det, 3, 9, loading=0.0)
        b = oracle.detect(y, det, 3, 9, loading=0.0)
        np.testing.assert_allclose(a, b, rtol=1e-8)


def test_similarity_invariance_with_trace_loading():
    rng = np.random.default_rng(8)
    H, W, D = 16, 16, 5
    x = rng.standard_normal((H, W, D))
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    y = 2.5 * x @ Q.T + rng.standard_normal(D)
    for det in (0, 1):
        np.testing.assert_allclose(oracle.detect(x, det, 3, 9, loading=1e-2),
                                   oracle.detect(y, det, 3, 9, loading=1e-2), rtol=1e-9)
    # DWEST projection-norm form is unchanged by a rotation of the bands (Eq. 4 up to sign)
    np.testing.assert_allclose(oracle.detect(x, 2, 3, 9, dwest_mode=1),
                               oracle.detect(x @ Q.T, 2, 3, 9, dwest_mode=1), rtol=1e-8)


def test_orthogonal_dwt_leaves_scores_unchanged():
    # all detectors are unchanged when every spectrum goes through the full orthogonal DWT (L=128)
    rng = np.random.default_rng(9)
    L = 16
    x = rng.standard_normal((10, 10, L))
    Wm = np.stack([oracle.dwt_full(e, 8) for e in np.eye(L)], axis=1)
    y = x @ Wm.T
    for det, m in ((0, 0), (1, 0), (2, 1)):
        np.testing.assert_allclose(oracle.detect(x, det, 3, 5, loading=1e-3, dwest_mode=m),
                                   oracle.detect(y, det, 3, 5, loading=1e-3, dwest_mode=m), rtol=1e-7)


def _f_ks(vals, d1, d2):
    from scipy import stats
    return stats.kstest(vals, stats.f(d1, d2).cdf).pvalue


@pytest.mark.parametrize("D,wi,wo", [(4, 3, 9), (3, 1, 7)])
def test_lrx_finite_sample_f_distribution(D, wi, wo):
    # iid Gaussian background, no loading: LRX (N-D)/(D(N+1)) ~ F(D, N-D) (Hotelling T^2)
    rng = np.random.default_rng(11)
    step = wo
    H = W = step * 48
    x = rng.standard_normal((H, W, D))
    N = wo * wo - wi * wi
    ys = np.arange(wo // 2, H - wo // 2, step)
    pix = (ys[:, None] * W + ys[None, :]).ravel()
    s = oracle.detect(x, 0, wi, wo, loading=0.0, pixels=pix)
    assert _f_ks(s * (N - D) / (D * (N + 1)), D, N - D) > 1e-3
    # a dropped "+1" (the test pixel's own variance) or 1/(N-1) normalisation must be rejected
    assert _f_ks(s * (N - D) / (D * N) * 1.2, D, N - D) < 1e-3


@pytest.mark.parametrize("D,wi,wo", [(4, 3, 9), (2, 5, 11)])
def test_dwrx_finite_sample_f_distribution(D, wi, wo):
    # DWRX c (N-D)/(D N) ~ F(D, N-D) with c = 1/(1/n_i + 1/N)
    rng = np.random.default_rng(12)
    H = W = wo * 48
    x = rng.standard_normal((H, W, D))
    N, ni = wo * wo - wi * wi, wi * wi
    ys = np.arange(wo // 2, H - wo // 2, wo)
    pix = (ys[:, None] * W + ys[None, :]).ravel()
    s = oracle.detect(x, 1, wi, wo, loading=0.0, pixels=pix)
    c = 1.0 / (1.0 / ni + 1.0 / N)
    assert _f_ks(s * c * (N - D) / (D * N), D, N - D) > 1e-3
    assert _f_ks(s * (N - D) / (D * N), D, N - D) < 1e-3


def test_dwest_one_band_closed_form():
    rng = np.random.default_rng(13)
    x = rng.standard_normal((12, 12, 1)) * rng.uniform(0.5, 2.0, (12, 12, 1))
    s = oracle.detect(x, 2, 3, 7)
    for y in range(3, 9):
        for xx in range(3, 9):
            inn = x[y - 1:y + 2, xx - 1:xx + 2, 0].ravel()
            out = np.concatenate([x[y - 3:y + 4, xx - 3:xx + 4, 0].ravel()])
            blk = x[y - 3:y + 4, xx - 3:xx + 4, 0].copy()
            blk[2:5, 2:5] = np.nan
            bg = blk[~np.isnan(blk)]
            want = abs(inn.mean() - bg.mean()) if inn.var() - bg.var() > 0 else 0.0
            assert abs(s[y, xx] - want) < 1e-12, (y, xx)
            del out


def test_inner_one_dwrx_equals_lrx_and_dwest_zero():
    rng = np.random.default_rng(14)
    x = rng.standard_normal((10, 10, 3))
    np.testing.assert_allclose(oracle.detect(x, 1, 1, 5), oracle.detect(x, 0, 1, 5), rtol=1e-12)
    assert np.all(oracle.detect(x, 2, 1, 5) == 0.0)


def test_loading_zero_singular_background_is_nan():
    # fewer background samples than bands and no loading: C_o is singular, Cholesky fails
    x = np.random.default_rng(15).standard_normal((8, 8, 12))
    s = oracle.detect(x, 0, 1, 3, loading=0.0)
    assert np.isnan(s).all()


# ---------------------------------------------------------------- evaluation (Sec. 5.3.1)
def test_auc_against_sklearn_and_special_cases():
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(16)
    s = np.round(rng.standard_normal(3000), 1)  # many ties
    m = (rng.uniform(size=3000) < 0.1).astype(np.uint8)
    assert abs(oracle.auc(s, m) - skm.roc_auc_score(m, s)) < 1e-12
    assert oracle.auc(np.array([0.1, 0.2, 0.9, 1.0]), np.array([0, 0, 1, 1])) == 1.0
    assert oracle.auc(np.ones(10), np.array([0, 1] * 5)) == 0.5


# ---------------------------------------------------------------- screening CNN (addition, no paper counterpart)
def test_cnn_gradient_matches_central_differences():
    rng = np.random.default_rng(31)
    K = 4
    n = oracle.cnn_nparam(K)
    assert n == 4 * 25 * 32 + 32 + 2 * (32 * 25 * 32 + 32) + 32 * 9 + 1
    params = rng.standard_normal(n) * 0.05
    x = rng.standard_normal((1, 16, 17, K))
    t = rng.standard_normal((1, 16, 17))
    loss, g = oracle.cnn_grad(params, x, t)
    idx = rng.choice(n, 40, replace=False)
    idx = np.concatenate([idx, [n - 1, 0, 3232 - 1]])  # last bias, first weight, first layer's last bias
    h = 1e-5
    for i in idx:
        pp = params.copy(); pp[i] += h
        lp, _ = oracle.cnn_grad(pp, x, t)
        pp[i] -= 2 * h
        lm, _ = oracle.cnn_grad(pp, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, fd, g[i])


def test_cnn_forward_is_linear_in_the_last_layer_and_zero_padding():
    # with every hidden weight zero, the output equals the last bias everywhere
    K = 4
    n = oracle.cnn_nparam(K)
    params = np.zeros(n)
    params[-1] = 0.75
    x = np.random.default_rng(32).standard_normal((2, 15, 15, K))
    np.testing.assert_allclose(oracle.cnn_forward(params, x), 0.75, atol=0)


def test_scene_whitening_is_the_unique_lower_triangular_whitener():
    # M C M^T = I with M lower triangular and a positive diagonal fixes M uniquely; the
    # whitened data has zero mean and identity (population) covariance
    rng = np.random.default_rng(33)
    for K in (1, 3, 4, 8):
        A = np.eye(K) + 0.5 * rng.standard_normal((K, K))
        x = 0.3 + rng.standard_normal((500, K)) @ A.T * 0.02
        mu, M = oracle.scene_whiten(x)
        C = np.cov(x.T, bias=True).reshape(K, K)
        np.testing.assert_allclose(mu, x.mean(0), rtol=1e-13)
        np.testing.assert_allclose(M @ C @ M.T, np.eye(K), atol=1e-9)
        assert np.all(np.triu(M, 1) == 0) and np.all(np.diag(M) > 0)
        z = (x - mu) @ M.T
        np.testing.assert_allclose(z.mean(0), 0, atol=1e-10)
        np.testing.assert_allclose(z.T @ z / len(z), np.eye(K), atol=1e-9)
    # K = 1: M = 1 / population standard deviation
    x = rng.standard_normal((77, 1))
    _, M = oracle.scene_whiten(x)
    assert abs(M[0, 0] - 1.0 / x.std()) <= 1e-12 / x.std()


def test_scene_whitening_degenerate_inputs_stay_finite():
    mu, M = oracle.scene_whiten(np.full((10, 4), 0.25))  # constant: trace 0 -> identity
    np.testing.assert_array_equal(M, np.eye(4))
    np.testing.assert_allclose(mu, 0.25)
    x = np.random.default_rng(34).standard_normal((50, 3))
    x[:, 1] = 2.0  # one constant band: its pivot is floored
    _, M = oracle.scene_whiten(x)
    assert np.isfinite(M).all()
    mu, M = oracle.scene_whiten(np.array([[1.0, 2.0]]))  # one pixel
    np.testing.assert_array_equal(M, np.eye(2))


def test_bf16_rounding_closed_forms():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2); halfway cases go to the even
    # neighbour
    assert oracle.bf16_round(1.0) == 1.0
    assert oracle.bf16_round(1.0 + 2.0 ** -8) == 1.0                      # tie -> even (1.0)
    assert oracle.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6       # tie -> even
    assert oracle.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7  # above the tie
    assert oracle.bf16_round(3.0) == 3.0 and oracle.bf16_round(0.0) == 0.0
    assert oracle.bf16_round(-1.0 - 3 * 2.0 ** -8) == -(1.0 + 2.0 ** -6)
    assert oracle.bf16_round(2.0 ** -130) == 0.0 or abs(oracle.bf16_round(2.0 ** -130)) < 2.0 ** -126


def test_cnn_bf16_activation_forward_bounds():
    K = 4
    n = oracle.cnn_nparam(K)
    rng = np.random.default_rng(35)
    params = rng.standard_normal(n) * 0.05
    x = rng.standard_normal((1, 12, 13, K))
    exact = oracle.cnn_forward(params, x)
    q = oracle.cnn_forward_bf16act(params, x)
    # rounding perturbs each rounded activation by at most 2^-8 relative; the output moves by
    # far less than the output scale, but does move
    assert 0 < np.abs(q - exact).max() <= 2.0 ** -6 * np.abs(exact).max()
    # identity when every rounded activation is already a bfloat16 value: all hidden weights
    # of layers 1 and 2 zero and bfloat16-exact biases
    p2 = params.copy()
    w1 = 4 * 25 * 32
    p2[:w1] = 0.0
    p2[w1:w1 + 32] = 0.25                                  # layer-1 biases (bfloat16-exact)
    o2 = w1 + 32
    p2[o2:o2 + 32 * 25 * 32] = 0.0
    p2[o2 + 32 * 25 * 32:o2 + 32 * 25 * 32 + 32] = 0.5    # layer-2 biases
    np.testing.assert_array_equal(oracle.cnn_forward_bf16act(p2, x), oracle.cnn_forward(p2, x))


# ---------------------------------------------------------------- adaptive threshold (Eq. 12)
def test_adaptive_threshold_worked_example():
    # scores 1..4: mean 2.5, population variance 1.25; z = 1 -> tau = 2.5 + sqrt(1.25)
    mu, sd, tau, mask = oracle.adaptive_threshold(np.array([1.0, 2.0, 3.0, 4.0]), 1.0)
    assert mu == 2.5 and abs(sd - np.sqrt(1.25)) < 1e-15 and abs(tau - (2.5 + np.sqrt(1.25))) < 1e-15
    assert mask.tolist() == [0, 0, 0, 1]
    # z = 0: the mean itself; equal scores are not above it
    _, _, tau0, mask0 = oracle.adaptive_threshold(np.array([1.0, 2.0, 2.5, 4.0, 3.0]), 0.0)
    assert tau0 == 2.5 and mask0.tolist() == [0, 0, 0, 1, 1]
    # NaN entries neither count nor get declared
    mu, sd, _, mask = oracle.adaptive_threshold(np.array([1.0, np.nan, 3.0]), 0.5)
    assert mu == 2.0 and sd == 1.0 and mask.tolist() == [0, 0, 1]


def test_adaptive_threshold_invariances_and_gaussian_rate():
    rng = np.random.default_rng(36)
    s = rng.standard_normal(200000)
    _, _, _, m = oracle.adaptive_threshold(s, 2.0)
    # shift and positive scale move tau with the scores: same decisions
    _, _, _, m2 = oracle.adaptive_threshold(3.0 * s + 7.0, 2.0)
    assert np.array_equal(m, m2)
    # Gaussian scores: the declared fraction is the upper tail 1 - Phi(z) (0.02275 at z = 2)
    from scipy.stats import norm
    assert abs(m.mean() - norm.sf(2.0)) < 4 * np.sqrt(norm.sf(2.0) / len(s))


# ---------------------------------------------------------------- global RX (Eq. 1)
def test_global_rx_trace_identity():
    # sum over the image of (x - mu)^T M^-1 (x - mu) = P tr(M^-1 C): P L without loading, and
    # P sum lambda / (lambda + delta) over the eigenvalues of C with it
    rng = np.random.default_rng(1)
    cube = rng.standard_normal((20, 25, 6)) @ (np.eye(6) + 0.4 * rng.standard_normal((6, 6))) + 3.0
    P = 500
    assert abs(oracle.global_rx(cube, loading=0.0).sum() - P * 6) < 1e-9 * P * 6
    X = cube.reshape(-1, 6)
    C = np.cov(X.T, bias=True)
    lam = np.linalg.eigvalsh(C)
    delta = 0.05 * lam.sum() / 6
    want = P * np.sum(lam / (lam + delta))
    assert abs(oracle.global_rx(cube, loading=0.05).sum() - want) < 1e-9 * want


def test_global_rx_affine_invariance():
    # without loading the score is invariant under any invertible affine band transform
    rng = np.random.default_rng(2)
    cube = rng.standard_normal((9, 11, 5))
    A = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    b = rng.standard_normal(5)
    np.testing.assert_allclose(oracle.global_rx(cube @ A.T + b, loading=0.0), oracle.global_rx(cube, loading=0.0),
                               rtol=1e-9)


def test_global_rx_chi_square_on_gaussian_background():
    # Gaussian pixels: the score follows chi-square with L degrees of freedom (Sec. 2.1), up to
    # the O(1/P) effect of the estimated mean and covariance
    from scipy import stats
    rng = np.random.default_rng(3)
    L, P = 5, 40000
    Sig = np.eye(L) + 0.5 * np.ones((L, L))
    X = rng.multivariate_normal(np.arange(L), Sig, size=P)
    s = oracle.global_rx(X.reshape(200, 200, L), loading=0.0).ravel()
    for q in (0.5, 0.9, 0.99):
        assert abs(np.quantile(s, q) / stats.chi2.ppf(q, L) - 1) < 0.03, q
    assert stats.kstest(s, "chi2", args=(L,)).statistic < 0.01


def test_global_rx_single_outlier_ranks_first():
    rng = np.random.default_rng(4)
    cube = 0.1 * rng.standard_normal((16, 16, 8)) + 1.0
    cube[5, 7] += 0.5 * rng.standard_normal(8)
    s = oracle.global_rx(cube)
    assert np.unravel_index(np.argmax(s), s.shape) == (5, 7)
