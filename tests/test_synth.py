"""The seeded input generator: the implant model of Eq. 10 and the adjacency effect of
Eq. 11, checked on noise-free scenes (CPU)."""
import numpy as np

from paper_1201_2025_gb300 import synth


def _convex_fit(E5, b):
    """Least squares b ~ c^T E5 with sum(c) = 1 (weighted row), c >= 0 (NNLS): (c, residual)."""
    from scipy.optimize import nnls
    A = np.vstack([E5.T, 1e3 * np.ones((1, E5.shape[0]))])
    y = np.concatenate([b, [1e3]])
    c, _ = nnls(A, y)
    return c, np.abs(E5.T @ c - b).max()


def test_implants_follow_eq10():
    # target pixel z = f t + (1 - f) b with b a Dirichlet mixture of the five background
    # endmembers: (z - f t) / (1 - f) must be an exact convex combination of them
    a = synth.make_scene(30, 32, 40, seed=5, n_anom=3, anom_side=(2, 2), abundance=(0.3, 0.3), margin=5, sigma=0.0)
    E = a.endmembers
    ys, xs = np.nonzero(a.mask)
    assert len(ys) > 0 and np.all(a.abundance[ys, xs] == 0.3)
    for y, x in zip(ys, xs):
        b = (a.cube[y, x].astype(np.float64) - 0.3 * E[5]) / 0.7
        c, res = _convex_fit(E[:5], b)
        assert res < 1e-6 and abs(c.sum() - 1.0) < 1e-6 and np.all(c >= 0)
    # negative control: the target spectrum itself is not such a mixture
    _, res = _convex_fit(E[:5], E[5])
    assert res > 1e-3


def test_adjacency_ring_follows_eq11():
    kw = dict(n_anom=4, anom_side=(1, 3), abundance=(0.2, 0.5), margin=5, sigma=0.0)
    plain = synth.make_scene(40, 44, 48, seed=9, **kw)
    adj = synth.make_scene(40, 44, 48, seed=9, adjacency_w=1.5, **kw)
    np.testing.assert_array_equal(plain.mask, adj.mask)
    t = adj.endmembers[5].astype(np.float64)
    frac = plain.abundance
    ring = 0
    for y in range(40):
        for x in range(44):
            if frac[y, x] > 0:
                np.testing.assert_array_equal(adj.cube[y, x], plain.cube[y, x])  # targets unchanged
                continue
            # Eq. 11 weight: exp(-rho^2 / w^2) f over the neighbouring target pixels (largest)
            g = 0.0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = y + dy, x + dx
                    if (dy or dx) and 0 <= yy < 40 and 0 <= xx < 44 and frac[yy, xx] > 0:
                        g = max(g, np.exp(-(dy * dy + dx * dx) / 1.5 ** 2) * frac[yy, xx])
            b = plain.cube[y, x].astype(np.float64)  # the pixel's own background (no noise)
            want = g * t + (1.0 - g) * b
            np.testing.assert_allclose(adj.cube[y, x], want, rtol=2e-7, atol=1e-7)
            ring += g > 0
    assert ring >= 8  # some background pixels were affected
