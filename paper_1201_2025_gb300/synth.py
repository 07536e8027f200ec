"""Seeded synthetic hyperspectral cubes shaped like the paper's AVIRIS scenes.

The AVIRIS San Diego scenes of Sec. 5.1 are not available, so every workload is
drawn from this generator instead.  It holds none of the detection method's
arithmetic: it only builds inputs, and both the CUDA path and the CPU oracle
consume what it returns.

Model (linear mixing with implanted sub-pixel targets, Eq. 10):

* endmembers: 5 background spectra and 1 anomaly spectrum, each the sum of
  three Gaussian bumps over the band index (centre U(0, L), width U(L/20, L/4),
  amplitude U(0.2, 1)), then mapped affinely onto reflectance [0.05, 0.6];
* background pixel = Dirichlet(alpha=1) mixture of the 5 background endmembers;
* anomaly pixel z = f*t + (1-f)*b (Eq. 10) with t the anomaly endmember;
* additive noise, iid N(0, sigma^2) per band, or band-correlated AR(1)
  (stationary variance sigma^2, lag-one correlation rho) for ill-conditioned
  covariances.

All arithmetic is plain elementwise float64 (no BLAS), so a seed gives the same
float32 cube on any machine up to the platform's exp().
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Scene:
    cube: np.ndarray  # [H][W][L] float32, band-interleaved-by-pixel
    mask: np.ndarray  # [H][W] uint8, 1 where an anomaly was implanted
    endmembers: np.ndarray  # [6][L] float64 (last row is the anomaly spectrum)
    abundance: np.ndarray  # [H][W] float64 anomaly fraction f (0 for background)


def endmember_spectra(rng: np.random.Generator, L: int, n: int = 6) -> np.ndarray:
    """n smooth spectra over L bands, each mapped onto reflectance [0.05, 0.6]."""
    band = np.arange(L, dtype=np.float64)
    out = np.empty((n, L), dtype=np.float64)
    for e in range(n):
        s = np.zeros(L, dtype=np.float64)
        for _ in range(3):
            c = rng.uniform(0.0, L)
            w = rng.uniform(L / 20.0, L / 4.0)
            a = rng.uniform(0.2, 1.0)
            s = s + a * np.exp(-0.5 * ((band - c) / w) ** 2)
        lo, hi = s.min(), s.max()
        span = hi - lo if hi > lo else 1.0
        out[e] = 0.05 + 0.55 * (s - lo) / span
    return out


def _noise(rng: np.random.Generator, shape, sigma: float, ar_rho: float) -> np.ndarray:
    e = rng.standard_normal(shape).astype(np.float64)
    if ar_rho == 0.0:
        return sigma * e
    # stationary AR(1) along the band axis: n[0] ~ N(0, s^2), n[l] = rho n[l-1] + sqrt(1-rho^2) s e[l]
    out = np.empty(shape, dtype=np.float64)
    out[..., 0] = sigma * e[..., 0]
    k = np.sqrt(1.0 - ar_rho * ar_rho) * sigma
    for l in range(1, shape[-1]):
        out[..., l] = ar_rho * out[..., l - 1] + k * e[..., l]
    return out


def adjacency_fraction(frac: np.ndarray, w: float) -> np.ndarray:
    """Eq. 11: background pixels within one pixel of a target (the 8-neighbourhood ring) take
    the target spectrum with weight exp(-rho^2 / w^2) f, rho their distance to the target pixel
    and f its abundance (the largest such weight over neighbouring target pixels).  Returns the
    effective fraction map: frac on targets, that weight on the ring, 0 elsewhere."""
    H, W = frac.shape
    g = np.zeros_like(frac)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            sh = np.zeros_like(frac)
            ys, yd = (slice(max(dy, 0), H + min(dy, 0)), slice(max(-dy, 0), H + min(-dy, 0)))
            xs, xd = (slice(max(dx, 0), W + min(dx, 0)), slice(max(-dx, 0), W + min(-dx, 0)))
            sh[yd, xd] = frac[ys, xs]  # abundance of the target pixel at offset (dy, dx)
            g = np.maximum(g, np.exp(-(dy * dy + dx * dx) / (w * w)) * sh)
    return np.where(frac > 0, frac, g)


def make_scene(H: int, W: int, L: int, seed: int = 0, *, n_anom: int = 10,
               anom_side=(2, 2), abundance=(0.3, 0.3), margin: int = 6,
               sigma: float = 0.005, ar_rho: float = 0.0, adjacency_w: float | None = None,
               row_block: int = 256) -> Scene:
    """Draw one scene.  anom_side=(a, b) draws square targets of side U{a..b};
    abundance=(lo, hi) draws f ~ U(lo, hi) per target (lo == hi: fixed); adjacency_w > 0 adds
    the adjacency effect of Eq. 11 with that width on the ring around the targets (the truth
    mask stays the target pixels).  No random numbers are drawn for the adjacency effect, so a
    seed gives the same targets and background with and without it."""
    rng = np.random.default_rng(seed)
    E = endmember_spectra(rng, L, 6)
    frac = np.zeros((H, W), dtype=np.float64)
    for _ in range(n_anom):
        side = int(rng.integers(anom_side[0], anom_side[1] + 1))
        f = float(abundance[0]) if abundance[0] == abundance[1] else float(rng.uniform(*abundance))
        lo_y, hi_y = margin, max(margin, H - margin - side)
        lo_x, hi_x = margin, max(margin, W - margin - side)
        y0 = int(rng.integers(lo_y, hi_y + 1))
        x0 = int(rng.integers(lo_x, hi_x + 1))
        frac[y0:y0 + side, x0:x0 + side] = f
    eff = adjacency_fraction(frac, adjacency_w) if adjacency_w else frac
    cube = np.empty((H, W, L), dtype=np.float32)
    # rows are drawn block by block so large cubes never need a float64 copy
    for r0 in range(0, H, row_block):
        r1 = min(H, r0 + row_block)
        ab = rng.dirichlet(np.ones(5), size=(r1 - r0, W))  # [rows][W][5]
        b = np.zeros((r1 - r0, W, L), dtype=np.float64)
        for k in range(5):
            b += ab[..., k:k + 1] * E[k][None, None, :]
        f = eff[r0:r1, :, None]
        z = f * E[5][None, None, :] + (1.0 - f) * b  # Eq. 10 / Eq. 11 (identity where f == 0)
        z += _noise(rng, (r1 - r0, W, L), sigma, ar_rho)
        cube[r0:r1] = z.astype(np.float32)
    return Scene(cube=cube, mask=(frac > 0).astype(np.uint8), endmembers=E, abundance=frac)


def make_scene_device(H: int, W: int, L: int, seed: int = 0, *, n_anom: int = 10, anom_side=(2, 2),
                      abundance=(0.3, 0.3), margin: int = 6, sigma: float = 0.005, device="cuda",
                      row_block: int = 256):
    """The same model as make_scene, drawn on a CUDA device for the large bench workloads.

    Endmembers and target placement come from numpy's generator exactly as in make_scene;
    the per-pixel Dirichlet(1) abundances (normalised Exp(1) draws) and the noise come from a
    torch generator on the device seeded with `seed`, so the cube is not the one make_scene
    returns for the same seed, only a draw from the same distribution.
    Returns (cube [H][W][L] float32 tensor on `device`, mask [H][W] uint8 numpy array)."""
    import torch
    rng = np.random.default_rng(seed)
    E = endmember_spectra(rng, L, 6)
    frac = np.zeros((H, W), dtype=np.float64)
    for _ in range(n_anom):
        side = int(rng.integers(anom_side[0], anom_side[1] + 1))
        f = float(abundance[0]) if abundance[0] == abundance[1] else float(rng.uniform(*abundance))
        y0 = int(rng.integers(margin, max(margin, H - margin - side) + 1))
        x0 = int(rng.integers(margin, max(margin, W - margin - side) + 1))
        frac[y0:y0 + side, x0:x0 + side] = f
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Ed = torch.from_numpy(E).to(device)
    fd = torch.from_numpy(frac).to(device)
    cube = torch.empty((H, W, L), device=device, dtype=torch.float32)
    for r0 in range(0, H, row_block):
        r1 = min(H, r0 + row_block)
        u = torch.rand((r1 - r0, W, 5), generator=g, device=device, dtype=torch.float64)
        e = -torch.log1p(-u)
        ab = e / e.sum(-1, keepdim=True)
        b = torch.einsum("hwk,kl->hwl", ab, Ed[:5])
        f = fd[r0:r1, :, None]
        z = f * Ed[5][None, None, :] + (1.0 - f) * b  # Eq. 10 (identity where f == 0)
        z += sigma * torch.randn((r1 - r0, W, L), generator=g, device=device, dtype=torch.float64)
        cube[r0:r1] = z.float()
    return cube, (frac > 0).astype(np.uint8)


# Workloads, named for what they are.
def scene_48x48(seed: int = 0) -> Scene:
    """48x48x224, ten 2x2 targets at abundance 0.3, >= 6 px from the border."""
    return make_scene(48, 48, 224, seed, n_anom=10, anom_side=(2, 2), abundance=(0.3, 0.3), margin=6)


def scene_512x512(seed: int = 0) -> Scene:
    """512x512x224, 200 targets of side 1-3 px at abundance U(0.1, 0.5)."""
    return make_scene(512, 512, 224, seed, n_anom=200, anom_side=(1, 3), abundance=(0.1, 0.5), margin=10)


def scene_ar1(H: int = 1024, W: int = 1024, L: int = 224, seed: int = 0, rho: float = 0.98) -> Scene:
    """Band-correlated AR(1) noise (ill-conditioned covariances)."""
    return make_scene(H, W, L, seed, n_anom=max(1, H * W // 5000), anom_side=(1, 3),
                      abundance=(0.1, 0.5), margin=10, ar_rho=rho)


def batch_specs(n: int = 64, seed: int = 0, side_lo: int = 128, side_hi: int = 1024):
    """Uneven batch: side U{side_lo..side_hi}, L in {128,188,224}, windows and detectors mixed."""
    rng = np.random.default_rng(seed)
    wins = [(3, 9), (5, 15), (7, 21)]
    out = []
    for i in range(n):
        side = int(rng.integers(side_lo, side_hi + 1))
        L = int(rng.choice([128, 188, 224]))
        w = wins[int(rng.integers(0, 3))]
        det = int(rng.integers(0, 3))
        out.append(dict(H=side, W=side, L=L, inner=w[0], outer=w[1], detector=det, seed=1000 + i))
    return out
