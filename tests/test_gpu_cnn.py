"""A9 learned screening: the CNN's forward and gradients against the FP64 oracle, training,
checkpoint/resume, and screened LRX against the exact detector."""
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


def bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)).view(np.float32)


def _batch(seed, B=2, H=24, W=26, K=4):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((B, H, W, K)).astype(np.float32), rng.standard_normal((B, H, W)).astype(np.float32))


@pytest.mark.parametrize("bf16,tol", [(False, 1e-4), (True, 1e-2)])
def test_gradients_match_fp64_oracle(wd, bf16, tol):
    net = wd.wdad_cnn(K=4, bf16_weights=bf16, seed=3)
    x, t = _batch(5)
    loss, g = net.grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    p = net.params().astype(np.float64)
    pf = bf16_round(p).astype(np.float64) if bf16 else p
    lo, go = oracle.cnn_grad(pf, x.astype(np.float64), t.astype(np.float64))
    # per-layer relative error of the gradient (norm-wise), and the loss
    n = [0, 3232, 3232 + 25632, 3232 + 2 * 25632, len(p)]
    for a, b in zip(n[:-1], n[1:]):
        err = np.linalg.norm(g[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert err <= tol, (a, err)
    assert abs(loss - lo) <= tol * abs(lo)
    net.close()


def test_forward_matches_fp64_oracle(wd):
    net = wd.wdad_cnn(K=4, bf16_weights=False, seed=4)
    norm = np.array([2.0, 2.5, 1.5, 3.0, 0.5, 0.8, 1.2, 0.4], np.float32)
    net.set_norm(norm)
    x = (2.0 + np.random.default_rng(6).standard_normal((2, 20, 33, 4))).astype(np.float32)
    got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    xn = (x.astype(np.float64) - norm[:4]) / norm[4:]
    want = oracle.cnn_forward(net.params().astype(np.float64), xn)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    net.close()


@pytest.fixture(scope="module")
def training_set(wd):  # 4 seeded 96x96x224 scenes, DWT-LRX (5,15) targets; the last is held out
    from paper_1201_2025_gb300 import synth
    out = []
    for seed in range(1, 5):
        sc = synth.make_scene(96, 96, 224, seed=seed, n_anom=12, anom_side=(1, 3), abundance=(0.1, 0.5), margin=4)
        x = torch.from_numpy(sc.cube).cuda()
        approx = wd.wdad_dwt_approx(x)
        lrx = wd.wdad_detect(approx, 0, reduce=False, inner=5, outer=15)
        out.append((approx, lrx))
    allv = torch.cat([a.reshape(-1, 4) for a, _ in out])
    norm = torch.cat([allv.mean(0), allv.std(0)]).cpu().numpy()
    return out, norm


def test_checkpoint_resume_is_bit_exact(wd, training_set, tmp_path):
    data, norm = training_set
    approx, lrx = data[0]
    a = wd.wdad_cnn(K=4, seed=9)
    a.set_norm(norm)
    a.train(approx, lrx, steps=3, batch=4, crop=32, lr=1e-3, seed=1)
    path = str(tmp_path / "cnn.ckpt")
    a.save(path)
    a.train(approx, lrx, steps=3, batch=4, crop=32, lr=1e-3, seed=1)
    b = wd.wdad_cnn.load(path)
    b.train(approx, lrx, steps=3, batch=4, crop=32, lr=1e-3, seed=1)
    assert np.array_equal(a.params(), b.params())
    a.close(); b.close()


def test_screening_recall_and_exact_values(wd, training_set):
    from paper_1201_2025_gb300 import synth
    data, norm = training_set
    net = wd.wdad_cnn(K=4, seed=11)
    net.set_norm(norm)
    # a fixed validation batch: the full (normalised) last training cube and its targets
    approx_v, lrx_v = data[-1]
    nt = torch.from_numpy(norm).cuda()
    xv = ((approx_v - nt[:4]) / nt[4:]).unsqueeze(0).contiguous()
    tv = torch.log1p(lrx_v.clamp_min(0)).unsqueeze(0).contiguous()
    before, _ = net.grad(xv, tv)
    for epoch in range(6):
        for approx, lrx in data[:-1]:
            net.train(approx, lrx, steps=40, batch=8, crop=32, lr=2e-3, seed=100 + epoch)
    after, _ = net.grad(xv, tv)
    assert after < 0.7 * before, (before, after)
    test = synth.make_scene(96, 96, 224, seed=77, n_anom=12, anom_side=(1, 3), abundance=(0.1, 0.5), margin=4)
    x = torch.from_numpy(test.cube).cuda()
    # screened DWT-LRX (the detector the network learned): recall of implanted anomalies that the
    # exact DWT-LRX map ranks in its top 5%, evaluating 6% of the pixels exactly
    score, pred, sel, nsel = wd.wdad_screen_run(net, x, top_frac=0.05, audit_frac=0.01, seed=3, tile_rows=40,
                                                exact_reduce=True, inner=5, outer=15)
    s = score.cpu().numpy()
    selm = sel.cpu().numpy() > 0
    assert nsel == selm.sum() and np.isfinite(s[selm]).all() and np.isneginf(s[~selm]).all()
    red = wd.wdad_detect(x, 0, reduce=True, inner=5, outer=15).cpu().numpy()
    assert np.array_equal(s[selm], red[selm])
    truth = (test.mask > 0) & (red >= np.quantile(red, 0.95))
    assert truth.sum() >= 5
    recall = (selm & truth).sum() / truth.sum()
    print(f"screened DWT-LRX recall {recall:.3f} with {selm.mean():.3f} of pixels evaluated")
    assert recall >= 0.8 and recall > 5 * selm.mean(), (recall, selm.mean())
    # screened full-band LRX: exact values bit-identical to the full map at the selected pixels
    score, _, sel, nsel = wd.wdad_screen_run(net, x, top_frac=0.05, audit_frac=0.01, seed=3, tile_rows=40,
                                             exact_reduce=False, inner=5, outer=15, want_pred=False)
    s = score.cpu().numpy()
    selm = sel.cpu().numpy() > 0
    full = wd.wdad_detect(x, 0, reduce=False, inner=5, outer=15).cpu().numpy()
    assert np.array_equal(s[selm], full[selm]) and np.isneginf(s[~selm]).all()
    truth = (test.mask > 0) & (full >= np.quantile(full, 0.95))
    recall_full = (selm & truth).sum() / truth.sum()
    print(f"screened full-band LRX recall {recall_full:.3f} (the approximation-space network cannot see "
          f"what only the full band separates)")
    assert recall_full > selm.mean()
    net.close()
