"""Pins of the oracle's Adam (reading R10) against torch.optim.Adam, and of the
lifecycle statistics and chunk scores (Supp. E.1, E.2; Sec. 3.3.2): a
hand-computed finalize example, the degenerate min = max chunk, aggregation
over chunks, and footprint counts against brute-force contributor lists."""
import math

import numpy as np
import torch

from paper_2606_30436_b300 import scenes


def test_adam_matches_torch(orc):
    rng = np.random.default_rng(0)
    n_groups = [(5, 1e-3), (7, 5e-2), (4, 2.5e-3)]
    ps = [rng.standard_normal(k) for k, _ in n_groups]
    tparams = [torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True) for p in ps]
    opt = torch.optim.Adam([{"params": [t], "lr": lr} for t, (_, lr) in zip(tparams, n_groups)],
                           betas=(0.9, 0.999), eps=1e-15)
    flat = np.concatenate(ps)
    lr = np.concatenate([np.full(k, lr) for k, lr in n_groups])
    m, v = np.zeros_like(flat), np.zeros_like(flat)
    for step in range(1, 11):
        grads = [rng.standard_normal(k) * (0.0 if step == 4 else 1.0) for k, _ in n_groups]
        for t, g in zip(tparams, grads):
            t.grad = torch.tensor(g)
        opt.step()
        g = np.concatenate(grads)
        orc.adam(flat, g, m, v, lr, step)
    ref = np.concatenate([t.detach().numpy() for t in tparams])
    assert np.abs(flat - ref).max() <= 1e-15 * np.abs(ref).max() * 10


def test_finalize_hand_computed(orc):
    e = math.e
    omega = [10, 0, 5, 3]
    kappa = [12, 0, 3, 0]
    gamma = [e - 1, 0, e * e - 1, 0]
    r = orc.prune_finalize(omega, kappa, gamma, n_views=2)
    # S_d = kappa / |V_c|; L = ln(1 + gamma) = (1, -, 2, 0) over the active set {0, 2, 3}
    assert np.allclose(r["S_d"], [6, 0, 1.5, 0], atol=0)
    assert np.allclose(r["S_p"], [0.5, 0, 1, 0], atol=1e-15)
    assert list(r["densify"]) == [1, 0, 0, 0]
    assert list(r["prune"]) == [0, 0, 1, 0]


def test_finalize_degenerate_and_aggregation(orc):
    r = orc.prune_finalize([1, 2, 0], [0, 0, 0], [3.0, 3.0, 0.0], n_views=4)
    assert np.all(r["S_p"] == 0) and not r["prune"].any()
    # two chunks: densify ORs, prune takes the max
    d, pm = np.zeros(3, np.uint8), np.zeros(3)
    r1 = orc.prune_finalize([1, 1, 1], [12, 0, 0], [0.0, 1.0, 3.0], 2, densify=d, prune_max=pm)
    r2 = orc.prune_finalize([1, 1, 1], [0, 11, 0], [3.0, 1.0, 0.0], 2, densify=d, prune_max=pm)
    assert list(r2["densify"]) == [1, 1, 0]
    assert list(r2["prune"]) == [1, 0, 1]
    assert np.allclose(r2["prune_max"], [1.0, math.log(2) / math.log(4), 1.0])


def _contributors(pr, cfg, W, H):
    lists = {}
    for j in range(H):
        for i in range(W):
            tx, ty = i // cfg.tile_w, j // cfg.tile_h
            mem = [g for g in range(pr.n) if pr["radius"][g] > 0 and pr["rect"][g][0] <= tx < pr["rect"][g][2]
                   and pr["rect"][g][1] <= ty < pr["rect"][g][3]]
            mem.sort(key=lambda g: (pr["z"][g], g))
            T, out = 1.0, []
            for g in mem:
                dx, dy = i + 0.5 - pr["u"][g], j + 0.5 - pr["v"][g]
                q = pr["conic"][g]
                pw = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy
                if pw > 0:
                    continue
                a = min(0.99, pr["opacity"][g] * math.exp(pw))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                out.append((g, a * T))
                T *= 1 - a
            lists[(j, i)] = out
    return lists


def test_footprint_stats_brute_force(orc):
    """Two views of a 40-Gaussian scene: |Omega|, kappa, gamma, max T*alpha and
    the view count equal counts over brute-force per-pixel contributor lists."""
    p = scenes.uniform_scene(40, seed=31, xy_range=1.2)
    p["log_scales"] += 1.0
    W, H = 48, 40
    cams = [scenes.pinhole(W, H, 50.0), scenes.pinhole(W, H, 50.0, t=np.array([0.3, 0.0, 0.2], np.float32))]
    cfg = orc.Cfg(fp32_positions=False)
    stats = np.zeros((40, 6))
    ref = np.zeros((40, 6))
    for v, cam in enumerate(cams):
        target = scenes.smooth_image(H, W, seed=50 + v)
        f_ = orc.loss_and_grads(p, cam, cfg, target, 0.2, tau_err=0.1, stats=stats)
        lists = _contributors(f_["proj"], cfg, W, H)
        err = np.abs(f_["img"] - target).sum(axis=0)
        om = np.zeros(40)
        for (j, i), lst in lists.items():
            for g, w in lst:
                om[g] += 1
                ref[g, 1] += err[j, i] > 0.1
                ref[g, 3] = max(ref[g, 3], w)
        ref[:, 0] += om
        ref[:, 2] += f_["loss"] * om
        ref[:, 5] += om > 0
    assert np.array_equal(stats[:, 0], ref[:, 0]) and stats[:, 0].sum() > 100
    assert np.array_equal(stats[:, 1], ref[:, 1]) and stats[:, 1].sum() > 0
    assert np.allclose(stats[:, 2], ref[:, 2], rtol=1e-12)
    assert np.allclose(stats[:, 3], ref[:, 3], rtol=1e-12)
    assert np.array_equal(stats[:, 5], ref[:, 5])
