"""Parity at the benchmark's own size: one whole 1280x720 corridor frame of
the 1M-Gaussian SH-degree-3 scene (frame 500), run through the default
mapping configuration -- 16x16 tiles and the split compositing of tile lists
longer than 512 pairs (and, as a second arm, 256), where the vanishing-point
tiles hold tens of thousands of pairs -- against the FP64 oracle on the same
inputs:

- pair ids and tile ranges bit-exact (Gaussians whose radius rounds the other
  way in FP32 next to an integer are dropped from both lists and counted);
- the image and T_final within 1e-4, `last` exact, away from near-threshold
  pixels;
- the L1 + D-SSIM loss, and the gradient of every parameter group within
  1e-3 relative L2, through the split backward walked from the forward's
  boundary states.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes

from _parity import GROUPS, near_integer, ocfg, projected_numpy, rel_l2

pytestmark = pytest.mark.gpu

N, W, H, F, FRAME = 1_000_000, 1280, 720, 900.0, 500


@pytest.fixture(scope="module")
def frame():
    scene = scenes.corridor_scene(N, seed=0, sh_degree=3)
    cam = scenes.corridor_camera(FRAME, W, H, F)
    cfg = gs.Config()
    assert cfg.segment == 512
    oc = ocfg(cfg)
    target = orc.forward(scenes.perturb(scene, 0.01, seed=1), cam, oc)["img"].astype(np.float32)
    tgt = torch.from_numpy(target.reshape(-1)).cuda()
    steps = {}
    for seg in (512, 256):
        model = gs.GaussianModel.from_scene(scene)
        st = gs.MappingStep(model, [cam], gs.Config(segment=seg), lambda_dssim=0.2, with_stats=True)
        st.fit_capacity()
        st.step(tgt, optimize=False)
        torch.cuda.synchronize()
        st.check_status()
        steps[seg] = st
    ref = orc.loss_and_grads(scene, cam, oc, target, 0.2)
    return dict(scene=scene, cam=cam, cfg=cfg, steps=steps, st=steps[512], ref=ref)


def _flagged(frame):
    g = projected_numpy(frame["st"])[0]
    pr = frame["ref"]["proj"]
    diff = np.nonzero(g["radius"] != pr["radius"])[0]
    assert np.all(near_integer(pr["radius_exact"][diff])), "radius differs away from an integer"
    assert np.all(np.abs(g["radius"][diff] - pr["radius"][diff]) <= 1)
    return g, diff


def _by_tile(ids, ranges):
    """(tile, id) of every pair, in list order; the ranges tile the list."""
    lens = ranges[:, 1] - ranges[:, 0]
    nonempty = lens > 0
    assert np.all(np.diff(ranges[nonempty, 0]) > 0)
    assert lens.sum() == len(ids)
    return np.repeat(np.arange(len(ranges)), lens), ids


def test_fullsize_split_is_exercised(frame):
    ranges = frame["ref"]["ranges"]
    longest = int((ranges[:, 1] - ranges[:, 0]).max())
    assert longest > 30_000, longest  # vanishing-point tiles: many segments each
    for st in frame["steps"].values():
        off, _ = st.buf.seg_needed()
        assert not off, "the split plan did not fit its workspace"


def test_fullsize_pairs_bit_exact(frame):
    st, ref = frame["st"], frame["ref"]
    g, flagged = _flagged(frame)
    assert len(flagged) <= N // 500
    counts = st.buf.counts.cpu().numpy()
    P = int(counts[1])
    assert counts[0] == int((g["radius"] > 0).sum()) and counts[2] == P
    ids = st.buf.gauss_ids[:P].cpu().numpy().astype(np.int64)
    ranges = st.buf.tile_ranges.cpu().numpy().astype(np.int64)
    t_gpu, i_gpu = _by_tile(ids, ranges)
    t_ref, i_ref = _by_tile(ref["vals"].astype(np.int64), ref["ranges"].astype(np.int64))
    keep_gpu = ~np.isin(i_gpu, flagged)
    keep_ref = ~np.isin(i_ref, flagged)
    assert np.array_equal(t_gpu[keep_gpu], t_ref[keep_ref])
    assert np.array_equal(i_gpu[keep_gpu], i_ref[keep_ref])
    if len(flagged) == 0:
        nonempty = ref["ranges"][:, 1] > ref["ranges"][:, 0]
        assert np.array_equal(ranges[nonempty], ref["ranges"][nonempty])


@pytest.mark.parametrize("seg", [512, 256])
def test_fullsize_image(frame, seg):
    st, ref, cfg = frame["steps"][seg], frame["ref"], frame["cfg"]
    _, flagged = _flagged(frame)
    b = st.buf
    img = b.view_image(0).cpu().numpy()
    Tf = b.view_plane(b.T_final, 0).cpu().numpy()
    last = b.view_plane(b.last, 0).cpu().numpy()
    mask = ref["flags"] & (orc.OR_FLAG_NEAR_ALPHA_MIN | orc.OR_FLAG_NEAR_T_CUT) != 0
    for gi in flagged:  # tiles a flagged Gaussian may or may not reach
        x0, y0, x1, y1 = ref["proj"]["rect"][gi]
        mask[max(0, y0 - 1) * cfg.tile_h:(y1 + 1) * cfg.tile_h, max(0, x0 - 1) * cfg.tile_w:(x1 + 1) * cfg.tile_w] = True
    assert mask.mean() < 1e-2, mask.mean()
    assert np.abs(img - ref["img"]).max(axis=0)[~mask].max() <= 1e-4
    assert np.abs(Tf - ref["T_final"])[~mask].max() <= 1e-4
    GW = (W + cfg.tile_w - 1) // cfg.tile_w
    jj, ii = np.mgrid[0:H, 0:W]
    start = ref["ranges"][(jj // cfg.tile_h) * GW + ii // cfg.tile_w, 0]
    exp_last = np.where(ref["last_pos"] >= 0, ref["last_pos"] - start + 1, 0)
    assert np.array_equal(last[~mask], exp_last[~mask])


@pytest.mark.parametrize("seg", [512, 256])
def test_fullsize_loss_and_gradients(frame, seg):
    st, ref = frame["steps"][seg], frame["ref"]
    assert abs(st.buf.loss.item() - ref["loss"]) <= 1e-4 * abs(ref["loss"])
    g = gs.unpack_planes(st.grads.data.cpu().numpy(), N, 3)
    for k in GROUPS:
        e = rel_l2(g[k], ref["grads"][k])
        assert e < 1e-3, (k, e)
