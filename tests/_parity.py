"""Helpers of the GPU-vs-oracle parity tests: run the same seeded inputs through
the C ABI (libgs.so) and through the FP64 oracle, and compare.

Tolerances (derived in the design notes from the FP32 arithmetic):
    images, T_final            <= 1e-4 max-abs, pixels with a near-threshold
                                  event (alpha ~ 1/255, T(1-alpha) ~ 1e-4) masked
    gradients                  <= 1e-3 relative L2 per parameter group
    pair lists, ranges, u, v, depth, cull decisions: bit-exact
    radius: exact except where 3 sqrt(lambda_max) lies within 2e-4 (relative)
            of an integer, where FP32 may round the other way (counted)
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as orc
from paper_2606_30436_b300 import gs

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def ocfg(cfg: gs.Config, fp32=True):
    return orc.Cfg(tile_w=cfg.tile_w, tile_h=cfg.tile_h, near_z=cfg.near_z, dilation=cfg.dilation,
                   alpha_min=cfg.alpha_min, alpha_max=cfg.alpha_max, t_min=cfg.t_min, tan_clamp=cfg.tan_clamp,
                   bg=tuple(cfg.bg), fp32_positions=fp32)


def near_integer(x, rel=2e-4):
    return np.abs(x - np.rint(x)) < rel * np.maximum(np.abs(x), 1.0)


def gpu_forward(scene, cams, cfg=None, max_pairs=None):
    cfg = cfg or gs.Config()
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, cfg, max_pairs=max_pairs)
    st.forward()
    torch.cuda.synchronize()
    return st


def projected_numpy(st: gs.MappingStep):
    b = st.buf
    n, ld = st.model.n, b.ld
    out = []
    for v in range(b.n_views):
        sl = slice(v * ld, v * ld + n)
        out.append(dict(xy=b.xy[sl].cpu().numpy(), co=b.conic_opacity[sl].cpu().numpy(),
                        rgbd=b.rgb_depth[sl].cpu().numpy(), radius=b.radius[sl].cpu().numpy(),
                        touched=b.tiles_touched[sl].cpu().numpy()))
    return out


def gpu_pairs(st: gs.MappingStep):
    b = st.buf
    counts = b.counts.cpu().numpy()
    P = int(counts[1])
    return counts, b.gauss_ids[:P].cpu().numpy(), b.tile_ranges.cpu().numpy()


def oracle_views(scene, cams, cfg: gs.Config, fp32=True):
    oc = ocfg(cfg, fp32)
    res = []
    for cam in cams:
        pr = orc.project(scene, cam, oc)
        keys, vals, ranges = orc.bin_pairs(pr, cam, oc)
        res.append(dict(proj=pr, keys=keys, vals=vals, ranges=ranges, cam=cam))
    return res


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
