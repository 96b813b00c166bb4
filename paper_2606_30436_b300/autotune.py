"""Autotuner of the compositing launch shape for a chunk of views.

Sweeps the tile shape (16x16, 8x32, 32x8) and the number of pairs each warp
scans per step (128, 256, 512), times forward + loss + backward of the chunk
on the device (CUDA events, after a warm-up), and returns the fastest
Config.  Results never depend on the choice (the tests check every shape);
only the time does.  Choices are cached per (Gaussian count, view sizes).
"""
from __future__ import annotations

import dataclasses

import torch

from . import gs

SHAPES = ((16, 16), (8, 32), (32, 8))
BATCHES = (128, 256, 512)
_cache: dict = {}


def _key(model, cams):
    return (model.n, model.sh_degree, tuple((int(c["width"]), int(c["height"])) for c in cams))


def autotune(model: gs.GaussianModel, cams, targets_for, base: gs.Config = None, reps=3, lambda_dssim=0.2,
             shapes=SHAPES, batches=BATCHES):
    """targets_for(cfg) -> target tensor in the frame layout of `cams`.
    Returns (best Config, {(tile_w, tile_h, batch): ms})."""
    key = _key(model, cams)
    if key in _cache:
        return _cache[key]
    base = base or gs.Config()
    times = {}
    best = None
    for (tw, th) in shapes:
        st = None
        for batch in batches:
            cfg = dataclasses.replace(base, tile_w=tw, tile_h=th, batch=batch)
            if st is None:
                st = gs.MappingStep(model, cams, cfg, lambda_dssim=lambda_dssim, with_stats=True)
                st.fit_capacity()
                target = targets_for(cfg)
            st.cfg = cfg
            st.buf.cfg = cfg
            for _ in range(2):
                st.step(target, optimize=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                st.step(target, optimize=False)
            e1.record()
            torch.cuda.synchronize()
            st.check_status()
            ms = e0.elapsed_time(e1) / reps
            times[(tw, th, batch)] = ms
            if best is None or ms < best[1]:
                best = (cfg, ms)
        del st
    _cache[key] = (best[0], times)
    return _cache[key]
