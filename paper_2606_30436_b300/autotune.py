"""Autotuner of the compositing launch shape for a chunk of views.

Sweeps the tile shape (16x16, 8x32, 32x8), the number of pairs each warp
scans per step (128, 256, 512) and the split length of long tile lists (none,
or a power of two: the split pays where a few tiles hold long lists that some
pixels never saturate, and costs where every tile is long and saturates
early), times forward + loss + backward of the chunk on the device (CUDA
events, after a warm-up), and returns the fastest Config.  Results never
depend on the choice beyond FP32 rounding (the tests check every shape); only
the time does.  Choices are cached per (Gaussian count, view sizes).
"""
from __future__ import annotations

import dataclasses
import itertools

import torch

from . import gs

SHAPES = ((16, 16), (8, 32), (32, 8))
BATCHES = (128, 256, 512)
SEGMENTS = (0, 256, 1024)
_cache: dict = {}


def _key(model, cams):
    return (model.n, model.sh_degree, tuple((int(c["width"]), int(c["height"])) for c in cams))


def autotune(model: gs.GaussianModel, cams, targets_for, base: gs.Config = None, reps=3, lambda_dssim=0.2,
             shapes=SHAPES, batches=BATCHES, segments=SEGMENTS):
    """targets_for(cfg) -> target tensor in the frame layout of `cams`.
    Returns (best Config, {(tile_w, tile_h, batch, segment): ms})."""
    key = _key(model, cams)
    if key in _cache:
        return _cache[key]
    base = base or gs.Config()
    times = {}
    best = None
    for (tw, th) in shapes:
        st = None
        for batch, segment in itertools.product(batches, segments):
            cfg = dataclasses.replace(base, tile_w=tw, tile_h=th, batch=batch, segment=segment)
            if st is None:
                st = gs.MappingStep(model, cams, cfg, lambda_dssim=lambda_dssim, with_stats=True)
                st.fit_capacity()
                target = targets_for(cfg)
            resize = st.buf.cfg.segment != segment
            st.cfg = cfg
            st.buf.cfg = cfg
            if resize:  # the split workspace follows the segment length and the items measured
                st.buf.seg_items = 0
                st.buf.set_max_pairs(st.buf.max_pairs)
                st.fit_capacity()
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
            times[(tw, th, batch, segment)] = ms
            if best is None or ms < best[1]:
                best = (cfg, ms)
        del st
    _cache[key] = (best[0], times)
    return _cache[key]
