"""Probabilistic initialisation of new anchors at a keyframe (Sec. 3.3.1) and
the voxel hash of the dynamic map expansion (Supp. D.5).

Thin binding of ``gs_init_probability``, ``gs_init_insert``,
``gs_voxel_lookup`` and ``gs_voxel_table_reset`` (``include/gs.h``), and the
``AnchorMap`` that owns the voxel table and the anchor records.  Per keyframe:

    prob = gs_init_probability(img, depth, img_r, depth_r)   # P, or P_kf against the render
    amap.insert(prob, uniform, depth, cam)                    # NMS, draw, voxels, new anchors

Every step runs in the library's kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import math

import torch

from . import gs

GS_INIT_MAX_LEVELS = 8
VOXEL_DEFAULT = (0.1, 0.25, 1.0, 5.0, 25.0)
MAX_DIST_DEFAULT = (10.0, 25.0, 100.0, 500.0, math.inf)


class InitCfg(C.Structure):
    _fields_ = [("sigma1", C.c_float), ("sigma2", C.c_float), ("lam", C.c_float), ("scale", C.c_float),
                ("near_z", C.c_float),
                ("levels", C.c_int32), ("voxel", C.c_float * GS_INIT_MAX_LEVELS),
                ("max_dist", C.c_float * GS_INIT_MAX_LEVELS)]


class VoxelTable(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("ids", C.c_void_p), ("owner", C.c_void_p), ("capacity", C.c_int64)]


class AnchorSet(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("level", C.c_void_p), ("pixel", C.c_void_p), ("count", C.c_void_p),
                ("ld", C.c_int64)]


_typed = False


def _lib():
    global _typed
    L = gs.lib()
    if not _typed:
        vp, i32, i64, sz, P = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.POINTER
        L.gs_voxel_table_reset.argtypes = [P(VoxelTable), vp]
        L.gs_init_workspace_size.argtypes = [i32, i32, P(sz)]
        L.gs_init_probability.argtypes = [vp, vp, vp, vp, i32, i32, P(InitCfg), vp, vp, sz, vp]
        L.gs_init_insert.argtypes = [vp, vp, vp, P(gs.Camera), P(InitCfg), P(VoxelTable), P(AnchorSet), vp, vp, vp,
                                     sz, vp]
        L.gs_voxel_lookup.argtypes = [P(VoxelTable), vp, i64, i64, vp, vp]
        _typed = True
    return L


def init_config(sigma1=1.0, sigma2=1.6, lam=0.9, scale=255.0, near_z=0.2, voxel=VOXEL_DEFAULT,
                max_dist=MAX_DIST_DEFAULT):
    """The initialisation constants (defaults: DoG widths 1 and 1.6 px on 8-bit
    intensity units, lambda = 0.9 of Supp. F, five LoD levels)."""
    assert len(voxel) == len(max_dist) and 1 <= len(voxel) <= GS_INIT_MAX_LEVELS
    v = (C.c_float * GS_INIT_MAX_LEVELS)(*voxel)
    d = (C.c_float * GS_INIT_MAX_LEVELS)(*max_dist)
    return InitCfg(sigma1, sigma2, lam, scale, near_z, len(voxel), v, d)


def init_workspace(width, height, device="cuda"):
    n = C.c_size_t()
    gs._check(_lib().gs_init_workspace_size(int(width), int(height), C.byref(n)), "gs_init_workspace_size")
    return torch.empty(n.value, dtype=torch.uint8, device=device)


def gs_init_probability(img, depth, img_r=None, depth_r=None, cfg=None, prob=None, ws=None, stream=None):
    """prob [H][W]: P of (img [3][H][W], depth [H][W]), or P_kf = max(P - P^, 0) against the rendered pair."""
    H, W = depth.shape[-2:]
    cfg = init_config() if cfg is None else cfg
    prob = torch.empty(H, W, dtype=torch.float32, device=depth.device) if prob is None else prob
    ws = init_workspace(W, H, depth.device) if ws is None else ws
    gs._check(_lib().gs_init_probability(gs._ptr(img), gs._ptr(depth), gs._ptr(img_r), gs._ptr(depth_r), W, H,
                                         C.byref(cfg), gs._ptr(prob), gs._ptr(ws), ws.numel(), gs._stream(stream)),
              "gs_init_probability")
    return prob


class AnchorMap:
    """Voxel table (open addressing, capacity a power of two) and anchor
    records (positions [3][capacity], level, spawning pixel) on the device."""

    def __init__(self, capacity, table_capacity=None, device="cuda"):
        # capacity = the plane stride of the records, a multiple of 4
        self.capacity = ld = max(4, (int(capacity) + 3) // 4 * 4)
        tc = table_capacity or max(1024, 1 << math.ceil(math.log2(2 * ld)))
        assert tc & (tc - 1) == 0
        self.keys = torch.empty(tc, dtype=torch.int64, device=device)
        self.ids = torch.empty(tc, dtype=torch.int32, device=device)
        self.owner = torch.empty(tc, dtype=torch.int32, device=device)
        self.pos = torch.zeros(3, ld, dtype=torch.float32, device=device)
        self.level = torch.zeros(ld, dtype=torch.int32, device=device)
        self.pixel = torch.zeros(ld, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.table = VoxelTable(self.keys.data_ptr(), self.ids.data_ptr(), self.owner.data_ptr(), tc)
        self.set = AnchorSet(self.pos.data_ptr(), self.level.data_ptr(), self.pixel.data_ptr(),
                             self.count.data_ptr(), self.capacity)
        self.ws = None
        self.reset()

    def reset(self, stream=None):
        self.count.zero_()
        self.status.zero_()
        gs._check(_lib().gs_voxel_table_reset(C.byref(self.table), gs._stream(stream)), "gs_voxel_table_reset")

    def insert(self, prob, uniform, depth, cam, cfg=None, selected=None, stream=None):
        """New anchors of one keyframe (cam: a camera dict); nothing synchronises the host."""
        H, W = depth.shape[-2:]
        assert int(cam["width"]) == W and int(cam["height"]) == H
        cfg = init_config() if cfg is None else cfg
        if self.ws is None or self.ws.numel() < _ws_bytes(W, H):
            self.ws = init_workspace(W, H, depth.device)
        camera = gs.make_camera(cam)
        gs._check(_lib().gs_init_insert(gs._ptr(prob), gs._ptr(uniform), gs._ptr(depth), C.byref(camera),
                                        C.byref(cfg), C.byref(self.table), C.byref(self.set), gs._ptr(selected),
                                        gs._ptr(self.status), gs._ptr(self.ws), self.ws.numel(), gs._stream(stream)),
                  "gs_init_insert")

    def lookup(self, vox, n, stream=None):
        """Anchor ids of the voxels (level, ix, iy, iz) = planes of vox [4][ld] int32; -1 where free."""
        out = torch.empty(max(n, 1), dtype=torch.int32, device=vox.device)
        gs._check(_lib().gs_voxel_lookup(C.byref(self.table), gs._ptr(vox), int(n), int(vox.shape[1]),
                                         gs._ptr(out), gs._stream(stream)), "gs_voxel_lookup")
        return out[:n]

    @property
    def n(self):
        return int(self.count.item())

    def check_status(self):
        st = int(self.status.item())
        if st:
            raise gs.GSError("anchor insertion status 0x%x" % st)


def _ws_bytes(W, H):
    n = C.c_size_t()
    gs._check(_lib().gs_init_workspace_size(int(W), int(H), C.byref(n)), "gs_init_workspace_size")
    return n.value
