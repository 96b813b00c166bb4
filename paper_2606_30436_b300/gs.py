"""Thin Python binding of the C ABI in ``include/gs.h`` (``libgs.so``).

The functions ``gs_project``, ``gs_sort``, ``gs_render_fwd``, ``gs_loss``,
``gs_render_bwd``, ``gs_adam`` and ``gs_prune_stats`` carry the names of the C
entry points and only marshal arguments: torch tensors give device pointers,
the current torch stream is passed as the CUDA stream, and every step of the
mapping path runs in the library's kernels.  There is no CPU fallback: if the
library is missing or no CUDA device is present, the calls raise.

The helper classes (``GaussianModel``, ``Buffers``, ``MappingStep``) own the
device buffers the C ABI expects and chain the calls into one mapping
iteration (Sec. 3.2.3: render, L_photo, backward, Adam; Supp. E: lifecycle
statistics).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import build as _build

# --------------------------------------------------------------------------
# C structs (mirror include/gs.h)

GS_MAX_VIEWS = 64
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "pair capacity exceeded",
                4: "bounded wait timed out", 5: "non-finite value"}
GS_ERR_CAPACITY = 3
GS_ERR_TIMEOUT = 4
GS_ERR_NUMERIC = 5


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class RasterCfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_z", C.c_float), ("dilation", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float),
                ("tan_clamp", C.c_float), ("bg", C.c_float * 3), ("batch", C.c_int32), ("segment", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n", C.c_int64), ("ld", C.c_int64), ("sh_degree", C.c_int32)]


class Projected(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("conic_opacity", C.c_void_p), ("rgb_depth", C.c_void_p),
                ("radius", C.c_void_p), ("tiles_touched", C.c_void_p), ("ld", C.c_int64),
                ("color_jac", C.c_void_p)]


class PlaneSet(C.Structure):
    _fields_ = [("data", C.c_void_p), ("ld", C.c_int64), ("planes", C.c_int32)]


class Binning(C.Structure):
    _fields_ = [("gauss_ids", C.c_void_p), ("tile_ranges", C.c_void_p), ("counts", C.c_void_p),
                ("block_mask", C.c_void_p), ("tile_order", C.c_void_p), ("max_pairs", C.c_int64)]


class Frame(C.Structure):
    _fields_ = [("img", C.c_void_p), ("T_final", C.c_void_p), ("last", C.c_void_p), ("depth", C.c_void_p),
                ("seg_ws", C.c_void_p), ("seg_ws_bytes", C.c_size_t)]


class Stats(C.Structure):
    _fields_ = [("acc", C.c_void_p), ("ld", C.c_int64)]


class ChunkScores(C.Structure):
    _fields_ = [("S_d", C.c_void_p), ("S_p", C.c_void_p), ("prune_max", C.c_void_p), ("densify", C.c_void_p),
                ("prune", C.c_void_p)]


EXPORTS = ("gs_status_string", "gs_version", "gs_view_layout", "gs_sort_workspace_size", "gs_block_mask_size",
           "gs_loss_workspace_size",
           "gs_bwd_workspace_size", "gs_prune_workspace_size", "gs_project", "gs_sort", "gs_render_fwd", "gs_loss",
           "gs_render_bwd", "gs_project_bwd", "gs_adam", "gs_prune_stats", "gs_loss_static",
           "gs_reg_workspace_size", "gs_geo_loss", "gs_iso_loss", "gs_actions_workspace_size", "gs_densify_prune",
           "gs_mlp_push_blend", "gs_mlp_features", "gs_mlp_forward", "gs_mlp_train_grad", "gs_mlp_adam",
           "gs_segment_workspace_size", "gs_project_bwd_adam", "gs_segment_workspace_size_items",
           "gs_voxel_table_reset", "gs_init_workspace_size", "gs_init_probability", "gs_init_insert",
           "gs_voxel_lookup", "gs_anchor_decode", "gs_anchor_decode_bwd", "gs_adam_flat",
           "gs_list_workspace_size", "gs_render_fwd_lists", "gs_render_bwd_lists", "gs_reorder_workspace_size",
           "gs_reorder", "gs_project_bwd_rows", "gs_adam_rows",
           "gs_adam_part")

_lib = None


def lib():
    """Loads libgs.so (building it when a source is newer); raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path) or _build._stale():
            path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64, f32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_size_t
        P = C.POINTER
        L.gs_status_string.argtypes = [C.c_int]
        L.gs_status_string.restype = C.c_char_p
        L.gs_version.restype = i32
        L.gs_view_layout.argtypes = [P(Camera), i32, P(RasterCfg), P(i64), P(i64), vp, vp]
        L.gs_sort_workspace_size.argtypes = [i64, i64, P(sz)]
        L.gs_block_mask_size.argtypes = [i64, P(sz)]
        L.gs_loss_workspace_size.argtypes = [i32, i32, P(sz)]
        L.gs_bwd_workspace_size.argtypes = [i64, P(sz)]
        L.gs_segment_workspace_size.argtypes = [i64, i32, P(sz)]
        L.gs_segment_workspace_size_items.argtypes = [i64, P(sz)]
        L.gs_prune_workspace_size.argtypes = [i64, P(sz)]
        L.gs_project.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), vp, vp]
        L.gs_sort.argtypes = [P(Projected), P(Camera), i32, P(RasterCfg), P(Binning), vp, sz, vp, vp]
        L.gs_render_fwd.argtypes = [P(Projected), P(Binning), P(Camera), i32, P(RasterCfg), P(Frame), vp]
        L.gs_loss.argtypes = [vp, vp, P(Camera), i32, f32, vp, vp, vp, sz, vp]
        L.gs_loss_static.argtypes = [vp, vp, P(Camera), i32, f32, vp, vp, vp]
        L.gs_reg_workspace_size.argtypes = [P(sz)]
        L.gs_geo_loss.argtypes = [vp, vp, P(Camera), i32, f32, vp, vp, vp, sz, vp]
        L.gs_iso_loss.argtypes = [P(Params), f32, vp, P(Params), vp, sz, vp]
        L.gs_render_bwd.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), P(Binning), P(Frame),
                                    vp, vp, vp, vp, f32, P(Params), i32, P(Stats), vp, sz, vp]
        L.gs_project_bwd.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), vp, sz, vp, P(Params), i32,
                                     P(Stats), vp]
        L.gs_adam.argtypes = [P(Params), P(Params), P(Params), P(Params), P(f32 * 6), f32, f32, f32, i64, vp, vp]
        L.gs_project_bwd_rows.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), vp, sz, vp,
                                          P(Params), P(Stats), vp, vp]
        L.gs_adam_rows.argtypes = [P(Params), P(Params), P(Params), P(Params), vp, P(f32 * 6), f32, f32, f32, i64,
                                   vp, vp]
        L.gs_adam_part.argtypes = [P(Params), P(Params), P(Params), P(Params), vp, vp, i32, i32, P(f32 * 6), f32,
                                   f32, f32, i64, vp, vp]
        L.gs_project_bwd_adam.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), vp, sz, vp,
                                          P(Params), f32, P(Params), P(Params), P(f32 * 6), f32, f32, f32, i64, vp,
                                          P(Stats), vp]
        L.gs_prune_stats.argtypes = [P(Stats), i64, i32, f32, f32, P(ChunkScores), vp, sz, vp]
        L.gs_actions_workspace_size.argtypes = [i64, P(sz)]
        L.gs_reorder_workspace_size.argtypes = [i64, i64, i32, P(sz)]
        L.gs_reorder.argtypes = [P(Params), P(PlaneSet), i32, vp, vp, sz, vp]
        L.gs_densify_prune.argtypes = [P(Params), P(Params), P(Params), vp, vp, vp, f32, f32, P(Params), P(Params),
                                       P(Params), vp, vp, vp, sz, vp]
        L.gs_mlp_push_blend.argtypes = [P(Stats), i64, vp, i64, i32, vp]
        L.gs_mlp_features.argtypes = [P(Params), P(Stats), vp, i32, P(f32 * 3), vp, vp]
        L.gs_mlp_forward.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, i64, vp]
        L.gs_mlp_train_grad.argtypes = [vp, vp, vp, i64, i64, vp, vp, vp, vp, vp]
        L.gs_mlp_adam.argtypes = [vp, vp, vp, vp, f32, f32, f32, f32, i64, vp]
        L.gs_list_workspace_size.argtypes = [i64, P(sz)]
        L.gs_render_fwd_lists.argtypes = [P(Projected), P(Binning), P(Camera), i32, P(RasterCfg), P(Frame), vp, vp, vp,
                                          i64, vp, sz, vp, vp]
        L.gs_render_bwd_lists.argtypes = [P(Params), P(Camera), i32, P(RasterCfg), P(Projected), P(Frame), vp, vp, vp,
                                          i64, vp, vp, vp, f32, P(Params), i32, P(Stats), vp, sz, vp]
        for name in EXPORTS:
            if name not in ("gs_status_string", "gs_version"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class GSError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise GSError("%s: %s" % (what, lib().gs_status_string(st).decode()))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------
# host-side descriptions

def make_camera(cam) -> Camera:
    R = np.asarray(cam["R"], np.float32).reshape(9)
    t = np.asarray(cam["t"], np.float32).reshape(3)
    return Camera((C.c_float * 9)(*R), (C.c_float * 3)(*t), cam["fx"], cam["fy"], cam["cx"], cam["cy"],
                  int(cam["width"]), int(cam["height"]))


def camera_array(cams):
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = make_camera(c)
    return arr


@dataclass
class Config:
    """Rasteriser constants (the standard EWA-splatting values)."""
    tile_w: int = 16
    tile_h: int = 16
    near_z: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    tan_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    batch: int = 512
    segment: int = 512  # split length of long tile lists, in pairs (0 = no split)
    # keep the colour's view-direction gradient per record (SH degree >= 1) for the backward:
    # None = where it moves fewer bytes than the backward's re-read of the SH coefficients
    color_jac: Optional[bool] = None
    # optimising steps: the projection backward writes only the gradient rows of Gaussians some
    # view sees and marks them; Adam reads the others as zero (None = wherever it applies)
    grad_rows: Optional[bool] = None
    # captured steps with grad_rows: the Adam of the Gaussians no view sees on a second stream,
    # beside the sort, compositing and losses (None = on)
    adam_overlap: Optional[bool] = None

    def c(self) -> RasterCfg:
        return RasterCfg(self.tile_w, self.tile_h, self.near_z, self.dilation, self.alpha_min, self.alpha_max,
                         self.t_min, self.tan_clamp, (C.c_float * 3)(*self.bg), self.batch, self.segment)


def planes(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def use_color_jac(cfg: Config, sh_degree: int, n_views: int) -> bool:
    """Whether the projection keeps the colour's direction gradient for the backward.
    Kept, it costs 48 bytes written and 48 read per visible record, at most
    96 n_views per Gaussian; it saves the backward's 4 (K - 11) bytes of SH
    coefficients per Gaussian.  Automatic (None): only where the bound says it
    saves, i.e. SH degree 3 with up to two views and degree 2 with one."""
    if sh_degree < 1:
        return False
    if cfg.color_jac is not None:
        return bool(cfg.color_jac)
    return 96 * n_views <= 4 * (planes(sh_degree) - 11)


def padded(n: int) -> int:
    return max(4, (n + 31) // 32 * 32)


def view_layout(cams, cfg: Config):
    arr = camera_array(cams)
    nt, npx = C.c_int64(), C.c_int64()
    toff = np.zeros(len(cams), np.int64)
    poff = np.zeros(len(cams), np.int64)
    _check(lib().gs_view_layout(arr, len(cams), C.byref(cfg.c()), C.byref(nt), C.byref(npx),
                                toff.ctypes.data_as(C.c_void_p), poff.ctypes.data_as(C.c_void_p)), "gs_view_layout")
    return nt.value, npx.value, toff, poff


# --------------------------------------------------------------------------
# Gaussian parameters in the plane-major layout

class GaussianModel:
    """Parameters of n Gaussians as one [K, ld] float32 device tensor."""

    def __init__(self, n, sh_degree, device="cuda", data=None, ld=None):
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.K = planes(self.sh_degree)
        self.ld = int(data.shape[1]) if data is not None else (padded(self.n) if ld is None else int(ld))
        assert self.ld >= self.n and self.ld % 4 == 0
        self.data = torch.zeros(self.K, self.ld, dtype=torch.float32, device=device) if data is None else data

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        m = cls(len(scene["means"]), scene["sh_degree"], device=device)
        m.data.copy_(torch.from_numpy(pack_planes(scene, m.ld)))
        return m

    def like(self):
        return GaussianModel(self.n, self.sh_degree, device=self.data.device, ld=self.ld)

    def c(self) -> Params:
        return Params(self.data.data_ptr(), self.n, self.ld, self.sh_degree)

    def to_scene(self):
        return unpack_planes(self.data.detach().cpu().numpy(), self.n, self.sh_degree)


def pack_planes(scene, ld):
    """Array-of-structures scene dict -> [K, ld] plane-major float32 array."""
    n, D = len(scene["means"]), int(scene["sh_degree"])
    K = planes(D)
    out = np.zeros((K, ld), np.float32)
    out[0:3, :n] = np.asarray(scene["means"], np.float32).T
    out[3:6, :n] = np.asarray(scene["log_scales"], np.float32).T
    out[6:10, :n] = np.asarray(scene["quats"], np.float32).T
    out[10, :n] = np.asarray(scene["opacity_logits"], np.float32)
    sh = np.asarray(scene["sh"], np.float32).reshape(n, -1)  # (n, (D+1)^2 * 3), coefficient-major, RGB minor
    out[11:, :n] = sh.T
    return out


def unpack_planes(arr, n, D):
    Kc = (D + 1) ** 2
    return dict(means=arr[0:3, :n].T.copy(), log_scales=arr[3:6, :n].T.copy(), quats=arr[6:10, :n].T.copy(),
                opacity_logits=arr[10, :n].copy(), sh=arr[11:, :n].T.reshape(n, Kc, 3).copy(), sh_degree=D)


# --------------------------------------------------------------------------
# device buffers of one (views, Gaussians) configuration

class Buffers:
    """Every device buffer the mapping step needs, sized once."""

    def __init__(self, model: GaussianModel, cams, cfg: Config, max_pairs: int, with_depth=False, with_stats=True):
        dev = model.data.device
        self.cams, self.cfg = list(cams), cfg
        self.n_views = len(self.cams)
        self.ld = model.ld
        self.nrec = self.n_views * self.ld
        self.total_tiles, self.total_pixels, self.tile_offset, self.pixel_offset = view_layout(self.cams, cfg)
        f32, i32 = torch.float32, torch.int32
        nr = self.nrec
        self.xy = torch.empty(nr, 2, dtype=f32, device=dev)
        self.conic_opacity = torch.empty(nr, 4, dtype=f32, device=dev)
        self.rgb_depth = torch.empty(nr, 4, dtype=f32, device=dev)
        self.radius = torch.empty(nr, dtype=i32, device=dev)
        self.tiles_touched = torch.empty(nr, dtype=i32, device=dev)
        # the projection keeps what the backward needs of the SH colour, so the backward reads
        # 48 bytes per visible record instead of every Gaussian's 3 (D+1)^2 coefficients
        self.color_jac = (torch.empty(nr, 12, dtype=f32, device=dev)
                          if use_color_jac(cfg, model.sh_degree, self.n_views) else None)
        self.counts = torch.zeros(4, dtype=i32, device=dev)
        self.status = torch.zeros(1, dtype=i32, device=dev)
        self.tile_ranges = torch.zeros(self.total_tiles, 2, dtype=i32, device=dev)
        self.tile_order = torch.zeros(self.total_tiles, dtype=i32, device=dev)
        self.img = torch.empty(3 * self.total_pixels, dtype=f32, device=dev)
        self.T_final = torch.empty(self.total_pixels, dtype=f32, device=dev)
        self.last = torch.empty(self.total_pixels, dtype=i32, device=dev)
        self.depth = torch.empty(self.total_pixels, dtype=f32, device=dev) if with_depth else None
        self.dL_dimg = torch.empty(3 * self.total_pixels, dtype=f32, device=dev)
        self.loss = torch.zeros(self.n_views, dtype=f32, device=dev)
        self.set_max_pairs(max_pairs)
        hmax = max(int(c["height"]) for c in self.cams)
        wmax = max(int(c["width"]) for c in self.cams)
        self.loss_ws = _workspace(lib().gs_loss_workspace_size, hmax, wmax, device=dev)
        self.bwd_ws = _workspace(lib().gs_bwd_workspace_size, self.nrec, device=dev)
        self.stats_acc = torch.zeros(6, model.ld, dtype=f32, device=dev) if with_stats else None

    def set_max_pairs(self, max_pairs):
        dev = self.xy.device
        self.max_pairs = int(max_pairs)
        self.gauss_ids = torch.empty(max(self.max_pairs, 1), dtype=torch.int32, device=dev)
        self.block_mask = _workspace(lib().gs_block_mask_size, self.max_pairs, device=dev)
        self.sort_ws = _workspace(lib().gs_sort_workspace_size, self.nrec, self.max_pairs, device=dev)
        if self.cfg.segment:
            if getattr(self, "seg_items", 0) == 0:
                # the worst case for max_pairs, up to 65,536 items; fit_capacity grows it to the count measured
                n = C.c_size_t()
                _check(lib().gs_segment_workspace_size(self.max_pairs, self.cfg.segment, C.byref(n)),
                       "gs_segment_workspace_size")
                self.seg_items = min(65536, int(n.value) // 1433 + 16)
            self.set_seg_items(self.seg_items)
        else:
            self.seg_ws = None

    def set_seg_items(self, items):
        """Split workspace for `items` forward segment items."""
        self.seg_items = int(items)
        self.seg_ws = _workspace(lib().gs_segment_workspace_size_items, self.seg_items, device=self.xy.device)

    def seg_needed(self):
        """(split off for lack of room in the last forward, segment items that forward needed)."""
        h = self.seg_ws[:24].view(torch.int32).cpu().numpy()
        return bool(h[4]), int(h[5])

    def projected(self) -> Projected:
        return Projected(self.xy.data_ptr(), self.conic_opacity.data_ptr(), self.rgb_depth.data_ptr(),
                         self.radius.data_ptr(), self.tiles_touched.data_ptr(), self.ld,
                         None if self.color_jac is None else self.color_jac.data_ptr())

    def binning(self) -> Binning:
        return Binning(self.gauss_ids.data_ptr(), self.tile_ranges.data_ptr(), self.counts.data_ptr(),
                       self.block_mask.data_ptr(), self.tile_order.data_ptr(), self.max_pairs)

    def frame(self) -> Frame:
        return Frame(self.img.data_ptr(), self.T_final.data_ptr(), self.last.data_ptr(),
                     None if self.depth is None else self.depth.data_ptr(),
                     None if self.seg_ws is None else self.seg_ws.data_ptr(),
                     0 if self.seg_ws is None else self.seg_ws.numel())

    def stats(self):
        return None if self.stats_acc is None else Stats(self.stats_acc.data_ptr(), self.stats_acc.shape[1])

    def view_image(self, v, t=None):
        t = self.img if t is None else t
        W, H = int(self.cams[v]["width"]), int(self.cams[v]["height"])
        o = 3 * int(self.pixel_offset[v])
        return t[o:o + 3 * H * W].view(3, H, W)

    def view_plane(self, t, v):
        W, H = int(self.cams[v]["width"]), int(self.cams[v]["height"])
        o = int(self.pixel_offset[v])
        return t[o:o + H * W].view(H, W)


def _workspace(fn, *args, device):
    n = C.c_size_t()
    _check(fn(*args, C.byref(n)), fn.__name__)
    return torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------
# the C entry points (argument marshalling only)

def gs_project(model: GaussianModel, buf: Buffers, stream=None):
    arr = camera_array(buf.cams)
    _check(lib().gs_project(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()), C.byref(buf.projected()),
                            _ptr(buf.status), _stream(stream)), "gs_project")


def gs_sort(buf: Buffers, stream=None):
    arr = camera_array(buf.cams)
    _check(lib().gs_sort(C.byref(buf.projected()), arr, buf.n_views, C.byref(buf.cfg.c()), C.byref(buf.binning()),
                         _ptr(buf.sort_ws), buf.sort_ws.numel(), _ptr(buf.status), _stream(stream)), "gs_sort")


def gs_render_fwd(buf: Buffers, stream=None):
    arr = camera_array(buf.cams)
    _check(lib().gs_render_fwd(C.byref(buf.projected()), C.byref(buf.binning()), arr, buf.n_views,
                               C.byref(buf.cfg.c()), C.byref(buf.frame()), _stream(stream)), "gs_render_fwd")


def gs_loss(buf: Buffers, target: torch.Tensor, lambda_dssim=0.2, stream=None, img=None):
    arr = camera_array(buf.cams)
    _check(lib().gs_loss(_ptr(buf.img if img is None else img), _ptr(target), arr, buf.n_views, float(lambda_dssim),
                         _ptr(buf.loss), _ptr(buf.dL_dimg), _ptr(buf.loss_ws), buf.loss_ws.numel(),
                         _stream(stream)), "gs_loss")


def reg_workspace(device="cuda"):
    n = C.c_size_t()
    _check(lib().gs_reg_workspace_size(C.byref(n)), "gs_reg_workspace_size")
    return torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=device)


def gs_geo_loss(buf: Buffers, prior, weight, loss_out, dL_ddepth, ws, stream=None):
    """weight * L_geo per view into loss_out, weight * dL/dD^ into dL_ddepth."""
    arr = camera_array(buf.cams)
    _check(lib().gs_geo_loss(_ptr(buf.depth), _ptr(prior), arr, buf.n_views, float(weight), _ptr(loss_out),
                             _ptr(dL_ddepth), _ptr(ws), ws.numel(), _stream(stream)), "gs_geo_loss")


def gs_iso_loss(model: GaussianModel, weight, loss_out, grads: GaussianModel, ws, stream=None):
    """weight * L_iso into loss_out[0]; adds its gradient into grads' log-scale planes."""
    _check(lib().gs_iso_loss(C.byref(model.c()), float(weight), _ptr(loss_out),
                             None if grads is None else C.byref(grads.c()), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_iso_loss")


def gs_loss_static(img, target, cams, loss_out, dL_dimg, lambda_dssim=0.2, stream=None):
    """gs_loss with the library's own scratch array (no workspace argument),
    for callers that cannot allocate device memory; views up to 1280x720."""
    arr = camera_array(cams)
    _check(lib().gs_loss_static(_ptr(img), _ptr(target), arr, len(cams), float(lambda_dssim), _ptr(loss_out),
                                _ptr(dL_dimg), _stream(stream)), "gs_loss_static")


def gs_render_bwd(model: GaussianModel, grads: GaussianModel, buf: Buffers, target=None, tau_err=0.1,
                  accumulate=False, with_stats=True, dL_ddepth=None, dL_dimg=None, stream=None):
    arr = camera_array(buf.cams)
    st = buf.stats() if with_stats else None
    _check(lib().gs_render_bwd(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()), C.byref(buf.projected()),
                               C.byref(buf.binning()), C.byref(buf.frame()),
                               _ptr(buf.dL_dimg if dL_dimg is None else dL_dimg), _ptr(dL_ddepth), _ptr(target),
                               _ptr(buf.loss), float(tau_err), None if grads is None else C.byref(grads.c()),
                               int(bool(accumulate)), None if st is None else C.byref(st), _ptr(buf.bwd_ws),
                               buf.bwd_ws.numel(), _stream(stream)), "gs_render_bwd")


def gs_project_bwd(model: GaussianModel, grads: GaussianModel, buf: Buffers, accumulate=False, with_stats=True,
                   stream=None, rows=None):
    """The projection half of the backward, from the per-record gradients
    that gs_render_bwd(grads=None) left in the workspace.  rows (a [ld] uint8
    device tensor): write only the rows of Gaussians some view sees and mark
    them there (gs_project_bwd_rows), for gs_adam(rows=...)."""
    arr = camera_array(buf.cams)
    st = buf.stats() if with_stats else None
    if rows is not None:
        assert not accumulate and rows.dtype == torch.uint8 and rows.numel() >= model.ld
        _check(lib().gs_project_bwd_rows(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()),
                                         C.byref(buf.projected()), _ptr(buf.bwd_ws), buf.bwd_ws.numel(),
                                         _ptr(buf.loss), C.byref(grads.c()), None if st is None else C.byref(st),
                                         _ptr(rows), _stream(stream)), "gs_project_bwd_rows")
        return
    _check(lib().gs_project_bwd(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()), C.byref(buf.projected()),
                                _ptr(buf.bwd_ws), buf.bwd_ws.numel(), _ptr(buf.loss), C.byref(grads.c()),
                                int(bool(accumulate)), None if st is None else C.byref(st), _stream(stream)),
           "gs_project_bwd")


class StoredLists:
    """Per-pixel blend lists (record id, alpha) of gs_render_fwd_lists, with
    their offsets; capacity in blend events (grown by MappingStep.fit_capacity)."""

    def __init__(self, total_pixels, capacity, device):
        self.total_pixels = int(total_pixels)
        self.offsets = torch.zeros(self.total_pixels + 1, dtype=torch.int64, device=device)
        self.scan_ws = _workspace(lib().gs_list_workspace_size, self.total_pixels, device=device)
        self.set_capacity(capacity)

    def set_capacity(self, capacity):
        dev = self.offsets.device
        self.capacity = int(capacity)
        self.ids = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=dev)
        self.alpha = torch.empty(max(self.capacity, 1), dtype=torch.float32, device=dev)

    def events(self):
        """Blend events of the last forward (host sync)."""
        return int(self.offsets[self.total_pixels].item())

    def nbytes(self):
        return self.offsets.numel() * 8 + self.ids.numel() * 4 + self.alpha.numel() * 4 + self.scan_ws.numel()


def gs_render_fwd_lists(buf: Buffers, lists: StoredLists, stream=None):
    arr = camera_array(buf.cams)
    _check(lib().gs_render_fwd_lists(C.byref(buf.projected()), C.byref(buf.binning()), arr, buf.n_views,
                                     C.byref(buf.cfg.c()), C.byref(buf.frame()), _ptr(lists.offsets), _ptr(lists.ids),
                                     _ptr(lists.alpha), lists.capacity, _ptr(lists.scan_ws), lists.scan_ws.numel(),
                                     _ptr(buf.status), _stream(stream)), "gs_render_fwd_lists")


def gs_render_bwd_lists(model: GaussianModel, grads: GaussianModel, buf: Buffers, lists: StoredLists, target=None,
                        tau_err=0.1, accumulate=False, with_stats=True, stream=None):
    arr = camera_array(buf.cams)
    st = buf.stats() if with_stats else None
    _check(lib().gs_render_bwd_lists(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()),
                                     C.byref(buf.projected()), C.byref(buf.frame()), _ptr(lists.offsets),
                                     _ptr(lists.ids), _ptr(lists.alpha), lists.capacity, _ptr(buf.dL_dimg),
                                     _ptr(target), _ptr(buf.loss), float(tau_err),
                                     None if grads is None else C.byref(grads.c()), int(bool(accumulate)),
                                     None if st is None else C.byref(st), _ptr(buf.bwd_ws), buf.bwd_ws.numel(),
                                     _stream(stream)), "gs_render_bwd_lists")


def gs_project_bwd_adam(model: GaussianModel, buf: Buffers, exp_avg: GaussianModel, exp_avg_sq: GaussianModel, lr,
                        step, beta1=0.9, beta2=0.999, eps=1e-15, iso_weight=0.0, grads_in: GaussianModel = None,
                        with_stats=True, stream=None, step_device=None):
    """Projection backward from the per-record gradients that gs_render_bwd(grads=None) left in buf.bwd_ws,
    fused with one Adam step (no gradient buffer)."""
    lrs = (C.c_float * 6)(*[float(x) for x in lr])
    st = buf.stats() if with_stats else None
    arr = camera_array(buf.cams)
    _check(lib().gs_project_bwd_adam(C.byref(model.c()), arr, buf.n_views, C.byref(buf.cfg.c()),
                                     C.byref(buf.projected()), _ptr(buf.bwd_ws), buf.bwd_ws.numel(), _ptr(buf.loss),
                                     C.byref(grads_in.c()) if grads_in is not None else None, float(iso_weight),
                                     C.byref(exp_avg.c()), C.byref(exp_avg_sq.c()), C.byref(lrs), beta1, beta2, eps,
                                     int(step), _ptr(step_device), C.byref(st) if st is not None else None,
                                     _stream(stream)), "gs_project_bwd_adam")


def gs_adam(model: GaussianModel, grads: GaussianModel, exp_avg: GaussianModel, exp_avg_sq: GaussianModel, lr,
            step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None, step_device=None, rows=None):
    """rows: the marks of gs_project_bwd(rows=...); unmarked rows take a zero gradient."""
    lrs = (C.c_float * 6)(*[float(x) for x in lr])
    if rows is not None:
        _check(lib().gs_adam_rows(C.byref(model.c()), C.byref(grads.c()), C.byref(exp_avg.c()),
                                  C.byref(exp_avg_sq.c()), _ptr(rows), C.byref(lrs), beta1, beta2, eps, int(step),
                                  _ptr(step_device), _stream(stream)), "gs_adam_rows")
        return
    _check(lib().gs_adam(C.byref(model.c()), C.byref(grads.c()), C.byref(exp_avg.c()), C.byref(exp_avg_sq.c()),
                         C.byref(lrs), beta1, beta2, eps, int(step), _ptr(step_device), _stream(stream)), "gs_adam")


def gs_adam_part(model: GaussianModel, grads, exp_avg: GaussianModel, exp_avg_sq: GaussianModel, buf: Buffers,
                 part, lr, step, rows=None, beta1=0.9, beta2=0.999, eps=1e-15, stream=None, step_device=None):
    """One of the two disjoint parts of gs_adam(rows=...): part 2 the Gaussians no view of
    buf sees (from the projection's radii; runs right after gs_project), part 1 the rows
    marked by gs_project_bwd(rows=...)."""
    lrs = (C.c_float * 6)(*[float(x) for x in lr])
    _check(lib().gs_adam_part(C.byref(model.c()), None if grads is None else C.byref(grads.c()),
                              C.byref(exp_avg.c()), C.byref(exp_avg_sq.c()), _ptr(rows), _ptr(buf.radius),
                              buf.n_views, int(part), C.byref(lrs), beta1, beta2, eps, int(step), _ptr(step_device),
                              _stream(stream)), "gs_adam_part")


def gs_prune_stats(stats_acc: torch.Tensor, n, n_views, scores: dict, ws: torch.Tensor, tau_d=5.0, tau_p=0.99,
                   stream=None):
    st = Stats(stats_acc.data_ptr(), stats_acc.shape[1])
    cs = ChunkScores(*[scores[k].data_ptr() for k in ("S_d", "S_p", "prune_max", "densify", "prune")])
    _check(lib().gs_prune_stats(C.byref(st), int(n), int(n_views), float(tau_d), float(tau_p), C.byref(cs),
                                _ptr(ws), ws.numel(), _stream(stream)), "gs_prune_stats")


def prune_buffers(n, device="cuda"):
    ws = _workspace(lib().gs_prune_workspace_size, n, device=device)
    f32, u8 = torch.float32, torch.uint8
    return dict(S_d=torch.zeros(n, dtype=f32, device=device), S_p=torch.zeros(n, dtype=f32, device=device),
                prune_max=torch.zeros(n, dtype=f32, device=device), densify=torch.zeros(n, dtype=u8, device=device),
                prune=torch.zeros(n, dtype=u8, device=device)), ws


def actions_workspace(n, device="cuda"):
    return _workspace(lib().gs_actions_workspace_size, n, device=device)


def gs_densify_prune(model: GaussianModel, densify, prune, noise, split_log_scale, split_factor=1.6, exp_avg=None,
                     exp_avg_sq=None, capacity=None, status=None, ws=None, stream=None):
    """Applies the densify / prune decisions ([n] uint8 device tensors); noise is a [6, ld] float32 tensor of
    standard normal samples.  Returns (model, exp_avg, exp_avg_sq, n_out) with n_out a device int64 tensor; the new
    model's n is the host count (one synchronisation)."""
    dev = model.data.device
    cap = padded(2 * model.n) if capacity is None else int(capacity)
    assert cap % 4 == 0

    def empty():
        return GaussianModel(0, model.sh_degree, device=dev,
                             data=torch.zeros(model.K, max(cap, 4), dtype=torch.float32, device=dev))

    out = empty()
    moments = exp_avg is not None
    mo, vo = (empty(), empty()) if moments else (None, None)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = actions_workspace(model.n, device=dev) if ws is None else ws
    _check(lib().gs_densify_prune(C.byref(model.c()), C.byref(exp_avg.c()) if moments else None,
                                  C.byref(exp_avg_sq.c()) if moments else None, _ptr(densify), _ptr(prune),
                                  _ptr(noise), float(split_log_scale), float(split_factor), C.byref(out.c()),
                                  C.byref(mo.c()) if moments else None, C.byref(vo.c()) if moments else None,
                                  _ptr(n_out), _ptr(status), _ptr(ws), ws.numel(), _stream(stream)),
           "gs_densify_prune")
    n = min(int(n_out.item()), cap)
    for m in (out, mo, vo):
        if m is not None:
            m.n = n
    return out, mo, vo, n_out


def gs_reorder(model: GaussianModel, extra=(), perm=None, ws=None, stream=None):
    """Puts the rows of model and of every extra [planes, ld] float32 tensor (Adam
    moments, per-Gaussian statistics) in the Morton order of the means, in place.
    perm: an [n] int32 device tensor receiving the previous row of each new row
    (allocated when None).  Returns perm."""
    dev = model.data.device
    extra = list(extra)
    for t in extra:
        assert t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == model.ld and t.is_contiguous()
    sets = (PlaneSet * max(1, len(extra)))(*[PlaneSet(t.data_ptr(), model.ld, t.shape[0]) for t in extra])
    perm = torch.empty(max(model.n, 1), dtype=torch.int32, device=dev) if perm is None else perm
    if ws is None:
        maxp = max([model.K] + [t.shape[0] for t in extra])
        ws = _workspace(lib().gs_reorder_workspace_size, model.n, model.ld, maxp, device=dev)
    _check(lib().gs_reorder(C.byref(model.c()), sets, len(extra), _ptr(perm), _ptr(ws), ws.numel(),
                            _stream(stream)), "gs_reorder")
    return perm[:model.n]


MLP_INPUTS, MLP_HIDDEN, MLP_WEIGHTS, MLP_RING = 16, 64, 5378, 8


def mlp_init(seed=0, device="cuda"):
    """He-normal weights and zero biases in the flat layout of gs_mlp_forward."""
    g = torch.Generator().manual_seed(int(seed))
    w = torch.zeros(MLP_WEIGHTS, dtype=torch.float32)
    w[0:1024] = torch.randn(1024, generator=g) * (2.0 / 16) ** 0.5
    w[1088:5184] = torch.randn(4096, generator=g) * (2.0 / 64) ** 0.5
    w[5248:5376] = torch.randn(128, generator=g) * (1.0 / 64) ** 0.5
    return w.to(device)


def gs_mlp_push_blend(stats_acc: torch.Tensor, n, ring: torch.Tensor, slot, stream=None):
    st = Stats(stats_acc.data_ptr(), stats_acc.shape[1])
    _check(lib().gs_mlp_push_blend(C.byref(st), int(n), _ptr(ring), ring.shape[1], int(slot), _stream(stream)),
           "gs_mlp_push_blend")


def gs_mlp_features(model: GaussianModel, stats_acc: torch.Tensor, ring: torch.Tensor, head, cam_centre,
                    feat: torch.Tensor, stream=None):
    st = Stats(stats_acc.data_ptr(), stats_acc.shape[1])
    cc = (C.c_float * 3)(*[float(x) for x in cam_centre])
    _check(lib().gs_mlp_features(C.byref(model.c()), C.byref(st), _ptr(ring), int(head), C.byref(cc), _ptr(feat),
                                 _stream(stream)), "gs_mlp_features")


def gs_mlp_forward(feat: torch.Tensor, n, weights, prob=None, densify=None, prune=None, status=None, stream=None,
                   max_polls=-1):
    _check(lib().gs_mlp_forward(_ptr(feat), int(n), feat.shape[1], _ptr(weights), _ptr(prob), _ptr(densify),
                                _ptr(prune), _ptr(status), int(max_polls), _stream(stream)), "gs_mlp_forward")


def gs_mlp_train_grad(feat: torch.Tensor, y_densify, y_prune, n, weights, grad, loss, status=None, stream=None):
    _check(lib().gs_mlp_train_grad(_ptr(feat), _ptr(y_densify), _ptr(y_prune), int(n), feat.shape[1], _ptr(weights),
                                   _ptr(grad), _ptr(loss), _ptr(status), _stream(stream)), "gs_mlp_train_grad")


def gs_mlp_adam(weights, grad, exp_avg, exp_avg_sq, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().gs_mlp_adam(_ptr(weights), _ptr(grad), _ptr(exp_avg), _ptr(exp_avg_sq), float(lr), float(beta1),
                             float(beta2), float(eps), int(step), _stream(stream)), "gs_mlp_adam")


# --------------------------------------------------------------------------
# one mapping iteration

# Learning rates per parameter group (means, log-scales, quaternion, opacity,
# SH degree 0, SH degree >= 1); the paper prints none, these are the usual
# 3DGS values with the mean rate scaled by the scene extent.
def default_lr(extent=1.0):
    return (1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)


class MappingStep:
    """render -> L_photo -> backward -> Adam over one chunk of views."""

    def __init__(self, model: GaussianModel, cams, cfg: Config = None, max_pairs=None, lambda_dssim=0.2,
                 tau_err=0.1, lr=None, with_stats=True, with_depth=False, depth_prior=None, lambda_geo=0.01,
                 lambda_iso=0.0, moments=None, step_count=0, fused_adam=False, stored_lists=False):
        self.model = model
        self.cfg = cfg or Config()
        self.lambda_dssim, self.tau_err = lambda_dssim, tau_err
        # L_total = L_photo + lambda_geo L_geo (when a depth prior is given) + lambda_iso L_iso
        self.depth_prior, self.lambda_geo, self.lambda_iso = depth_prior, lambda_geo, lambda_iso
        with_depth = with_depth or depth_prior is not None
        self.lr = lr or default_lr()
        self.with_stats = with_stats
        self._grads = None  # allocated on first use: the fused path needs no gradient buffer
        self._reorder_ws = None
        self._rows = None
        self._adam_stream = None
        # Adam moments: zero, or carried over (e.g. through gs_densify_prune)
        self.exp_avg, self.exp_avg_sq = moments if moments is not None else (model.like(), model.like())
        assert self.exp_avg.ld == model.ld and self.exp_avg_sq.ld == model.ld
        self.step_count = int(step_count)
        # Adam inside the projection backward: no gradient buffer (236 MB less at 1M
        # Gaussians, SH3) but, at its occupancy, slower than projection backward + Adam
        self.fused_adam = fused_adam
        if max_pairs is None:  # a first guess; fit_capacity sizes it to the count measured
            max_pairs = min(max(1 << 16, 8 * model.n * len(cams)), 1 << 25)
        if stored_lists:  # the stored-list backward: no split, no depth term, no fused Adam
            assert not with_depth and not fused_adam and lambda_iso == 0.0
            self.cfg = Config(**{**self.cfg.__dict__, "segment": 0})
        self.buf = Buffers(model, cams, self.cfg, max_pairs, with_depth=with_depth, with_stats=with_stats)
        self.lists = (StoredLists(self.buf.total_pixels, 4 * self.buf.total_pixels, model.data.device)
                      if stored_lists else None)
        dev = model.data.device
        self.reg_ws = reg_workspace(dev) if (depth_prior is not None or lambda_iso > 0) else None
        self.geo_loss = torch.zeros(len(cams), dtype=torch.float32, device=dev)
        self.iso_loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.dL_ddepth = (torch.empty(self.buf.total_pixels, dtype=torch.float32, device=dev)
                          if depth_prior is not None else None)

    @property
    def grads(self) -> GaussianModel:
        if self._grads is None:
            self._grads = self.model.like()
        return self._grads

    @grads.setter
    def grads(self, value: GaussianModel):
        self._grads = value

    def set_cameras(self, cams):
        assert len(cams) == self.buf.n_views
        for c_new, c_old in zip(cams, self.buf.cams):
            assert (c_new["width"], c_new["height"]) == (c_old["width"], c_old["height"])
        self.buf.cams = list(cams)

    def forward(self, stream=None):
        b = self.buf
        b.status.zero_()
        gs_project(self.model, b, stream)
        gs_sort(b, stream)
        if self.lists is not None:
            gs_render_fwd_lists(b, self.lists, stream)
        else:
            gs_render_fwd(b, stream)

    @property
    def grad_rows(self):
        """Whether an optimising step writes only the gradient rows of the Gaussians some
        view sees (gs_project_bwd_rows) and Adam reads the others as zero (gs_adam_rows);
        not with the isotropy term, whose gradient reaches every Gaussian."""
        if self.fused_adam or self.lists is not None or self.lambda_iso > 0:
            return False
        return self.cfg.grad_rows is not False

    @property
    def adam_split(self):
        """Whether a captured step runs the Adam of the Gaussians no view sees (which needs only
        the projection) on a second stream beside the rest of the step."""
        return self.grad_rows and self.cfg.adam_overlap is not False

    @property
    def rows(self) -> torch.Tensor:
        if self._rows is None or self._rows.numel() != self.model.ld:
            self._rows = torch.zeros(self.model.ld, dtype=torch.uint8, device=self.model.data.device)
        return self._rows

    def _losses_and_backward(self, target, stream=None):
        gs_loss(self.buf, target, self.lambda_dssim, stream)
        if self.lists is not None:
            gs_render_bwd_lists(self.model, self.grads, self.buf, self.lists, target, self.tau_err,
                                with_stats=self.with_stats, stream=stream)
            return
        if self.depth_prior is not None:
            gs_geo_loss(self.buf, self.depth_prior, self.lambda_geo, self.geo_loss, self.dL_ddepth, self.reg_ws, stream)
        gs_render_bwd(self.model, self.grads, self.buf, target, self.tau_err, with_stats=self.with_stats,
                      dL_ddepth=self.dL_ddepth, stream=stream)
        if self.lambda_iso > 0:
            gs_iso_loss(self.model, self.lambda_iso, self.iso_loss, self.grads, self.reg_ws, stream)

    def _losses_backward_adam(self, target, stream=None, step=None, step_device=None):
        """Losses, the compositing backward, then the projection backward fused
        with the Adam step (the gradient is never stored)."""
        gs_loss(self.buf, target, self.lambda_dssim, stream)
        if self.depth_prior is not None:
            gs_geo_loss(self.buf, self.depth_prior, self.lambda_geo, self.geo_loss, self.dL_ddepth, self.reg_ws, stream)
        gs_render_bwd(self.model, None, self.buf, target, self.tau_err, with_stats=self.with_stats,
                      dL_ddepth=self.dL_ddepth, stream=stream)
        if self.lambda_iso > 0:
            gs_iso_loss(self.model, self.lambda_iso, self.iso_loss, None, self.reg_ws, stream)
        gs_project_bwd_adam(self.model, self.buf, self.exp_avg, self.exp_avg_sq, self.lr,
                            1 if step is None else step, iso_weight=self.lambda_iso, with_stats=self.with_stats,
                            stream=stream, step_device=step_device)

    def total_loss(self):
        """L_total = sum over views of L_photo (+ lambda_geo L_geo) + lambda_iso L_iso (device tensor)."""
        t = self.buf.loss.sum()
        if self.depth_prior is not None:
            t = t + self.geo_loss.sum()
        if self.lambda_iso > 0:
            t = t + self.iso_loss[0]
        return t

    def step(self, target, stream=None, optimize=True):
        """One iteration on device-resident targets (frame layout).  An optimising step
        with grad_rows leaves the gradient rows of Gaussians no view sees as they were."""
        self.forward(stream)
        if optimize and self.fused_adam:
            self.step_count += 1
            self._losses_backward_adam(target, stream, step=self.step_count)
            return self.buf.loss
        if optimize and self.grad_rows:
            gs_loss(self.buf, target, self.lambda_dssim, stream)
            if self.depth_prior is not None:
                gs_geo_loss(self.buf, self.depth_prior, self.lambda_geo, self.geo_loss, self.dL_ddepth, self.reg_ws,
                            stream)
            gs_render_bwd(self.model, None, self.buf, target, self.tau_err, with_stats=self.with_stats,
                          dL_ddepth=self.dL_ddepth, stream=stream)
            gs_project_bwd(self.model, self.grads, self.buf, with_stats=self.with_stats, stream=stream, rows=self.rows)
            self.step_count += 1
            gs_adam(self.model, self.grads, self.exp_avg, self.exp_avg_sq, self.lr, self.step_count, stream=stream,
                    rows=self.rows)
            return self.buf.loss
        self._losses_and_backward(target, stream)
        if optimize:
            self.step_count += 1
            gs_adam(self.model, self.grads, self.exp_avg, self.exp_avg_sq, self.lr, self.step_count, stream=stream)
        return self.buf.loss

    def reorder(self, stream=None):
        """Puts the map's rows (parameters, Adam moments, statistics) in the Morton
        order of the means (gs_reorder): the Gaussians one view sees then share
        memory sectors.  Every buffer keeps its address, so captured graphs stay
        valid.  Returns the [n] int32 device permutation (new row i is previous
        row perm[i])."""
        if self._reorder_ws is None:
            maxp = max(self.model.K, 6)
            self._reorder_ws = _workspace(lib().gs_reorder_workspace_size, self.model.n, self.model.ld, maxp,
                                          device=self.model.data.device)
        extra = [self.exp_avg.data, self.exp_avg_sq.data]
        if self.buf.stats_acc is not None:
            extra.append(self.buf.stats_acc)
        return gs_reorder(self.model, extra, ws=self._reorder_ws, stream=stream)

    # stage boundaries that capture(events=...) marks, in order
    STAGES = ("project", "sort", "render_fwd", "loss", "render_bwd", "project_bwd", "adam")
    STAGES_FUSED = ("project", "sort", "render_fwd", "loss", "render_bwd", "project_bwd_adam")

    def capture(self, target, stream=None, events=None, keep_graph=False):
        """Captures one whole iteration (status reset, project, sort, render,
        loss, backward, Adam) for the current cameras and `target` buffer into
        a CUDA graph.  Adam reads its step from a device counter that the graph
        advances, so replays are successive iterations.  The pair buffer keeps
        the capacity it has now (size it with fit_capacity first).
        events: optional timing events created with external=True, one more
        than the stages (STAGES, or STAGES_FUSED with fused_adam); the graph
        records them at the stage boundaries, so every replay times its stages."""
        dev = self.model.data.device
        if getattr(self, "step_dev", None) is None:
            self.step_dev = torch.full((1,), self.step_count, dtype=torch.int64, device=dev)
        stages = self.STAGES_FUSED if self.fused_adam else self.STAGES
        assert events is None or len(events) == len(stages) + 1
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        graph = torch.cuda.CUDAGraph(keep_graph=keep_graph)  # keep_graph: its nodes stay readable

        def mark(i):
            if events is not None:
                events[i].record(side)

        with torch.cuda.graph(graph, stream=side):
            b = self.buf
            b.status.zero_()
            self.step_dev.add_(1)
            mark(0)
            gs_project(self.model, b)
            mark(1)
            split = self.adam_split
            if split:
                # Adam of the Gaussians no view sees needs only the projection: it runs on a
                # second stream beside the rest of the step (little DRAM traffic)
                if self._adam_stream is None:
                    self._adam_stream = torch.cuda.Stream(device=dev)
                fork = torch.cuda.Event()
                fork.record(side)
                self._adam_stream.wait_event(fork)
                with torch.cuda.stream(self._adam_stream):
                    gs_adam_part(self.model, None, self.exp_avg, self.exp_avg_sq, self.buf, 2, self.lr, 1,
                                 step_device=self.step_dev)
                join = torch.cuda.Event()
                join.record(self._adam_stream)
            gs_sort(b)
            mark(2)
            gs_render_fwd(b)
            mark(3)
            gs_loss(self.buf, target, self.lambda_dssim)
            if self.depth_prior is not None:
                gs_geo_loss(self.buf, self.depth_prior, self.lambda_geo, self.geo_loss, self.dL_ddepth, self.reg_ws)
            mark(4)
            # the compositing backward leaves per-record gradients in the workspace
            gs_render_bwd(self.model, None, self.buf, target, self.tau_err, with_stats=self.with_stats,
                          dL_ddepth=self.dL_ddepth)
            mark(5)
            if self.fused_adam:
                if self.lambda_iso > 0:
                    gs_iso_loss(self.model, self.lambda_iso, self.iso_loss, None, self.reg_ws)
                gs_project_bwd_adam(self.model, self.buf, self.exp_avg, self.exp_avg_sq, self.lr, 1,
                                    iso_weight=self.lambda_iso, with_stats=self.with_stats,
                                    step_device=self.step_dev)
                mark(6)
            else:
                grads, rows = self.grads, (self.rows if self.grad_rows else None)
                gs_project_bwd(self.model, grads, self.buf, with_stats=self.with_stats, rows=rows)
                if self.lambda_iso > 0:
                    gs_iso_loss(self.model, self.lambda_iso, self.iso_loss, grads, self.reg_ws)
                mark(6)
                if split:
                    gs_adam_part(self.model, grads, self.exp_avg, self.exp_avg_sq, self.buf, 1, self.lr, 1,
                                 rows=rows, step_device=self.step_dev)
                    mark(7)
                    side.wait_event(join)
                else:
                    gs_adam(self.model, grads, self.exp_avg, self.exp_avg_sq, self.lr, 1, step_device=self.step_dev,
                            rows=rows)
                    mark(7)
        torch.cuda.current_stream(dev).wait_stream(side)
        return graph

    def replay(self, graph):
        graph.replay()
        self.step_count += 1
        return self.buf.loss

    def check_status(self):
        """Host check after the stream completed: raises on capacity overflow."""
        st = int(self.buf.status.item())
        if st & (1 << GS_ERR_CAPACITY):
            needed = int(self.buf.counts[2].item())
            if needed > self.buf.max_pairs:
                raise GSError("pair capacity exceeded: %d pairs needed, %d available" % (needed, self.buf.max_pairs))
            if self.lists is not None and self.lists.events() > self.lists.capacity:
                raise GSError("stored-list capacity exceeded: %d blend events, %d slots"
                              % (self.lists.events(), self.lists.capacity))
            raise GSError("capacity exceeded")
        return st

    def fit_capacity(self, slack=1.25):
        """Runs the forward once and sizes the pair buffer (and the split
        workspace) to the counts seen."""
        self.forward()
        torch.cuda.synchronize()
        needed = int(self.buf.counts[2].item())
        if needed > self.buf.max_pairs or needed * slack * 2 < self.buf.max_pairs:
            self.buf.set_max_pairs(max(1024, int(needed * slack)))
            self.forward()
            torch.cuda.synchronize()
        if self.lists is not None:
            ev = self.lists.events()
            if ev > self.lists.capacity:
                self.lists.set_capacity(int(ev * max(slack, 1.1)) + 1024)
                self.forward()
                torch.cuda.synchronize()
        if self.buf.seg_ws is not None:
            off, items = self.buf.seg_needed()
            if off or items > self.buf.seg_items:
                self.buf.set_seg_items(int(items * max(slack, 1.25)) + 64)
                self.forward()
                torch.cuda.synchronize()
        self.check_status()
        return needed


def launches_per_step(total_tiles, views=1, lambda_dssim=0.2, segment=512, fused_adam=False, adam_split=False):
    """Kernel launches of the library in one mapping iteration (memsets not
    counted): project 1; sort 2 (visible records: count, compact) + 3 per LSD
    pass (count, scan, scatter: 4 depth passes, 1 view pass with several views,
    one per 8 tile bits, or 1 unpack for a single tile) + 4 (pair counts,
    offsets, emission, long records) + 2 (render schedule); render 1 (4 with
    the split: plan, segments, combine, re-runs); loss 2 per view; backward 2
    (compositing, projection); Adam 1 unless fused into the projection backward
    (2 when split into the seen rows and the background part)."""
    tile_bits = 0
    while (1 << tile_bits) < total_tiles:
        tile_bits += 1
    tile_passes = (tile_bits + 7) // 8
    sort = 2 + 3 * (4 + (1 if views > 1 else 0) + tile_passes) + (0 if tile_passes else 1) + 4 + 2
    loss = 2 * views
    return 1 + sort + (4 if segment else 1) + loss + 2 + (0 if fused_adam else 2 if adam_split else 1)
