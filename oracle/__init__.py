"""FP64 CPU oracle of the differentiable 3D Gaussian splatting mapping step.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this module; the product package never imports
it and shares no code with it.  The arithmetic lives in ``gs_oracle.c`` (plain
C, FP64, written from the mathematics); this file only marshals numpy arrays.

Paper anchors: compositing and transmittance (Supp. D.2), the photometric loss
(Supp. D.4), the lifecycle scores (Supp. E.1, E.2) and their aggregation over
chunks (Sec. 3.3.2).  The readings the paper leaves open (projection, SH colour,
binning order, thresholds, SSIM window, Adam) are listed in the C header.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

# pixel flags of or_render (near-threshold events, see gs_oracle.h)
OR_FLAG_NEAR_ALPHA_MIN = 1
OR_FLAG_NEAR_T_CUT = 2
OR_FLAG_NEAR_ALPHA_MAX = 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
          "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard"]


def build(force: bool = False) -> str:
    """Compile the oracle library (plain gcc; no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gs_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class _Cfg(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_z", C.c_double),
                ("dilation", C.c_double), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("t_min", C.c_double), ("tan_clamp", C.c_double), ("bg", C.c_double * 3),
                ("fp32_positions", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class _Projected(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in (
        "u", "v", "z", "conic", "cov2d", "rgb", "rgb_clamped", "rgb_raw", "opacity", "radius",
        "radius_exact", "rect", "tiles_touched", "u32", "v32", "z32")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        L.or_sh_eval.argtypes = [i32, vp, vp, vp]
        L.or_quat_to_rot.argtypes = [vp, vp]
        L.or_project.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Cfg), C.POINTER(_Projected)]
        L.or_bin.argtypes = [C.POINTER(_Projected), i64, C.POINTER(_Camera), C.POINTER(_Cfg), i64, vp, vp, vp]
        L.or_bin.restype = i64
        L.or_render.argtypes = [C.POINTER(_Projected), vp, vp, C.POINTER(_Camera), C.POINTER(_Cfg),
                                vp, vp, vp, vp, vp, vp]
        L.or_loss.argtypes = [vp, vp, i32, i32, i32, d, vp, vp]
        L.or_loss.restype = d
        L.or_ssim_map.argtypes = [vp, vp, i32, i32, i32, vp]
        L.or_render_backward.argtypes = [C.POINTER(_Projected), i64, vp, vp, C.POINTER(_Camera), C.POINTER(_Cfg),
                                         vp, vp, vp, vp, d, d, d, vp, vp, vp]
        L.or_project_backward.argtypes = [C.POINTER(_Params), C.POINTER(_Camera), C.POINTER(_Cfg),
                                          C.POINTER(_Projected), vp, vp, vp, vp, vp, vp]
        L.or_adam.argtypes = [i64, vp, vp, vp, vp, vp, d, d, d, i64]
        L.or_prune_finalize.argtypes = [i64, vp, vp, vp, i32, d, d, vp, vp, vp, vp, vp]
        L.or_geo_loss.argtypes = [vp, vp, i64, vp]
        L.or_geo_loss.restype = d
        L.or_iso_loss.argtypes = [i64, vp, vp]
        L.or_iso_loss.restype = d
        L.or_mlp_num_weights.restype = i32
        L.or_mlp_forward.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        L.or_mlp_bce_grad.argtypes = [i64, vp, vp, vp, i32, vp, vp, vp]
        L.or_mlp_bce_grad.restype = d
        L.or_mlp_features.argtypes = [i64, vp, vp, vp, vp, vp, i32, vp, vp]
        L.or_densify_prune.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, d, d, i64, vp, vp, vp]
        L.or_densify_prune.restype = i64
        L.or_init_saliency.argtypes = [i32, i32, vp, vp, d, d, d, vp, vp]
        L.or_init_probability.argtypes = [i32, i32, vp, vp, vp, vp, d, d, d, d, vp]
        L.or_init_select.argtypes = [i32, i32, vp, vp, vp, C.POINTER(_Camera), d, i32, vp, vp, i64, vp, i64,
                                     vp, vp, vp, vp, vp, vp, d, d]
        L.or_init_select.restype = i64
        L.or_anchor_num_weights.restype = i32
        L.or_anchor_decode.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, d, i32]
        L.or_anchor_decode_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp]
        L.or_anchor_hidden.argtypes = [i64, vp, vp, vp, vp, i32, vp, vp]
        L.or_morton_order.argtypes = [i64, vp, vp, vp]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


@dataclass
class Cfg:
    """Rasteriser constants (readings R2-R8 of the C header)."""
    tile_w: int = 16
    tile_h: int = 16
    near_z: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    tan_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    fp32_positions: bool = True

    def c(self):
        return _Cfg(self.tile_w, self.tile_h, self.near_z, self.dilation, self.alpha_min, self.alpha_max,
                    self.t_min, self.tan_clamp, (C.c_double * 3)(*self.bg), int(self.fp32_positions))


def _cam(cam):
    R = np.asarray(cam["R"], dtype=np.float64).reshape(9)
    t = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    return _Camera((C.c_double * 9)(*R), (C.c_double * 3)(*t), float(cam["fx"]), float(cam["fy"]),
                   float(cam["cx"]), float(cam["cy"]), int(cam["width"]), int(cam["height"]))


def grid(cam, cfg: Cfg):
    return ((int(cam["width"]) + cfg.tile_w - 1) // cfg.tile_w,
            (int(cam["height"]) + cfg.tile_h - 1) // cfg.tile_h)


class Params:
    """FP64 array-of-structures parameters (keeps the arrays alive for ctypes)."""

    def __init__(self, p):
        n = int(np.asarray(p["means"]).shape[0])
        self.n = n
        self.sh_degree = int(p["sh_degree"])
        K = (self.sh_degree + 1) ** 2
        self.means = _f64(p["means"], (n, 3))
        self.log_scales = _f64(p["log_scales"], (n, 3))
        self.quats = _f64(p["quats"], (n, 4))
        self.opacity_logits = _f64(p["opacity_logits"], (n,))
        self.sh = _f64(p["sh"], (n, K, 3))

    def c(self):
        return _Params(self.n, self.sh_degree, _ptr(self.means), _ptr(self.log_scales), _ptr(self.quats),
                       _ptr(self.opacity_logits), _ptr(self.sh))

    def as_dict(self):
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh, sh_degree=self.sh_degree)


@dataclass
class Projected:
    n: int
    arrays: dict = field(default_factory=dict)

    def __getitem__(self, k):
        return self.arrays[k]

    def c(self):
        return _Projected(*[_ptr(self.arrays[k]) for k, _ in _Projected._fields_])


def sh_eval(D, d):
    """Real SH values (and Cartesian partial derivatives) at direction d."""
    K = (D + 1) ** 2
    d = _f64(d, (3,))
    Y = np.zeros(K)
    dY = np.zeros((K, 3))
    lib().or_sh_eval(D, _ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY


def quat_to_rot(q):
    q = _f64(q, (4,))
    R = np.zeros(9)
    lib().or_quat_to_rot(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def project(params, cam, cfg: Cfg) -> Projected:
    P = params if isinstance(params, Params) else Params(params)
    n = P.n
    a = dict(
        u=np.zeros(n), v=np.zeros(n), z=np.zeros(n), conic=np.zeros((n, 3)), cov2d=np.zeros((n, 3)),
        rgb=np.zeros((n, 3)), rgb_clamped=np.zeros((n, 3), np.int32), rgb_raw=np.zeros((n, 3)),
        opacity=np.zeros(n), radius=np.zeros(n, np.int32), radius_exact=np.zeros(n),
        rect=np.zeros((n, 4), np.int32), tiles_touched=np.zeros(n, np.int32),
        u32=np.zeros(n, np.float32), v32=np.zeros(n, np.float32), z32=np.zeros(n, np.float32))
    pr = Projected(n, a)
    cp, cc, cf, co = P.c(), _cam(cam), cfg.c(), pr.c()
    lib().or_project(C.byref(cp), C.byref(cc), C.byref(cf), C.byref(co))
    return pr


def bin_pairs(pr: Projected, cam, cfg: Cfg):
    """Pair list ordered by (tile, depth, Gaussian index): keys, values, ranges."""
    GW, GH = grid(cam, cfg)
    cc, cf, co = _cam(cam), cfg.c(), pr.c()
    total = lib().or_bin(C.byref(co), pr.n, C.byref(cc), C.byref(cf), 0, None, None, None)
    keys = np.zeros(max(total, 1), np.uint64)
    vals = np.zeros(max(total, 1), np.int32)
    ranges = np.zeros((GW * GH, 2), np.int64)
    lib().or_bin(C.byref(co), pr.n, C.byref(cc), C.byref(cf), total, _ptr(keys), _ptr(vals), _ptr(ranges))
    return keys[:total], vals[:total], ranges


def render(pr: Projected, vals, ranges, cam, cfg: Cfg):
    W, H = int(cam["width"]), int(cam["height"])
    out = dict(img=np.zeros((3, H, W)), depth=np.zeros((H, W)), T_final=np.zeros((H, W)),
               n_contrib=np.zeros((H, W), np.int32), last_pos=np.zeros((H, W), np.int64),
               flags=np.zeros((H, W), np.int32))
    vals = np.ascontiguousarray(vals, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    cc, cf, co = _cam(cam), cfg.c(), pr.c()
    lib().or_render(C.byref(co), _ptr(vals), _ptr(ranges), C.byref(cc), C.byref(cf),
                    *[_ptr(out[k]) for k in ("img", "depth", "T_final", "n_contrib", "last_pos", "flags")])
    return out


def loss(img, target, lambda_dssim=0.2, grad=True):
    img = _f64(img)
    target = _f64(target)
    Cc, H, W = img.shape
    dL = np.zeros_like(img) if grad else None
    ssim = np.zeros(1)
    L = lib().or_loss(_ptr(img), _ptr(target), Cc, H, W, float(lambda_dssim), _ptr(dL), _ptr(ssim))
    return L, dL, float(ssim[0])


def ssim_map(x, y):
    x = _f64(x)
    y = _f64(y)
    Cc, H, W = x.shape
    out = np.zeros_like(x)
    lib().or_ssim_map(_ptr(x), _ptr(y), Cc, H, W, _ptr(out))
    return out


def render_backward(pr: Projected, vals, ranges, cam, cfg: Cfg, dL_dimg, img, target, *,
                    dL_ddepth=None, tau_err=0.1, loss_v=0.0, mask_tol=1e-4, stats=None):
    """Returns grad2d (n,10), stats (n,6) (accumulated into `stats` if given) and kappa_amb (n,)."""
    n = pr.n
    grad2d = np.zeros((n, 10))
    if stats is None:
        stats = np.zeros((n, 6))
    kappa_amb = np.zeros(n)
    vals = np.ascontiguousarray(vals, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    dL_dimg = _f64(dL_dimg)
    img = _f64(img)
    target = _f64(target)
    dL_ddepth = None if dL_ddepth is None else _f64(dL_ddepth)
    cc, cf, co = _cam(cam), cfg.c(), pr.c()
    lib().or_render_backward(C.byref(co), n, _ptr(vals), _ptr(ranges), C.byref(cc), C.byref(cf),
                             _ptr(dL_dimg), _ptr(dL_ddepth), _ptr(img), _ptr(target), float(tau_err),
                             float(loss_v), float(mask_tol), _ptr(grad2d), _ptr(stats), _ptr(kappa_amb))
    return grad2d, stats, kappa_amb


def project_backward(params, cam, cfg: Cfg, pr: Projected, grad2d):
    P = params if isinstance(params, Params) else Params(params)
    n, K = P.n, (P.sh_degree + 1) ** 2
    g = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)))
    grad2d = _f64(grad2d, (n, 10))
    cp, cc, cf, co = P.c(), _cam(cam), cfg.c(), pr.c()
    lib().or_project_backward(C.byref(cp), C.byref(cc), C.byref(cf), C.byref(co), _ptr(grad2d),
                              *[_ptr(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")])
    return g


def adam(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """In-place Adam on flat FP64 arrays; lr is per element (broadcast if scalar)."""
    n = p.size
    lr = np.broadcast_to(np.asarray(lr, np.float64), p.shape).reshape(-1).copy()
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_adam(n, _ptr(p), _ptr(g), _ptr(m), _ptr(v), _ptr(lr), beta1, beta2, eps, int(step))


def prune_finalize(omega, kappa, gamma, n_views, tau_d=5.0, tau_p=0.99, densify=None, prune_max=None):
    omega, kappa, gamma = _f64(omega), _f64(kappa), _f64(gamma)
    n = omega.size
    S_d, S_p = np.zeros(n), np.zeros(n)
    densify = np.zeros(n, np.uint8) if densify is None else densify
    prune_max = np.zeros(n) if prune_max is None else prune_max
    prune = np.zeros(n, np.uint8)
    lib().or_prune_finalize(n, _ptr(omega), _ptr(kappa), _ptr(gamma), int(n_views), tau_d, tau_p,
                            _ptr(S_d), _ptr(S_p), _ptr(densify), _ptr(prune_max), _ptr(prune))
    return dict(S_d=S_d, S_p=S_p, densify=densify, prune_max=prune_max, prune=prune)


def geo_loss(depth, prior, grad=True):
    """L_geo = mean over pixels of [prior > 0] |prior - depth| and its gradient."""
    depth, prior = _f64(depth), _f64(prior)
    dL = np.zeros_like(depth) if grad else None
    L = lib().or_geo_loss(_ptr(depth), _ptr(prior), depth.size, _ptr(dL))
    return L, dL


def iso_loss(log_scales, grad=True):
    """L_iso = mean over Gaussians of sum_k |s_k - mean(s)| and dL/dlog-scale."""
    ls = _f64(log_scales)
    n = ls.shape[0]
    g = np.zeros_like(ls) if grad else None
    L = lib().or_iso_loss(n, _ptr(ls), _ptr(g))
    return L, g


def mlp_num_weights():
    return lib().or_mlp_num_weights()


def mlp_forward(x, w, bf16=True):
    """Probabilities (densify, prune) and hidden activations for features x[n][16]."""
    x, w = _f64(x), _f64(w)
    n = x.shape[0]
    p, h1, h2 = np.zeros((n, 2)), np.zeros((n, 64)), np.zeros((n, 64))
    lib().or_mlp_forward(n, _ptr(x), _ptr(w), int(bool(bf16)), _ptr(p), _ptr(h1), _ptr(h2))
    return p, h1, h2


def mlp_bce_grad(x, y, w, bf16=True, rows=False):
    """Mean BCE over rows and outputs, and its gradient with respect to w.
    bf16 rounds the forward's hidden-layer operands only; the backward is
    plain FP64.  rows=True also returns the per-row pre-activation gradients
    (dh2, dh1), each [n][64]."""
    x, y, w = _f64(x), _f64(y), _f64(w)
    g = np.zeros_like(w)
    n = x.shape[0]
    dh2, dh1 = (np.zeros((n, 64)), np.zeros((n, 64))) if rows else (None, None)
    L = lib().or_mlp_bce_grad(n, _ptr(x), _ptr(y), _ptr(w), int(bool(bf16)), _ptr(g),
                              _ptr(dh2) if rows else None, _ptr(dh1) if rows else None)
    return (L, g, dh2, dh1) if rows else (L, g)


def mlp_features(means, log_scales, opacity_logits, stats, ring, head, cam_centre):
    """Predictor inputs feat[n][16] from parameters, stats[n][6] and ring[8][n]."""
    means, log_scales, opl = _f64(means), _f64(log_scales), _f64(opacity_logits)
    stats, ring, cc = _f64(stats), _f64(ring), _f64(cam_centre, (3,))
    n = opl.size
    feat = np.zeros((n, 16))
    lib().or_mlp_features(n, _ptr(means), _ptr(log_scales), _ptr(opl), _ptr(stats), _ptr(ring), int(head),
                          _ptr(cc), _ptr(feat))
    return feat


def densify_prune(P, densify, prune, noise, split_log_scale, split_factor=1.6, m=None, v=None, cap=None):
    """Rows P[n][K_row] after the densify / prune actions; returns (P, m, v, needed)."""
    P = _f64(P)
    n, K = P.shape
    assert K <= 192
    densify = np.ascontiguousarray(densify, np.uint8)
    prune = np.ascontiguousarray(prune, np.uint8)
    noise = _f64(noise, (n, 6)) if n else np.zeros((0, 6))
    m = None if m is None else _f64(m)
    v = None if v is None else _f64(v)
    cap = 2 * n if cap is None else int(cap)
    Po, mo, vo = np.zeros((cap, K)), np.zeros((cap, K)), np.zeros((cap, K))
    need = lib().or_densify_prune(n, K, _ptr(P), _ptr(m) if m is not None else None,
                                  _ptr(v) if v is not None else None, _ptr(densify), _ptr(prune), _ptr(noise),
                                  float(split_log_scale), float(split_factor), cap, _ptr(Po), _ptr(mo), _ptr(vo))
    k = min(need, cap)
    return Po[:k], mo[:k], vo[:k], need


# --------------------------------------------------------------------------
# Probabilistic initialisation (Sec. 3.3.1, Supp. D.5; readings R19-R24)
# --------------------------------------------------------------------------

@dataclass
class InitCfg:
    sigma1: float = 1.0
    sigma2: float = 1.6
    lam: float = 0.9
    scale: float = 255.0
    near_z: float = 0.2
    voxel: tuple = (0.1, 0.25, 1.0, 5.0, 25.0)
    max_dist: tuple = (10.0, 25.0, 100.0, 500.0, float("inf"))


def init_saliency(img, depth, sigma1=1.0, sigma2=1.6, scale=255.0):
    """DoG [H][W] of the channel mean of img [3][H][W] (times scale) and ||grad depth|| [H][W]."""
    img, depth = _f64(img), _f64(depth)
    H, W = depth.shape
    dog, grad = np.zeros((H, W)), np.zeros((H, W))
    lib().or_init_saliency(H, W, _ptr(img), _ptr(depth), float(sigma1), float(sigma2), float(scale), _ptr(dog),
                           _ptr(grad))
    return dog, grad


def init_probability(img, depth, img_r=None, depth_r=None, cfg: InitCfg = InitCfg()):
    """P (or P_kf = max(P - P^, 0) when the rendered pair is given), [H][W]."""
    img, depth = _f64(img), _f64(depth)
    H, W = depth.shape
    img_r = None if img_r is None else _f64(img_r)
    depth_r = None if depth_r is None else _f64(depth_r)
    prob = np.zeros((H, W))
    lib().or_init_probability(H, W, _ptr(img), _ptr(depth), _ptr(img_r), _ptr(depth_r), float(cfg.sigma1),
                              float(cfg.sigma2), float(cfg.scale), float(cfg.lam), _ptr(prob))
    return prob


def init_select(prob, uniform, depth, cam, cfg: InitCfg = InitCfg(), old_keys=None, cap=None, tol=1e-5,
                tol_rel=1e-5):
    """New anchors of a keyframe: dict with keys [k][4] (level, ix, iy, iz), pos [k][3], level, pixel,
    n_new (all new voxels, k = min(n_new, cap)), selected and uncertain [H][W] masks."""
    prob, uniform, depth = _f64(prob), _f64(uniform), _f64(depth)
    H, W = prob.shape
    old = np.zeros((0, 4), np.int64) if old_keys is None else np.ascontiguousarray(old_keys, np.int64)
    cap = H * W if cap is None else int(cap)
    keys, pos = np.zeros((max(cap, 1), 4), np.int64), np.zeros((max(cap, 1), 3))
    level, pixel = np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1), np.int32)
    sel, unc = np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8)
    m = len(cfg.voxel)
    n = lib().or_init_select(H, W, _ptr(prob), _ptr(uniform), _ptr(depth), C.byref(_cam(cam)), float(cfg.near_z),
                             m, _ptr(_f64(cfg.voxel)), _ptr(_f64(cfg.max_dist)), old.shape[0], _ptr(old), cap,
                             _ptr(keys), _ptr(pos), _ptr(level), _ptr(pixel), _ptr(sel), _ptr(unc), float(tol),
                             float(tol_rel))
    k = min(n, cap)
    return dict(keys=keys[:k], pos=pos[:k], level=level[:k], pixel=pixel[:k], n_new=n, selected=sel,
                uncertain=unc)


# --------------------------------------------------------------------------
# Scaffold-GS anchors (Supp. D.1, D.3; readings R25-R29)
# --------------------------------------------------------------------------

ANCHOR_K = 10
ANCHOR_F = 32


def anchor_num_weights():
    return lib().or_anchor_num_weights()


def _anchor_args(A):
    n = len(A["level"])
    return (n, _f64(A["pos"], (n, 3)), np.ascontiguousarray(A["level"], np.int32), _f64(A["feat"], (n, ANCHOR_F)),
            _f64(A["log_l"], (n, 3)), _f64(A["offs"], (n, ANCHOR_K, 3)))


def anchor_decode(A, w, cam_centre, max_dist, tol=1e-6, bf16=False):
    """Decoded Gaussians of anchors A (dict pos, level, feat, log_l, offs): rows [10 n][14], keep and unsure.
    bf16 rounds the decoder's hidden-layer operands to bfloat16 (reading R30)."""
    n, pos, lv, feat, log_l, offs = _anchor_args(A)
    w, cc, md = _f64(w), _f64(cam_centre, (3,)), _f64(max_dist)
    rows = np.zeros((ANCHOR_K * n, 14))
    keep, unsure = np.zeros(ANCHOR_K * n, np.uint8), np.zeros(ANCHOR_K * n, np.uint8)
    lib().or_anchor_decode(n, _ptr(pos), _ptr(lv), _ptr(feat), _ptr(log_l), _ptr(offs), _ptr(w), _ptr(cc), _ptr(md),
                           _ptr(rows), _ptr(keep), _ptr(unsure), float(tol), int(bool(bf16)))
    return rows, keep.astype(bool), unsure.astype(bool)


def anchor_decode_backward(A, w, cam_centre, max_dist, g_rows, bf16=False, rows=False):
    """Gradients (feat, log_l, offs, w) of a loss with dL/drows = g_rows (bf16: of the bfloat16-operand
    forward, plain FP64 chain rule); rows=True also returns each anchor's dL/dz [n][140] and
    dL/dpre [n][64]."""
    n, pos, lv, feat, log_l, offs = _anchor_args(A)
    w, cc, md, g = _f64(w), _f64(cam_centre, (3,)), _f64(max_dist), _f64(g_rows, (ANCHOR_K * n, 14))
    gf, gl, go, gw = np.zeros_like(feat), np.zeros_like(log_l), np.zeros_like(offs), np.zeros_like(w)
    dz, dp = (np.zeros((n, 14 * ANCHOR_K)), np.zeros((n, 64))) if rows else (None, None)
    lib().or_anchor_decode_backward(n, _ptr(pos), _ptr(lv), _ptr(feat), _ptr(log_l), _ptr(offs), _ptr(w), _ptr(cc),
                                    _ptr(md), _ptr(g), _ptr(gf), _ptr(gl), _ptr(go), _ptr(gw), int(bool(bf16)),
                                    _ptr(dz) if rows else None, _ptr(dp) if rows else None)
    return (gf, gl, go, gw, dz, dp) if rows else (gf, gl, go, gw)


def anchor_hidden(A, w, cam_centre, bf16=False):
    """The decoder's unrounded input x [n][36] and hidden pre-activations [n][64] (bf16 as in anchor_decode)."""
    n, pos, lv, feat, log_l, offs = _anchor_args(A)
    w, cc = _f64(w), _f64(cam_centre, (3,))
    x, pre = np.zeros((n, 36)), np.zeros((n, 64))
    lib().or_anchor_hidden(n, _ptr(pos), _ptr(feat), _ptr(w), _ptr(cc), int(bool(bf16)), _ptr(x), _ptr(pre))
    return x, pre


def rows_to_params(rows):
    """Decoded rows [m][14] as SH-degree-0 Gaussian parameters for forward / loss_and_grads."""
    m = rows.shape[0]
    return dict(means=rows[:, 0:3].copy(), log_scales=rows[:, 3:6].copy(), quats=rows[:, 6:10].copy(),
                opacity_logits=rows[:, 10].copy(), sh=rows[:, 11:14].reshape(m, 1, 3).copy(), sh_degree=0)


def grads_to_rows(g):
    """Parameter gradients of loss_and_grads back to the row layout."""
    m = g["opacity_logits"].shape[0]
    return np.concatenate([g["means"], g["log_scales"], g["quats"], g["opacity_logits"].reshape(m, 1),
                           g["sh"].reshape(m, 3)], axis=1)


# --------------------------------------------------------------------------
# Whole-view compositions used by the tests and the CPU baseline
# --------------------------------------------------------------------------

def forward(params, cam, cfg: Cfg):
    P = params if isinstance(params, Params) else Params(params)
    pr = project(P, cam, cfg)
    keys, vals, ranges = bin_pairs(pr, cam, cfg)
    out = render(pr, vals, ranges, cam, cfg)
    out.update(proj=pr, keys=keys, vals=vals, ranges=ranges, params=P)
    return out


def loss_and_grads(params, cam, cfg: Cfg, target, lambda_dssim=0.2, tau_err=0.1, stats=None):
    """One view: forward, loss, backward to every parameter (FP64)."""
    f = forward(params, cam, cfg)
    L, dL, ssim = loss(f["img"], target, lambda_dssim)
    grad2d, stats, kamb = render_backward(f["proj"], f["vals"], f["ranges"], cam, cfg, dL, f["img"], target,
                                          tau_err=tau_err, loss_v=L, stats=stats)
    g = project_backward(f["params"], cam, cfg, f["proj"], grad2d)
    f.update(loss=L, dL_dimg=dL, ssim=ssim, grad2d=grad2d, stats=stats, kappa_amb=kamb, grads=g)
    return f


def morton_order(means):
    """(perm int32 [n], codes uint32 [n]) of FP32 means [n, 3]: the rows in the
    Morton order of the library's spatial reordering, ties in row order."""
    m = np.ascontiguousarray(np.asarray(means, np.float32).reshape(-1, 3))
    n = m.shape[0]
    perm = np.zeros(n, np.int32)
    codes = np.zeros(n, np.uint32)
    lib().or_morton_order(n, _ptr(m), _ptr(codes), _ptr(perm))
    return perm, codes
