"""Scaffold-GS anchors (Sec. 3.2.1; Supp. D.1 decoding, Supp. D.3 LoD mask).

Thin binding of ``gs_anchor_decode``, ``gs_anchor_decode_bwd`` and
``gs_adam_flat`` (``include/gs.h``), the ``AnchorModel`` that owns the anchor
planes, positions, levels and the decoder's weights, and ``AnchorStep``: one
mapping iteration of an anchor map on one view

    decode (view-dependent Gaussians) -> project -> sort -> render -> L_photo
    -> backward to the decoded Gaussians -> backward through the decoder -> Adam

Every step runs in the library's kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import gs

K = 10
FEAT = 32
PLANES = 65          # 0-31 feature, 32-34 log-scale, 35 + 3k + c offset k
WEIGHTS = 11468      # W1[64][36], b1[64], W2[140][64], b2[140]
W1, B1, W2, B2 = 0, 64 * 36, 64 * 36 + 64, 64 * 36 + 64 + 140 * 64
MAX_DIST_DEFAULT = (10.0, 25.0, 100.0, 500.0, math.inf)
VOXEL_DEFAULT = (0.1, 0.25, 1.0, 5.0, 25.0)


class AnchorParams(C.Structure):
    _fields_ = [("data", C.c_void_p), ("pos", C.c_void_p), ("level", C.c_void_p), ("n", C.c_int64),
                ("ld", C.c_int64)]


_typed = False


def _lib():
    global _typed
    L = gs.lib()
    if not _typed:
        vp, i32, i64, f32, P = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.POINTER
        L.gs_anchor_decode.argtypes = [P(AnchorParams), vp, P(f32 * 3), vp, i32, P(gs.Params), vp, i64, vp]
        L.gs_anchor_decode_bwd.argtypes = [P(AnchorParams), vp, P(f32 * 3), vp, i32, P(gs.Params), vp, vp, vp, i64,
                                           vp]
        L.gs_adam_flat.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i64, vp, vp]
        _typed = True
    return L


def init_weights(seed=0, device="cuda", opacity_bias=0.5):
    """Decoder weights: W1 ~ N(0, 2/36), W2 ~ N(0, 0.01/64), b1 = 0; output
    biases give every Gaussian opacity tanh(0.5) and colour 1/2 at start."""
    g = np.random.default_rng(seed)
    w = np.zeros(WEIGHTS, np.float32)
    w[W1:B1] = g.normal(0.0, math.sqrt(2.0 / 36.0), B1 - W1)
    w[W2:B2] = g.normal(0.0, 0.1 / 8.0, B2 - W2)
    w[B2 + 3::14] = opacity_bias
    return torch.from_numpy(w).to(device)


class AnchorModel:
    """n anchors: planes [65][ld] (feature, log-scale, offsets), fixed
    positions [3][ld] and levels [ld], and the decoder's weights."""

    def __init__(self, n, device="cuda", weights=None, seed=0):
        self.n = int(n)
        self.ld = max(4, gs.padded(self.n))
        self.data = torch.zeros(PLANES, self.ld, dtype=torch.float32, device=device)
        self.pos = torch.zeros(3, self.ld, dtype=torch.float32, device=device)
        self.level = torch.zeros(self.ld, dtype=torch.int32, device=device)
        self.weights = init_weights(seed, device) if weights is None else weights

    @classmethod
    def from_arrays(cls, pos, level, feat, log_l, offs, weights, device="cuda"):
        """Array-of-structures inputs: pos [n][3], level [n], feat [n][32], log_l [n][3], offs [n][10][3]."""
        n = len(level)
        m = cls(n, device, weights=torch.as_tensor(np.asarray(weights, np.float32)).to(device))
        m.pos[:, :n] = torch.from_numpy(np.asarray(pos, np.float32).T.copy())
        m.level[:n] = torch.from_numpy(np.asarray(level, np.int32))
        planes = np.concatenate([np.asarray(feat, np.float32).reshape(n, FEAT), np.asarray(log_l, np.float32),
                                 np.asarray(offs, np.float32).reshape(n, 3 * K)], axis=1).T
        m.data[:, :n] = torch.from_numpy(planes.copy())
        return m

    @classmethod
    def from_anchor_map(cls, amap, voxel=VOXEL_DEFAULT, seed=0, device="cuda"):
        """Anchors of gs_init_insert: zero features (Supp. D.5), base scale = the
        voxel size of the anchor's level, zero offsets."""
        n = min(amap.n, amap.capacity)
        m = cls(n, device, seed=seed)
        m.pos[:, :n] = amap.pos[:, :n]
        m.level[:n] = amap.level[:n]
        eps = torch.log(torch.tensor(voxel, dtype=torch.float32, device=device))
        m.data[FEAT:FEAT + 3, :n] = eps[amap.level[:n].long()].unsqueeze(0)
        return m

    def c(self) -> AnchorParams:
        return AnchorParams(self.data.data_ptr(), self.pos.data_ptr(), self.level.data_ptr(), self.n, self.ld)

    def decoded(self) -> gs.GaussianModel:
        """An SH-degree-0 Gaussian buffer for the K ld decoded slots."""
        return gs.GaussianModel(K * self.ld, 0, device=self.data.device, ld=K * self.ld)


def _bands(max_dist):
    md = (C.c_float * len(max_dist))(*[min(float(x), 3.0e38) for x in max_dist])
    return md, len(max_dist)


def gs_anchor_decode(model: AnchorModel, cam_centre, out: gs.GaussianModel, max_dist=MAX_DIST_DEFAULT, stream=None,
                     status=None, max_polls=-1):
    md, lv = _bands(max_dist)
    cc = (C.c_float * 3)(*[float(x) for x in cam_centre])
    gs._check(_lib().gs_anchor_decode(C.byref(model.c()), gs._ptr(model.weights), C.byref(cc), md, lv,
                                      C.byref(out.c()), gs._ptr(status), int(max_polls), gs._stream(stream)),
              "gs_anchor_decode")


def gs_anchor_decode_bwd(model: AnchorModel, cam_centre, grad_out: gs.GaussianModel, grad_anchor, grad_weights,
                         max_dist=MAX_DIST_DEFAULT, stream=None, status=None, max_polls=-1):
    md, lv = _bands(max_dist)
    cc = (C.c_float * 3)(*[float(x) for x in cam_centre])
    gs._check(_lib().gs_anchor_decode_bwd(C.byref(model.c()), gs._ptr(model.weights), C.byref(cc), md, lv,
                                          C.byref(grad_out.c()), gs._ptr(grad_anchor), gs._ptr(grad_weights),
                                          gs._ptr(status), int(max_polls), gs._stream(stream)),
              "gs_anchor_decode_bwd")


def gs_adam_flat(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None, step_device=None):
    gs._check(_lib().gs_adam_flat(gs._ptr(p), gs._ptr(g), gs._ptr(m), gs._ptr(v), p.numel(), float(lr),
                                  float(beta1), float(beta2), float(eps), int(step), gs._ptr(step_device),
                                  gs._stream(stream)),
              "gs_adam_flat")


def camera_centre(cam):
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    return -(R.T @ np.asarray(cam["t"], np.float64).reshape(3))


# learning rates of the anchor groups and the decoder (the paper is silent: Scaffold-GS's values)
LR_DEFAULT = dict(feat=7.5e-3, log_l=7e-3, offs=1e-2, weights=4e-3)


class AnchorStep:
    """One view per iteration: decode, render, L_photo, backward, decoder
    backward, Adam on the anchors and the decoder."""

    def __init__(self, model: AnchorModel, cam, cfg: gs.Config = None, lambda_dssim=0.2, lr=None,
                 max_dist=MAX_DIST_DEFAULT):
        self.model, self.cam, self.max_dist = model, cam, tuple(max_dist)
        self.lr = dict(LR_DEFAULT, **(lr or {}))
        self.gauss = model.decoded()
        gs_anchor_decode(model, camera_centre(cam), self.gauss, self.max_dist)
        self.map = gs.MappingStep(self.gauss, [cam], cfg, lambda_dssim=lambda_dssim, with_stats=False)
        self.g_anchor = torch.zeros_like(model.data)
        self.g_w = torch.zeros_like(model.weights)
        self.m_a, self.v_a = torch.zeros_like(model.data), torch.zeros_like(model.data)
        self.m_w, self.v_w = torch.zeros_like(model.weights), torch.zeros_like(model.weights)
        self.step_count = 0

    def fit_capacity(self, slack=1.25):
        return self.map.fit_capacity(slack)

    def set_camera(self, cam):
        self.cam = cam
        self.map.set_cameras([cam])

    def gradients(self, target, stream=None):
        """Decode, forward, loss and every gradient (anchors, decoder) without an update."""
        cc = camera_centre(self.cam)
        status = self.map.buf.status
        gs_anchor_decode(self.model, cc, self.gauss, self.max_dist, stream, status=status)
        loss = self.map.step(target, stream, optimize=False)
        gs_anchor_decode_bwd(self.model, cc, self.map.grads, self.g_anchor, self.g_w, self.max_dist, stream,
                             status=status)
        return loss

    def _adam(self, t, stream=None, step_device=None):
        A, G, M, V = self.model.data, self.g_anchor, self.m_a, self.v_a
        for name, lo, hi in (("feat", 0, FEAT), ("log_l", FEAT, FEAT + 3), ("offs", FEAT + 3, PLANES)):
            gs_adam_flat(A[lo:hi], G[lo:hi], M[lo:hi], V[lo:hi], self.lr[name], t, stream=stream,
                         step_device=step_device)
        gs_adam_flat(self.model.weights, self.g_w, self.m_w, self.v_w, self.lr["weights"], t, stream=stream,
                     step_device=step_device)

    def step(self, target, stream=None):
        loss = self.gradients(target, stream)
        self.step_count += 1
        self._adam(self.step_count, stream)
        return loss

    STAGES = ("decode", "render_fwd", "loss_bwd", "decode_bwd", "adam")

    def capture(self, target, events=None):
        """One whole iteration for the current camera (its centre is a decoder argument, so a
        graph per camera) in a CUDA graph: decode, project / sort / render, losses and
        backward, decoder backward, Adam with a device step counter that the graph advances.
        events: optional timing events (external=True), one more than STAGES."""
        dev = self.model.data.device
        if getattr(self, "step_dev", None) is None:
            self.step_dev = torch.full((1,), self.step_count, dtype=torch.int64, device=dev)
        assert events is None or len(events) == len(self.STAGES) + 1
        cc = camera_centre(self.cam)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        graph = torch.cuda.CUDAGraph()

        def mark(i):
            if events is not None:
                events[i].record(side)

        with torch.cuda.graph(graph, stream=side):
            b = self.map.buf
            b.status.zero_()
            self.step_dev.add_(1)
            mark(0)
            gs_anchor_decode(self.model, cc, self.gauss, self.max_dist, status=b.status)
            mark(1)
            gs.gs_project(self.gauss, b)
            gs.gs_sort(b)
            gs.gs_render_fwd(b)
            mark(2)
            self.map._losses_and_backward(target)
            mark(3)
            gs_anchor_decode_bwd(self.model, cc, self.map.grads, self.g_anchor, self.g_w, self.max_dist,
                                 status=b.status)
            mark(4)
            self._adam(1, step_device=self.step_dev)
            mark(5)
        torch.cuda.current_stream(dev).wait_stream(side)
        return graph

    def replay(self, graph):
        graph.replay()
        self.step_count += 1
        return self.map.buf.loss
