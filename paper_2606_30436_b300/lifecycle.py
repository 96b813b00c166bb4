"""Gaussian lifecycle over keyframe chunks (Sec. 3.3.2; scores of Supp. E.1,
E.2).  The mapping iterations of a chunk accumulate the per-Gaussian
statistics (|Omega|, kappa, gamma, max T*alpha, ||dL/d(u,v)||, views seen) in
the backward pass; at the end of the chunk one of two deciders turns them into
densify / prune bits, and ``gs_densify_prune`` applies the bits to the
parameters and the Adam moments:

* ``plain``: the paper's criterion, ``gs_prune_stats`` (S_d > tau_d,
  min-max-normalised S_p > tau_p over the active Gaussians);
* ``learned``: the BF16 tensor-core predictor (``gs_mlp_features`` +
  ``gs_mlp_forward``), trained on labels the plain criterion produces
  (``future_labels``: a Gaussian is labelled for pruning when the plain
  criterion prunes it in this chunk or any later one, so the predictor acts
  before the plain criterion would); where its probability lies within
  ``margin`` of 1/2 the plain bit of the same chunk is used instead (the
  fallback), and the plain criterion stays the reference for its error
  (``agreement``).  Both deciders act only on Gaussians the chunk saw.

Readings: the statistics of a chunk are summed over its iterations and views,
so |V_c| = iterations x views; decisions are taken and applied per chunk (the
OR / max aggregation over chunks of Sec. 3.3.2 would need the bits of
Gaussians that no longer exist after the actions); the blend-weight ring takes
one slot per iteration (each slot the maximum over that iteration's views).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import gs


class Predictor:
    """Weights, Adam state and the training loop of the learned decider."""

    def __init__(self, seed=0, device="cuda", lr=3e-3):
        self.w = gs.mlp_init(seed, device=device)
        self.m, self.v = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.grad = torch.zeros_like(self.w)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.lr, self.step = lr, 0

    def train(self, batches, epochs=200):
        """Full-batch Adam over (feat [16, ld], n, y_densify, y_prune) tuples; returns the last mean BCE."""
        losses = []
        for _ in range(epochs):
            for feat, n, yd, yp in batches:
                gs.gs_mlp_train_grad(feat, yd, yp, n, self.w, self.grad, self.loss, self.status)
                self.step += 1
                gs.gs_mlp_adam(self.w, self.grad, self.m, self.v, self.lr, self.step)
                losses.append(self.loss)
        if self.status.item():
            raise gs.GSError("predictor status %d" % self.status.item())
        return float(losses[-1].item()) if losses else float("nan")

    def predict(self, feat, n, densify, prune, prob=None):
        gs.gs_mlp_forward(feat, n, self.w, prob, densify, prune, self.status)


class Lifecycle:
    """Statistics, decisions and actions of one chunk at a time."""

    def __init__(self, mode="plain", tau_d=5.0, tau_p=0.99, split_log_scale=-2.5, split_factor=1.6,
                 predictor: Predictor = None, collect=False, seed=0, margin=0.1, n_initial=None, reorder=True):
        assert mode in ("plain", "learned")
        assert mode == "plain" or predictor is not None
        self.mode, self.tau_d, self.tau_p = mode, tau_d, tau_p
        self.split_log_scale, self.split_factor = split_log_scale, split_factor
        self.predictor, self.collect = predictor, collect
        self.margin = margin  # learned: the plain bit where |p - 1/2| < margin
        # after the actions, put the new map's rows in the Morton order of the means, so that
        # the next chunk's views read contiguous rows (ids follow the rows)
        self.reorder = reorder
        # identity of every Gaussian of the current map (host), carried through the actions; numbered
        # 0 .. n - 1 at the first chunk unless n_initial says otherwise
        self.ids = None if n_initial is None else np.arange(n_initial, dtype=np.int64)
        self.next_id = 0 if n_initial is None else n_initial
        self.samples = []   # per chunk, with collect=True: (feat, n, densify, prune, active, ids)
        self.history = []   # per chunk: n before / after, bits set, agreement with the plain criterion
        self.gen = torch.Generator(device="cuda").manual_seed(int(seed))
        self.ring = None
        self.head = gs.MLP_RING - 1
        self._buffers = {}
        self.iterations = 0

    def start(self, step: gs.MappingStep):
        """Zeroes the accumulators before the chunk's first iteration."""
        assert step.buf.stats_acc is not None, "the mapping step must accumulate statistics"
        step.buf.stats_acc.zero_()
        if self.ids is None:
            self.ids, self.next_id = np.arange(step.model.n, dtype=np.int64), step.model.n
        assert len(self.ids) == step.model.n, "the map changed outside the lifecycle's actions"
        ld = step.model.ld
        if self.ring is None or self.ring.shape[1] != ld:
            self.ring = torch.zeros(gs.MLP_RING, ld, dtype=torch.float32, device=step.model.data.device)
        else:
            self.ring.zero_()
        self.head = gs.MLP_RING - 1
        self.iterations = 0
        # the decisions' buffers at this chunk's size, so that deciding allocates nothing
        dev, f32, u8 = step.model.data.device, torch.float32, torch.uint8
        n = step.model.n
        for k, t in (("S_d", f32), ("S_p", f32), ("prune_max", f32), ("densify", u8), ("prune", u8)):
            self._buffer(k, n, t, dev)
        size = C.c_size_t()
        gs._check(gs.lib().gs_prune_workspace_size(n, C.byref(size)), "gs_prune_workspace_size")
        self._buffer("prune_ws", max(int(size.value), 256), u8, dev)
        if self.mode == "learned" or self.collect:
            self._buffer("feat", gs.MLP_INPUTS * ld, f32, dev)
            self._buffer("prob", 2 * ld, f32, dev)

    def after_iteration(self, step: gs.MappingStep):
        """Moves this iteration's max T*alpha into the ring."""
        self.head = (self.head + 1) % gs.MLP_RING
        gs.gs_mlp_push_blend(step.buf.stats_acc, step.model.n, self.ring, self.head)
        self.iterations += 1

    def _features(self, step, cam_centre):
        model = step.model
        feat = self._buffer("feat", gs.MLP_INPUTS * model.ld, torch.float32, model.data.device)
        feat = feat.view(gs.MLP_INPUTS, model.ld)
        gs.gs_mlp_features(model, step.buf.stats_acc, self.ring, self.head, cam_centre, feat)
        return feat

    def _buffer(self, name, numel, dtype, device):
        """A reused device buffer of at least numel elements (the first numel returned),
        grown by start() to the chunk's size so that the decisions allocate nothing."""
        buf = self._buffers.get(name)
        if buf is None or buf.numel() < numel or buf.device != device:
            self._buffers[name] = buf = None  # the old one is released first
            buf = torch.empty(numel, dtype=dtype, device=device)
            self._buffers[name] = buf
        return buf[:numel]

    def plain_bits(self, step: gs.MappingStep):
        """The plain criterion's bits (Supp. E.1, E.2) from the chunk's accumulators."""
        n, dev = step.model.n, step.model.data.device
        n_views = max(1, self.iterations * step.buf.n_views)
        f32, u8 = torch.float32, torch.uint8
        scores = {k: self._buffer(k, n, t, dev) for k, t in (("S_d", f32), ("S_p", f32), ("prune_max", f32),
                                                                ("densify", u8), ("prune", u8))}
        scores["prune_max"].zero_()  # running over the chunks of one decision: this chunk alone
        scores["densify"].zero_()
        size = C.c_size_t()
        gs._check(gs.lib().gs_prune_workspace_size(n, C.byref(size)), "gs_prune_workspace_size")
        ws = self._buffer("prune_ws", max(int(size.value), 256), u8, dev)
        gs.gs_prune_stats(step.buf.stats_acc, n, n_views, scores, ws, self.tau_d, self.tau_p)
        return scores["densify"], scores["prune"]

    def active(self, step: gs.MappingStep):
        """[n] bool: the Gaussians blended somewhere in this chunk (|Omega| > 0)."""
        return step.buf.stats_acc[0, :step.model.n] > 0

    def decide(self, step: gs.MappingStep, cam_centre):
        """Densify / prune bits ([n] uint8) of the chunk's Gaussians, by the
        chosen decider; nothing here synchronises the host."""
        model, dev = step.model, step.model.data.device
        n = model.n
        self._last = None
        self._fallback = None
        if self.mode == "plain":
            dens, prune = self.plain_bits(step)
            if self.collect:
                self.samples.append((self._features(step, cam_centre).clone(), n, dens.clone(), prune.clone(),
                                     self.active(step).clone(), self.ids.copy()))
        else:
            feat = self._features(step, cam_centre)
            prob = self._buffer("prob", 2 * model.ld, torch.float32, dev).view(2, model.ld)
            self.predictor.predict(feat, n, None, None, prob)
            pd, pp = self.plain_bits(step)
            act = self.active(step)
            unsure_d = (prob[0, :n] - 0.5).abs() < self.margin
            unsure_p = (prob[1, :n] - 0.5).abs() < self.margin
            dens = (torch.where(unsure_d, pd.bool(), prob[0, :n] > 0.5) & act).to(torch.uint8)
            prune = (torch.where(unsure_p, pp.bool(), prob[1, :n] > 0.5) & act).to(torch.uint8)
            self._fallback = (unsure_d & act, unsure_p & act, act)
        self._last = (n, dens, prune)
        return dens, prune

    def assess(self, step: gs.MappingStep):
        """Records the chunk's bit counts and, for the learned decider, its
        agreement with the plain criterion on the same accumulators (call after
        decide, before apply)."""
        n, dens, prune = self._last
        rec = dict(n=n, densify=int(dens.sum().item()), prune=int(prune.sum().item()))
        if self.mode == "learned":
            rec.update(agreement(dens, prune, *self.plain_bits(step)))
            ud, up, act = self._fallback
            na = max(1, int(act.sum().item()))
            rec.update(fallback_densify_rate=round(int(ud.sum().item()) / na, 4),
                       fallback_prune_rate=round(int(up.sum().item()) / na, 4), active=na)
        self.history.append(rec)
        return rec

    def apply(self, step: gs.MappingStep, dens, prune):
        """New parameters and moments after the actions."""
        model = step.model
        noise = torch.randn(6, model.ld, generator=self.gen, device=model.data.device)
        out, m, v, _ = gs.gs_densify_prune(model, dens, prune, noise, self.split_log_scale, self.split_factor,
                                           exp_avg=step.exp_avg, exp_avg_sq=step.exp_avg_sq,
                                           capacity=gs.padded(model.n + int(dens.sum().item())))
        if self.history:
            self.history[-1]["n_after"] = out.n
        self.ids, self.next_id = carry_ids(self.ids, dens.cpu().numpy(), prune.cpu().numpy(), self.next_id)
        assert len(self.ids) == out.n
        if self.reorder and out.n > 0:
            perm = gs.gs_reorder(out, [m.data, v.data])
            self.ids = self.ids[perm.cpu().numpy()]
        return out, (m, v)


def agreement(dens, prune, ref_d, ref_p):
    """Precision / recall of the learned bits against the plain criterion's."""
    out = {}
    for name, a, b in (("densify", dens, ref_d), ("prune", prune, ref_p)):
        a, b = a.bool(), b.bool()
        tp = int((a & b).sum().item())
        pa, pb = int(a.sum().item()), int(b.sum().item())
        out[name + "_precision"] = tp / pa if pa else 1.0
        out[name + "_recall"] = tp / pb if pb else 1.0
        out[name + "_accuracy"] = float((a == b).float().mean().item()) if a.numel() else 1.0
    return out


def carry_ids(ids, dens, prune, next_id):
    """Identities after gs_densify_prune's rows (source order; a pruned
    Gaussian emits none, a kept one its own row, a densified one its own row
    followed by a new one): the first row keeps the source's id, a second row
    takes the next fresh id.  Returns (ids, next_id)."""
    keep = np.asarray(prune) == 0
    rows = 1 + ((np.asarray(dens) != 0) & keep)[keep].astype(np.int64)
    src = np.repeat(np.arange(int(keep.sum())), rows)
    out = np.repeat(np.asarray(ids, np.int64)[keep], rows)
    second = np.zeros(len(src), bool)
    second[1:] = src[1:] == src[:-1]
    out[second] = next_id + np.arange(int(second.sum()))
    return out, next_id + int(second.sum())


def future_labels(samples, device="cuda"):
    """Training rows from the plain criterion's chunks (Lifecycle(collect=True)
    samples, in chunk order): the densify label is the chunk's own plain bit,
    the prune label is set when the plain criterion prunes the Gaussian in
    that chunk or in any later chunk of the run; only Gaussians the chunk saw
    can carry a label.  Returns (feat, n, y_densify, y_prune) tuples."""
    pruned_later = set()
    rows = []
    for feat, n, dens, prune, act, ids in reversed(samples):
        pr = prune.cpu().numpy().astype(bool)
        pruned_later.update(ids[pr].tolist())
        later = np.isin(ids, np.fromiter(pruned_later, dtype=np.int64, count=len(pruned_later)))
        a = act.cpu().numpy()
        yp = torch.from_numpy((later & a).astype(np.uint8)).to(device)
        yd = (dens.to(torch.bool) & act).to(torch.uint8)
        rows.append((feat, n, yd, yp))
    return rows[::-1]
