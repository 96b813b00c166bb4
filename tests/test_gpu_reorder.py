"""GPU spatial reordering (gs_reorder) against the oracle's Morton order:
the permutation bit for bit (ragged sizes over several radix rounds, ties,
degenerate boxes, the 1M-Gaussian corridor), every plane set moved with it
bit for bit and the padding rows untouched; and a mapping step that gives
the same loss and image, and its gradients permuted, after the reorder,
including through a graph captured before it."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2606_30436_b300 import gs, scenes

from _parity import rel_l2

pytestmark = pytest.mark.gpu


def _model(scene):
    return gs.GaussianModel.from_scene(scene, device="cuda")


def _extras(model, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return [torch.randn(model.K, model.ld, generator=g, device="cuda"),
            torch.rand(model.K, model.ld, generator=g, device="cuda"),
            torch.randn(6, model.ld, generator=g, device="cuda")]


def _check(model, extras, before, perm):
    """perm equals the oracle's order of the means before; every set moved by it, padding kept."""
    n = model.n
    want, _ = orc.morton_order(before[0][0:3, :n].T)
    got = perm.cpu().numpy()
    assert np.array_equal(got, want)
    for new, old in zip([model.data] + extras, before):
        new = new.cpu().numpy()
        assert np.array_equal(new[:, :n], old[:, :n][:, want])
        assert np.array_equal(new[:, n:], old[:, n:])


@pytest.mark.parametrize("n,D", [(100_003, 3), (4097, 0), (1, 1), (70_000, 2)])
def test_reorder_matches_oracle(n, D):
    scene = scenes.corridor_scene(n, seed=n % 97, sh_degree=D)
    model = _model(scene)
    extras = _extras(model, 1)
    before = [t.cpu().numpy().copy() for t in [model.data] + extras]
    perm = gs.gs_reorder(model, extras)
    torch.cuda.synchronize()
    _check(model, extras, before, perm)


def test_reorder_ties_and_degenerate_boxes():
    # many rows on a few lattice points: the stable order among equal codes
    rng = np.random.default_rng(11)
    scene = scenes.uniform_scene(50_000, seed=3, sh_degree=0)
    pts = rng.integers(0, 5, (50_000, 3)).astype(np.float32)
    scene["means"] = pts
    model = _model(scene)
    extras = _extras(model, 2)
    before = [t.cpu().numpy().copy() for t in [model.data] + extras]
    _check(model, extras, before, gs.gs_reorder(model, extras))
    # every mean equal: zero extent, the identity
    scene["means"] = np.full((50_000, 3), 1.5, np.float32)
    model = _model(scene)
    perm = gs.gs_reorder(model)
    assert np.array_equal(perm.cpu().numpy(), np.arange(50_000))
    # no rows: nothing launched, nothing changed
    empty = gs.GaussianModel(0, 1, device="cuda")
    assert gs.gs_reorder(empty).numel() == 0


def test_reorder_fullsize_corridor():
    scene = scenes.corridor_scene(1_000_000, seed=0, sh_degree=3)
    model = _model(scene)
    means = model.data[0:3, :model.n].T.cpu().numpy().copy()
    perm = gs.gs_reorder(model).cpu().numpy()
    want, _ = orc.morton_order(means)
    assert np.array_equal(perm, want)
    assert np.array_equal(model.data[0:3, :model.n].T.cpu().numpy(), means[want])


def test_mapping_step_invariant_under_reorder():
    # Gaussians of equal depth blend in row order, which the reorder changes: give every
    # Gaussian its own depth (distinct z far apart, a camera looking straight down z), so
    # that the compositing order, and with it the image, is the same in both row orders
    n, length = 60_000, 200.0
    scene = scenes.corridor_scene(n, seed=4, sh_degree=3, length=length)
    scene["means"][:, 2] = (np.random.default_rng(6).permutation(n) * (length / n)).astype(np.float32)
    tscene = scenes.perturb(scene, 0.01, seed=5)
    cam = scenes.corridor_camera(40, 320, 240, 260.0)
    cfg = gs.Config()
    ts = gs.MappingStep(_model(tscene), [cam], cfg, with_stats=False)
    ts.fit_capacity()
    target = ts.buf.img.clone()

    st = gs.MappingStep(_model(scene), [cam], cfg, lambda_dssim=0.2)
    st.fit_capacity()
    st.buf.stats_acc.zero_()
    st.step(target, optimize=False)
    torch.cuda.synchronize()
    loss0, img0 = st.buf.loss.clone(), st.buf.img.clone()
    g0 = st.grads.data[:, :st.model.n].clone()
    stats0 = st.buf.stats_acc[:, :st.model.n].clone()
    graph = st.capture(target)  # captured before the reorder: the buffers keep their addresses

    perm = st.reorder().long()
    assert torch.equal(st.buf.stats_acc[:, :st.model.n], stats0[:, perm])
    st.buf.stats_acc.zero_()
    st.step(target, optimize=False)
    torch.cuda.synchronize()
    st.check_status()
    assert abs(st.buf.loss.item() - loss0.item()) <= 1e-6 * abs(loss0.item())
    assert torch.equal(st.buf.img, img0)
    g1 = st.grads.data[:, :st.model.n]
    assert rel_l2(g1.cpu().numpy(), g0[:, perm].cpu().numpy()) < 1e-5

    # the graph from before the reorder runs the reordered map (one optimisation step)
    m_ref = st.model.data.clone()
    st.replay(graph)
    torch.cuda.synchronize()
    st.check_status()
    assert abs(st.buf.loss.item() - loss0.item()) <= 1e-6 * abs(loss0.item())
    assert not torch.equal(st.model.data, m_ref)  # Adam moved the reordered parameters
