"""The projection backward that writes only the gradient rows of the Gaussians
some view sees (gs_project_bwd_rows) and the Adam step that reads the other
rows as zero (gs_adam_rows), against the plain pair (every row written, gs_adam).
On one compositing backward: the marks equal "some view has a radius", the
written rows equal the plain gradient bit for bit, the others keep their old
contents, and the updated parameters and moments are bit-identical (SH degrees
0 and 3, one and two views, host and device step counters).  Over several
optimising steps, eager and graph-replayed, the two agree as two runs of the
plain sequence do (the compositing backward sums with atomics)."""
import numpy as np
import pytest
import torch

from paper_2606_30436_b300 import gs, scenes

from _parity import rel_l2

pytestmark = pytest.mark.gpu


def _case(multi, D, n=10000):
    if multi:
        s = scenes.uniform_scene(3000, seed=7, sh_degree=D, xy_range=3.0)
        cams = [scenes.pinhole(100, 70, 90.0),
                scenes.pinhole(150, 90, 140.0, R=scenes.yaw_matrix(4.0), t=np.array([0.2, -0.1, 0.3], np.float32))]
    else:
        # a wide spread, so that many Gaussians fall outside the view
        s = scenes.uniform_scene(n, seed=D, sh_degree=D, xy_range=12.0)
        cams = [scenes.pinhole(320, 240, 300.0)]
    return s, cams


def _target(scene, cams):
    tm = gs.GaussianModel.from_scene(scenes.perturb(scene, 0.02, seed=9))
    st = gs.MappingStep(tm, cams, gs.Config(), with_stats=False)
    st.fit_capacity()
    return st.buf.img.clone()


@pytest.mark.parametrize("multi,D,device_step", [(False, 3, False), (True, 3, True), (False, 0, True),
                                                 (True, 0, False)])
def test_rows_bit_identical_on_one_backward(multi, D, device_step):
    scene, cams = _case(multi, D)
    target = _target(scene, cams)
    st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, gs.Config(), with_stats=False)
    st.fit_capacity(slack=2.0)
    st.forward()
    gs.gs_loss(st.buf, target, 0.2)
    gs.gs_render_bwd(st.model, None, st.buf, target, with_stats=False)
    full, part = st.model.like(), st.model.like()
    part.data.fill_(7.0)
    rows = torch.full((st.model.ld,), 9, dtype=torch.uint8, device="cuda")
    gs.gs_project_bwd(st.model, full, st.buf, with_stats=False)
    gs.gs_project_bwd(st.model, part, st.buf, with_stats=False, rows=rows)
    torch.cuda.synchronize()
    rad = st.buf.radius.view(st.buf.n_views, st.model.ld)
    seen = (rad > 0).any(dim=0)
    seen[st.model.n:] = False
    assert torch.equal(rows.bool(), seen) and int(rows.max()) <= 1
    assert 0 < int(seen.sum()) < st.model.n  # some rows of each kind
    assert torch.equal(part.data[:, seen], full.data[:, seen])
    assert bool((part.data[:, ~seen] == 7.0).all())
    assert not full.data[:, ~seen].any()

    g = torch.Generator(device="cuda").manual_seed(3)
    m0 = torch.randn(st.model.data.shape, generator=g, device="cuda") * 1e-3
    v0 = torch.rand(st.model.data.shape, generator=g, device="cuda") * 1e-6
    runs = []
    for use_rows in (False, True):
        p, m, v = st.model.like(), st.model.like(), st.model.like()
        p.data.copy_(st.model.data)
        m.data.copy_(m0)
        v.data.copy_(v0)
        step_dev = torch.full((1,), 4, dtype=torch.int64, device="cuda") if device_step else None
        if use_rows:
            gs.gs_adam(p, part, m, v, st.lr, 4, step_device=step_dev, rows=rows)
        else:
            gs.gs_adam(p, full, m, v, st.lr, 4, step_device=step_dev)
        runs.append((p.data, m.data, v.data))
    torch.cuda.synchronize()
    for a, b in zip(*runs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("multi", [False, True])
def test_adam_parts_equal_adam_rows(multi):
    """Part 2 (the Gaussians no view sees, from the radii alone) and part 1 (the marked rows)
    write disjoint elements and together give gs_adam_rows bit for bit."""
    scene, cams = _case(multi, 3)
    target = _target(scene, cams)
    st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, gs.Config(), with_stats=False)
    st.fit_capacity(slack=2.0)
    st.forward()
    gs.gs_loss(st.buf, target, 0.2)
    gs.gs_render_bwd(st.model, None, st.buf, target, with_stats=False)
    grads = st.model.like()
    rows = torch.zeros(st.model.ld, dtype=torch.uint8, device="cuda")
    gs.gs_project_bwd(st.model, grads, st.buf, with_stats=False, rows=rows)
    g = torch.Generator(device="cuda").manual_seed(5)
    m0 = torch.randn(st.model.data.shape, generator=g, device="cuda") * 1e-3
    v0 = torch.rand(st.model.data.shape, generator=g, device="cuda") * 1e-6
    step_dev = torch.full((1,), 3, dtype=torch.int64, device="cuda")
    out = []
    for split in (False, True):
        p, m, v = st.model.like(), st.model.like(), st.model.like()
        p.data.copy_(st.model.data)
        m.data.copy_(m0)
        v.data.copy_(v0)
        if split:
            gs.gs_adam_part(p, None, m, v, st.buf, 2, st.lr, 3, step_device=step_dev)
            p2 = p.data.clone()
            seen = rows.bool()
            assert torch.equal(p2[:, seen], st.model.data[:, seen])  # part 2 left the seen rows alone
            gs.gs_adam_part(p, grads, m, v, st.buf, 1, st.lr, 3, rows=rows, step_device=step_dev)
            assert torch.equal(p.data[:, ~seen], p2[:, ~seen])        # part 1 left the unseen rows alone
        else:
            gs.gs_adam(p, grads, m, v, st.lr, 3, step_device=step_dev, rows=rows)
        out.append((p.data, m.data, v.data))
    torch.cuda.synchronize()
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_overlapped_graph_matches_serial_graph():
    """The captured step with the unseen Gaussians' Adam on a second stream against the same
    step captured on one stream (the tolerances of two runs, atomics in the backward)."""
    scene, cams = _case(False, 3)
    target = _target(scene, cams)
    p0 = gs.GaussianModel.from_scene(scene).data
    runs = []
    for overlap in (True, False):
        st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, gs.Config(adam_overlap=overlap),
                            lr=gs.default_lr(extent=5.0))
        st.fit_capacity(slack=2.0)
        g = st.capture(target)
        for _ in range(3):
            st.replay(g)
        torch.cuda.synchronize()
        st.check_status()
        runs.append(st)
    a, b = runs
    n = a.model.n
    assert rel_l2(a.exp_avg.data[:, :n].cpu().numpy(), b.exp_avg.data[:, :n].cpu().numpy()) < 1e-4
    da = (a.model.data - p0)[:, :n].cpu().numpy()
    db = (b.model.data - p0)[:, :n].cpu().numpy()
    close = np.abs(da - db) <= 1e-6 + 1e-4 * np.abs(db)
    assert close.mean() > 0.999, close.mean()
    assert torch.equal(a.model.data[:, n:], p0[:, n:])


def _run(scene, cams, target, rows, iters, graph, lambda_iso=0.0):
    st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, gs.Config(grad_rows=rows),
                        lr=gs.default_lr(extent=5.0), lambda_iso=lambda_iso)
    st.fit_capacity(slack=2.0)
    if graph:
        g = st.capture(target)
        for _ in range(iters):
            st.replay(g)
    else:
        for _ in range(iters):
            st.step(target)
    torch.cuda.synchronize()
    st.check_status()
    return st


@pytest.mark.parametrize("multi,graph", [(False, False), (True, False), (False, True)])
def test_rows_steps_match_plain_steps(multi, graph):
    scene, cams = _case(multi, 3)
    target = _target(scene, cams)
    p0 = gs.GaussianModel.from_scene(scene).data
    a = _run(scene, cams, target, None, 3, graph)
    b = _run(scene, cams, target, False, 3, graph)
    assert a.grad_rows and not b.grad_rows
    n = a.model.n
    # the tolerances of two runs of the plain sequence (atomics in the compositing backward)
    assert rel_l2(a.exp_avg.data[:, :n].cpu().numpy(), b.exp_avg.data[:, :n].cpu().numpy()) < 1e-4
    assert rel_l2(a.exp_avg_sq.data[:, :n].cpu().numpy(), b.exp_avg_sq.data[:, :n].cpu().numpy()) < 1e-4
    da = (a.model.data - p0)[:, :n].cpu().numpy()
    db = (b.model.data - p0)[:, :n].cpu().numpy()
    close = np.abs(da - db) <= 1e-6 + 1e-4 * np.abs(db)
    assert close.mean() > 0.999, close.mean()
    assert rel_l2(da, db) < 2e-2
    assert torch.equal(a.model.data[:, n:], p0[:, n:])
    assert rel_l2(a.buf.stats_acc[:, :n].cpu().numpy(), b.buf.stats_acc[:, :n].cpu().numpy()) < 1e-5


def test_rows_off_with_isotropy():
    scene, cams = _case(False, 0, n=500)
    st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, gs.Config(), lambda_iso=1.0)
    assert not st.grad_rows
