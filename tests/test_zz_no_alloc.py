"""The allocation-free loss entry point, gs_loss_static.

Callers that cannot allocate device memory where they need the loss (for
example code running while its allocator is unavailable, or a plain C host
that only gets image pointers from its framework) call gs_loss_static, whose
scratch is a device array inside the library instead of a caller workspace.
Its results must equal those of gs_loss, the workspace entry point, on two
calls in a row (the second reuses the array and must not see the first's
leftovers).  This file is collected last so a failure here cannot hide the
other GPU tests."""
import ctypes as C

import pytest
import torch

from paper_2606_30436_b300 import gs, scenes

pytestmark = pytest.mark.gpu


def _reference(x, y, cams, lam):
    model = gs.GaussianModel.from_scene(scenes.uniform_scene(8, seed=1))
    st = gs.MappingStep(model, cams, gs.Config(), max_pairs=1024, lambda_dssim=lam)
    gs.gs_loss(st.buf, y, lam, img=x)
    torch.cuda.synchronize()
    return st.buf.loss.clone(), st.buf.dL_dimg.clone()


def _images(shapes, seed):
    x = torch.cat([torch.from_numpy(scenes.smooth_image(H, W, seed=seed + k)).reshape(-1)
                   for k, (H, W) in enumerate(shapes)]).cuda()
    y = torch.cat([torch.from_numpy(scenes.smooth_image(H, W, seed=seed + 50 + k)).reshape(-1)
                   for k, (H, W) in enumerate(shapes)]).cuda()
    return x, y


@pytest.mark.parametrize("lam", [0.2, 0.0])
def test_loss_static_matches_workspace_entry_point(lam):
    """Both entry points launch the same kernels on the same inputs, so their
    losses and gradients are identical bit for bit: the largest allowed view,
    then a smaller one over the first call's leftovers, then one call with two
    views of different sizes (the array is reused view after view)."""
    calls = [[(720, 1280)], [(240, 320)], [(720, 1280), (240, 320)]]
    for k, shapes in enumerate(calls):
        x, y = _images(shapes, seed=20 + 10 * k)
        cams = [scenes.pinhole(W, H, 300.0) for (H, W) in shapes]
        L_ref, dL_ref = _reference(x, y, cams, lam)
        loss = torch.full((len(shapes),), float("nan"), device="cuda")
        dL = torch.full_like(x, float("nan"))
        gs.gs_loss_static(x, y, cams, loss, dL, lam)
        torch.cuda.synchronize()
        assert torch.equal(loss, L_ref), (loss, L_ref)
        assert torch.equal(dL, dL_ref)


def test_loss_static_rejects_views_beyond_its_array():
    L = gs.lib()
    cams = gs.camera_array([scenes.pinhole(1920, 1080, 900.0)])
    loss = torch.zeros(1, device="cuda")
    buf = torch.zeros(3 * 16, device="cuda")
    st = L.gs_loss_static(C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), cams, 1, 0.2,
                          C.c_void_p(loss.data_ptr()), C.c_void_p(buf.data_ptr()), None)
    assert st == 1  # GS_ERR_INVALID, nothing enqueued
