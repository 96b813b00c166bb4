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

import numpy as np
import pytest
import torch

from paper_2606_30436_b300 import gs, scenes

pytestmark = pytest.mark.gpu


def _reference(x, y, cam, lam):
    model = gs.GaussianModel.from_scene(scenes.uniform_scene(8, seed=1))
    st = gs.MappingStep(model, [cam], gs.Config(), max_pairs=1024, lambda_dssim=lam)
    gs.gs_loss(st.buf, y, lam, img=x)
    torch.cuda.synchronize()
    return st.buf.loss.item(), st.buf.dL_dimg.clone()


@pytest.mark.parametrize("lam", [0.2, 0.0])
def test_loss_static_matches_workspace_entry_point(lam):
    shapes = [(720, 1280), (240, 320)]  # largest allowed view, then a smaller one over the leftovers
    for call, (H, W) in enumerate(shapes):
        x = torch.from_numpy(scenes.smooth_image(H, W, seed=20 + call)).cuda().reshape(-1)
        y = torch.from_numpy(scenes.smooth_image(H, W, seed=40 + call)).cuda().reshape(-1)
        cam = scenes.pinhole(W, H, 300.0)
        L_ref, dL_ref = _reference(x, y, cam, lam)
        loss = torch.full((1,), float("nan"), device="cuda")
        dL = torch.full_like(x, float("nan"))
        gs.gs_loss_static(x, y, [cam], loss, dL, lam)
        torch.cuda.synchronize()
        assert abs(loss.item() - L_ref) <= 1e-6 * max(1.0, abs(L_ref))
        assert torch.isfinite(dL).all()
        err = (dL - dL_ref).abs().max().item()
        assert err <= 1e-3 * dL_ref.abs().max().item(), err


def test_loss_static_rejects_views_beyond_its_array():
    L = gs.lib()
    cams = gs.camera_array([scenes.pinhole(1920, 1080, 900.0)])
    loss = torch.zeros(1, device="cuda")
    buf = torch.zeros(3 * 16, device="cuda")
    st = L.gs_loss_static(C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), cams, 1, 0.2,
                          C.c_void_p(loss.data_ptr()), C.c_void_p(buf.data_ptr()), None)
    assert st == 1  # GS_ERR_INVALID, nothing enqueued
