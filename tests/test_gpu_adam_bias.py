"""Adam's bias corrections from a device step counter (graph replay; formed on the GPU in
double-float arithmetic, no FP64) against those the host forms in FP64 from the same step:
the Gaussians' Adam and the flat Adam give bit-identical parameters and moments for small and
large steps and for other betas."""
import numpy as np
import pytest
import torch

from paper_2606_30436_b300 import anchors, gs, scenes

pytestmark = pytest.mark.gpu
STEPS = [1, 2, 3, 7, 10, 99, 1000, 4097, 123457, 10**6, 2**40 + 3]
BETAS = [(0.9, 0.999), (0.5, 0.99), (0.95, 0.9999)]


def _flat(seed, n=4096):
    rng = np.random.default_rng(seed)
    x = [rng.normal(size=n).astype(np.float32) for _ in range(3)] + [rng.random(n).astype(np.float32) * 1e-3]
    return [torch.from_numpy(v).cuda() for v in x]


@pytest.mark.parametrize("b1,b2", BETAS)
def test_flat_adam_device_step_is_host_step(b1, b2):
    for t in STEPS:
        a, b = _flat(t % 1000), _flat(t % 1000)
        anchors.gs_adam_flat(*a, 1e-3, t, beta1=b1, beta2=b2)
        anchors.gs_adam_flat(*b, 1e-3, 1, beta1=b1, beta2=b2,
                             step_device=torch.full((1,), t, dtype=torch.int64, device="cuda"))
        torch.cuda.synchronize()
        for u, w in zip(a, b):
            assert torch.equal(u, w), t


@pytest.mark.parametrize("b1,b2", BETAS)
def test_gaussian_adam_device_step_is_host_step(b1, b2):
    model = gs.GaussianModel.from_scene(scenes.uniform_scene(1000, seed=2, sh_degree=1))
    g = torch.Generator(device="cuda").manual_seed(3)
    grads = model.like()
    grads.data.copy_(torch.randn(model.data.shape, generator=g, device="cuda"))
    m0 = torch.randn(model.data.shape, generator=g, device="cuda") * 1e-3
    v0 = torch.rand(model.data.shape, generator=g, device="cuda") * 1e-6
    lr = gs.default_lr(10.0)
    for t in STEPS:
        out = []
        for device_step in (False, True):
            p, m, v = model.like(), model.like(), model.like()
            p.data.copy_(model.data)
            m.data.copy_(m0)
            v.data.copy_(v0)
            sd = torch.full((1,), t, dtype=torch.int64, device="cuda") if device_step else None
            gs.gs_adam(p, grads, m, v, lr, 1 if device_step else t, beta1=b1, beta2=b2, step_device=sd)
            out.append((p.data, m.data, v.data))
        torch.cuda.synchronize()
        for u, w in zip(*out):
            assert torch.equal(u, w), t
