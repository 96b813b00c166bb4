"""The number of the library's kernel launches in one captured mapping iteration (the nodes of
the CUDA graph whose kernels live in the library's namespace) equals gs.launches_per_step, the
count the benchmark reports as gpu_launches: single view with the split compositing, several
views, no split, and the fused projection backward + Adam."""
import numpy as np
import pytest
import torch

from paper_2606_30436_b300 import gs, scenes

pytestmark = pytest.mark.gpu


def _library_kernels(graph):
    import cuda.bindings.driver as dr
    raw = dr.CUgraph(graph.raw_cuda_graph())
    err, _, n = dr.cuGraphGetNodes(raw, 0)
    assert err == dr.CUresult.CUDA_SUCCESS
    err, nodes, n = dr.cuGraphGetNodes(raw, n)
    assert err == dr.CUresult.CUDA_SUCCESS
    names = []
    for node in nodes[:n]:
        err, kind = dr.cuGraphNodeGetType(node)
        assert err == dr.CUresult.CUDA_SUCCESS
        if kind != dr.CUgraphNodeType.CU_GRAPH_NODE_TYPE_KERNEL:
            continue
        err, params = dr.cuGraphKernelNodeGetParams(node)
        assert err == dr.CUresult.CUDA_SUCCESS
        err, name = dr.cuFuncGetName(params.func)
        if err != dr.CUresult.CUDA_SUCCESS:  # a kernel handle rather than a function
            err, name = dr.cuKernelGetName(params.kern)
        assert err == dr.CUresult.CUDA_SUCCESS
        names.append(name.decode() if isinstance(name, bytes) else str(name))
    return [nm for nm in names if nm.startswith("_ZN2gs")], names


@pytest.mark.parametrize("case", ["single", "multi", "nosplit", "fused"])
def test_graph_launches_match_count(case):
    if case == "multi":
        scene = scenes.uniform_scene(3000, seed=7, sh_degree=3, xy_range=3.0)
        cams = [scenes.pinhole(100, 70, 90.0),
                scenes.pinhole(150, 90, 140.0, R=scenes.yaw_matrix(4.0), t=np.array([0.2, -0.1, 0.3], np.float32))]
    else:
        scene = scenes.corridor_scene(40_000, seed=2, sh_degree=3, length=100.0)
        cams = [scenes.corridor_camera(20, 320, 240, 260.0)]
    cfg = gs.Config(segment=0) if case == "nosplit" else gs.Config(segment=64)
    st = gs.MappingStep(gs.GaussianModel.from_scene(scene), cams, cfg, lambda_dssim=0.2,
                        fused_adam=case == "fused")
    st.fit_capacity(slack=2.0)
    target = torch.rand(3 * st.buf.total_pixels, device="cuda")
    g = st.capture(target, keep_graph=True)
    ours, _ = _library_kernels(g)
    want = gs.launches_per_step(st.buf.total_tiles, views=len(cams), lambda_dssim=0.2, segment=cfg.segment,
                                fused_adam=st.fused_adam, adam_split=st.adam_split and not st.fused_adam)
    assert len(ours) == want, (len(ours), want, sorted(set(ours)))
    st.replay(g)
    torch.cuda.synchronize()
    st.check_status()
