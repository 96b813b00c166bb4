"""One mapping iteration on the synthetic corridor (or a chunk), for trying
the library and for profiling a single launch of each kernel:

    python -m paper_2606_30436_b300.example --frame 500
    python -m paper_2606_30436_b300.example --chunk 16 --gaussians 2000000
    python -m paper_2606_30436_b300.example --mlp 4000000
    python -m paper_2606_30436_b300.example --keyframe --iters 60

Renders the frame(s), evaluates L = 0.8 L1 + 0.2 (1 - SSIM) against a random
target, back-propagates to every parameter and applies one Adam update,
then prints the visible-record and pair counts and the loss.  With --mlp N:
one inference, one training gradient and one Adam step of the learned
densify / prune predictor over N rows of random inputs.  With --keyframe: a
synthetic 360x640 driving keyframe spawns anchors (probability map, 3x3 NMS,
voxel hash), which are then mapped on the keyframe's own image for --iters
anchor iterations (prints the anchor count and the loss before and after).
"""
from __future__ import annotations

import argparse

import torch

from . import gs, scenes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frame", type=int, default=500)
    ap.add_argument("--gaussians", type=int, default=1_000_000)
    ap.add_argument("--chunk", type=int, default=0, help="keyframes of a batched chunk (0: one corridor view)")
    ap.add_argument("--iters", type=int, default=1)
    ap.add_argument("--mlp", type=int, default=0, help="rows for the predictor instead of a mapping iteration")
    ap.add_argument("--keyframe", action="store_true",
                    help="initialise anchors at a synthetic keyframe and map them on its image")
    ap.add_argument("--keyframe-size", type=int, nargs=2, default=(360, 640), metavar=("H", "W"))
    ap.add_argument("--segment", type=int, default=None,
                    help="split length of long tile lists (default: 512 for a corridor view, none for a chunk)")
    ap.add_argument("--graph", action="store_true",
                    help="capture the iteration in a CUDA graph and replay it (as the benchmark does)")
    ap.add_argument("--no-reorder", action="store_true",
                    help="keep the scene's row order (default: the Morton order of the means, gs_reorder)")
    args = ap.parse_args()
    if args.keyframe:
        # a new keyframe: probability map, voxel insertion, anchors, anchor mapping on its image
        from . import anchors, spawn
        H, W = args.keyframe_size
        img, depth, U = scenes.keyframe(H, W, seed=51)
        cam = scenes.keyframe_camera(H, W, seed=52, centre=(0.0, -1.6, 20.0))
        prob = spawn.gs_init_probability(torch.from_numpy(img).cuda(), torch.from_numpy(depth).cuda())
        amap = spawn.AnchorMap(H * W // 4 + 16)
        amap.insert(prob, torch.from_numpy(U).cuda(), torch.from_numpy(depth).cuda(), cam)
        torch.cuda.synchronize()
        amap.check_status()
        model = anchors.AnchorModel.from_anchor_map(amap)
        st = anchors.AnchorStep(model, cam, gs.Config(), lambda_dssim=0.2)
        st.fit_capacity(slack=3.0)
        tgt = torch.from_numpy(img.reshape(-1)).cuda()
        losses = [float(st.step(tgt).item()) for _ in range(args.iters)]
        st.map.check_status()
        print("anchors %d, loss %.5f -> %.5f over %d iterations" % (model.n, losses[0], losses[-1], len(losses)))
        return
    if args.mlp:
        n = args.mlp
        ld = gs.padded(n)
        g = torch.Generator(device="cuda").manual_seed(0)
        feat = torch.rand(gs.MLP_INPUTS, ld, device="cuda", generator=g)
        y = (torch.rand(2, n, device="cuda", generator=g) < 0.2).to(torch.uint8)
        w = gs.mlp_init(0)
        grad, m, v = torch.zeros_like(w), torch.zeros_like(w), torch.zeros_like(w)
        loss = torch.zeros(1, device="cuda")
        prob = torch.empty(2, ld, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        for it in range(args.iters):
            gs.gs_mlp_forward(feat, n, w, prob, None, None, status)
            gs.gs_mlp_train_grad(feat, y[0].contiguous(), y[1].contiguous(), n, w, grad, loss, status)
            gs.gs_mlp_adam(w, grad, m, v, 1e-3, it + 1)
        torch.cuda.synchronize()
        print("rows %d bce %.6f status %d" % (n, float(loss), int(status)))
        return
    if args.chunk:
        scene = scenes.uniform_scene(args.gaussians, seed=0, sh_degree=0)
        cams = scenes.chunk_cameras(args.chunk, seed=2)
    else:
        scene = scenes.corridor_scene(args.gaussians, seed=0, sh_degree=3)
        cams = [scenes.corridor_camera(args.frame)]
    model = gs.GaussianModel.from_scene(scene)
    segment = args.segment if args.segment is not None else (0 if args.chunk else 512)
    st = gs.MappingStep(model, cams, gs.Config(segment=segment), lambda_dssim=0.2, lr=gs.default_lr(extent=10.0))
    if not args.no_reorder:
        st.reorder()
    st.fit_capacity()
    target = torch.rand(3 * st.buf.total_pixels, device="cuda")
    if args.graph:
        g = st.capture(target)
        for _ in range(args.iters):
            st.replay(g)
    else:
        for _ in range(args.iters):
            st.step(target)
    torch.cuda.synchronize()
    st.check_status()
    print("visible %d pairs %d loss %.6f" % (int(st.buf.counts[0]), int(st.buf.counts[1]), float(st.buf.loss.sum())))


if __name__ == "__main__":
    main()
