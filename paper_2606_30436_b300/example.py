"""One mapping iteration on the synthetic corridor (or a chunk), for trying
the library and for profiling a single launch of each kernel:

    python -m paper_2606_30436_b300.example --frame 500
    python -m paper_2606_30436_b300.example --chunk 16 --gaussians 2000000

Renders the frame(s), evaluates L = 0.8 L1 + 0.2 (1 - SSIM) against a random
target, back-propagates to every parameter and applies one Adam update,
then prints the visible-record and pair counts and the loss.
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
    args = ap.parse_args()
    if args.chunk:
        scene = scenes.uniform_scene(args.gaussians, seed=0, sh_degree=0)
        cams = scenes.chunk_cameras(args.chunk, seed=2)
    else:
        scene = scenes.corridor_scene(args.gaussians, seed=0, sh_degree=3)
        cams = [scenes.corridor_camera(args.frame)]
    model = gs.GaussianModel.from_scene(scene)
    st = gs.MappingStep(model, cams, gs.Config(), lambda_dssim=0.2, lr=gs.default_lr(extent=10.0))
    st.fit_capacity()
    target = torch.rand(3 * st.buf.total_pixels, device="cuda")
    for _ in range(args.iters):
        st.step(target)
    torch.cuda.synchronize()
    st.check_status()
    print("visible %d pairs %d loss %.6f" % (int(st.buf.counts[0]), int(st.buf.counts[1]), float(st.buf.loss.sum())))


if __name__ == "__main__":
    main()
