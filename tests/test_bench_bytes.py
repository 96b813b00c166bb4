"""Host checks of the benchmark's byte accounting: the per-stage algorithmic
bytes of one view follow the minimum-traffic formulas of each step, the whole
iteration counts only the stages that ran (the fused projection backward +
Adam stage replaces two stages and is not added on top), and a chunk reads
its parameters once."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_single_view_stage_bytes():
    N, K, V, P, px, tiles = 1_000_000, 59, 494_279, 1_177_411, 921_600, 3600
    b = bench.step_bytes(N, K, [(V, P, px, tiles)])
    assert b["project"] == 12 * N + 4 * (K - 3) * V + 56 * V + 4 * N
    assert b["sort"] == 8 * N + 16 * V + 12 * P + 24 * P + 8 * P + 8 * tiles
    assert b["render_fwd"] == 4 * P + 36 * P + 20 * px
    assert b["loss"] == 36 * px
    assert b["render_bwd"] == 40 * P + 12 * px + 20 * px + 36 * V
    assert b["project_bwd"] == 4 * K * V + 4 * K * N + 32 * V
    assert b["adam"] == 28 * K * N
    # about 2.44 GB per iteration at the corridor's mean counts
    total = bench.executed_bytes(b, bench.STAGES)
    assert total == pytest.approx(2.436e9, rel=2e-3)


def test_fused_stage_not_counted_twice():
    b = bench.step_bytes(1000, 14, [(600, 2000, 4096, 16)])
    unfused = bench.executed_bytes(b, bench.STAGES)
    fused = bench.executed_bytes(b, bench.STAGES_FUSED)
    assert unfused == fused == sum(b[s] for s in bench.STAGES)
    assert "project_bwd_adam" not in bench.STAGES


def test_chunk_reads_parameters_once():
    N, K = 1000, 14
    one = (600, 2000, 4096, 16)
    b1 = bench.step_bytes(N, K, [one])
    b4 = bench.step_bytes(N, K, [one] * 4)
    # per-view terms scale with the views; the parameter reads are bounded by N
    assert b4["render_fwd"] == 4 * b1["render_fwd"] and b4["sort"] == 4 * b1["sort"]
    assert b4["adam"] == b1["adam"]
    assert b4["project"] == 12 * N + 4 * (K - 3) * N + 4 * (56 * 600 + 4 * N)
    assert b4["project_bwd"] == 4 * K * N + 4 * K * N + 4 * 32 * 600


def test_color_jacobian_bytes():
    """The kept colour gradient moves 48 bytes per record out and back in place of
    the projection backward's 4(K-11) bytes of SH coefficients per visible Gaussian."""
    N, K, V, P, px, tiles = 1_000_000, 59, 494_279, 1_177_411, 921_600, 3600
    b0 = bench.step_bytes(N, K, [(V, P, px, tiles)])
    b1 = bench.step_bytes(N, K, [(V, P, px, tiles)], color_jac=True)
    assert b1["project"] == b0["project"] + 48 * V
    assert b1["project_bwd"] == 4 * 11 * V + 4 * K * N + 32 * V + 48 * V
    assert b1["adam"] == b0["adam"] and b1["render_bwd"] == b0["render_bwd"]
    # SH degree 0 keeps nothing
    assert bench.step_bytes(N, 14, [(V, P, px, tiles)], color_jac=True) == bench.step_bytes(N, 14, [(V, P, px, tiles)])


def test_grad_rows_bytes():
    """Writing and reading only the gradient rows of the visible union saves 8 bytes per
    parameter element of the Gaussians no view sees, for one mark byte per Gaussian each way."""
    N, K, V, P, px, tiles = 1_000_000, 59, 494_279, 1_177_411, 921_600, 3600
    b0 = bench.step_bytes(N, K, [(V, P, px, tiles)], color_jac=True)
    b1 = bench.step_bytes(N, K, [(V, P, px, tiles)], color_jac=True, grad_rows=True)
    assert b0["project_bwd"] - b1["project_bwd"] == 4 * K * (N - V) - N
    assert b0["adam"] - b1["adam"] == 4 * K * (N - V) - N
    assert b1["project"] == b0["project"] and b1["render_bwd"] == b0["render_bwd"]


def test_adam_split_bytes():
    """The split Adam moves the same bytes as the marked-rows Adam, the unseen Gaussians' share
    in the background kernel (which reads the radii instead of the marks), counted once."""
    N, K, V, P, px, tiles = 1_000_000, 59, 494_279, 1_177_411, 921_600, 3600
    b1 = bench.step_bytes(N, K, [(V, P, px, tiles)], color_jac=True, grad_rows=True)
    b2 = bench.step_bytes(N, K, [(V, P, px, tiles)], color_jac=True, grad_rows=True, adam_split=True)
    assert b2["adam"] == 28 * K * V + N
    assert b2["adam_unseen"] == 24 * K * (N - V) + 4 * N
    assert b2["adam"] + b2["adam_unseen"] == b1["adam"] + 4 * N
    assert bench.executed_bytes(b2, bench.STAGES) == sum(b2[s] for s in bench.STAGES) + b2["adam_unseen"]
    assert "adam_unseen" not in b1
