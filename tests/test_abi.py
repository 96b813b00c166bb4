"""The C-ABI library builds, loads without a GPU, exports exactly the symbols
that include/gs.h declares, and rejects bad arguments on the host before
touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2606_30436_b300 import build as gsbuild
from paper_2606_30436_b300 import gs, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = gsbuild.build()
    assert os.path.exists(path)
    L = gs.lib()
    assert L.gs_version() == 10000 + 1030


def test_exports_match_header():
    gs.lib()
    declared = _declared()
    assert len(declared) >= 14
    out = subprocess.check_output(["nm", "-D", "--defined-only", gsbuild.LIB], text=True)
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("gs_")})
    assert exported == declared
    assert set(gs.EXPORTS) == set(declared)


def test_status_strings():
    L = gs.lib()
    for code, name in gs.STATUS_NAMES.items():
        assert L.gs_status_string(code).decode() == name


def test_workspace_sizes_and_layout():
    L = gs.lib()
    n = C.c_size_t()
    assert L.gs_sort_workspace_size(1000, 5000, C.byref(n)) == 0 and n.value > 8 * 5000
    assert L.gs_sort_workspace_size(-1, 5000, C.byref(n)) == 1
    assert L.gs_loss_workspace_size(48, 64, C.byref(n)) == 0 and n.value >= 9 * 48 * 64 * 4
    assert L.gs_loss_workspace_size(0, 64, C.byref(n)) == 1
    cams = scenes.chunk_cameras(5)
    nt, npx, toff, poff = gs.view_layout(cams, gs.Config())
    tiles = [((c["width"] + 15) // 16) * ((c["height"] + 15) // 16) for c in cams]
    assert nt == sum(tiles) and list(toff) == list(np.cumsum([0] + tiles[:-1]))
    assert npx == sum(c["width"] * c["height"] for c in cams)


def test_invalid_arguments_rejected_on_host():
    L = gs.lib()
    cam = gs.camera_array([scenes.pinhole(64, 48, 60.0)])
    bad_tiles = gs.Config(tile_w=16, tile_h=8).c()
    nt = C.c_int64()
    assert L.gs_view_layout(cam, 1, C.byref(bad_tiles), C.byref(nt), None, None, None) == 1
    assert L.gs_view_layout(cam, 0, C.byref(gs.Config().c()), C.byref(nt), None, None, None) == 1
    assert L.gs_view_layout(cam, 65, C.byref(gs.Config().c()), C.byref(nt), None, None, None) == 1
    # misaligned / null parameter buffers never reach the device
    p = gs.Params(None, 10, 12, 0)
    proj = gs.Projected(16, 32, 48, 64, 80, 12)
    assert L.gs_project(C.byref(p), cam, 1, C.byref(gs.Config().c()), C.byref(proj), None, None) == 1
    p = gs.Params(4, 10, 12, 0)  # not 16-byte aligned
    assert L.gs_project(C.byref(p), cam, 1, C.byref(gs.Config().c()), C.byref(proj), None, None) == 1
    p = gs.Params(16, 10, 10, 0)  # ld not a multiple of 4
    assert L.gs_project(C.byref(p), cam, 1, C.byref(gs.Config().c()), C.byref(proj), None, None) == 1
    p = gs.Params(16, 10, 12, 4)  # SH degree beyond 3
    assert L.gs_project(C.byref(p), cam, 1, C.byref(gs.Config().c()), C.byref(proj), None, None) == 1
    lrs = (C.c_float * 6)(*([1e-3] * 6))
    q = gs.Params(16, 10, 12, 0)
    q2 = gs.Params(32, 10, 16, 0)  # ld mismatch
    assert L.gs_adam(C.byref(q), C.byref(q2), C.byref(q), C.byref(q), C.byref(lrs), 0.9, 0.999, 1e-15, 1, None,
                     None) == 1
    assert L.gs_adam(C.byref(q), C.byref(q), C.byref(q), C.byref(q), C.byref(lrs), 0.9, 0.999, 1e-15, 0, None,
                     None) == 1
    bad_batch = gs.Config(batch=64).c()
    assert L.gs_view_layout(cam, 1, C.byref(bad_batch), C.byref(nt), None, None, None) == 1
    # a kept colour gradient that is not 16-byte aligned
    p = gs.Params(16, 10, 12, 3)
    proj = gs.Projected(16, 32, 48, 64, 80, 12, 8)
    assert L.gs_project(C.byref(p), cam, 1, C.byref(gs.Config().c()), C.byref(proj), None, None) == 1


def test_reorder_arguments_rejected_on_host():
    L = gs.lib()
    p = gs.Params(256, 10, 12, 0)
    n = C.c_size_t()
    assert L.gs_reorder_workspace_size(10, 12, 14, C.byref(n)) == 0 and n.value > 0
    assert L.gs_reorder_workspace_size(10, 8, 14, C.byref(n)) == 1  # ld < n
    assert L.gs_reorder_workspace_size(10, 12, 0, C.byref(n)) == 1
    need = n.value
    L.gs_reorder_workspace_size(10, 12, 14, C.byref(n))
    ok = (gs.PlaneSet * 2)(gs.PlaneSet(512, 12, 14), gs.PlaneSet(768, 12, 6))
    # misaligned workspace, too small a workspace, an extra set of another ld, misaligned, too many sets
    assert L.gs_reorder(C.byref(p), ok, 2, None, 1024 + 16, need, None) == 1
    assert L.gs_reorder(C.byref(p), ok, 2, None, 1024, 64, None) == 1
    bad_ld = (gs.PlaneSet * 1)(gs.PlaneSet(512, 16, 14))
    assert L.gs_reorder(C.byref(p), bad_ld, 1, None, 1024, need, None) == 1
    bad_al = (gs.PlaneSet * 1)(gs.PlaneSet(520, 12, 14))
    assert L.gs_reorder(C.byref(p), bad_al, 1, None, 1024, need, None) == 1
    same = (gs.PlaneSet * 1)(gs.PlaneSet(256, 12, 14))  # the parameters themselves
    assert L.gs_reorder(C.byref(p), same, 1, None, 1024, need, None) == 1
    many = (gs.PlaneSet * 17)(*[gs.PlaneSet(512 + 256 * k, 12, 1) for k in range(17)])
    assert L.gs_reorder(C.byref(p), many, 17, None, 1024, need, None) == 1
    assert L.gs_reorder(C.byref(p), None, 1, None, 1024, need, None) == 1
    assert L.gs_reorder(C.byref(p), ok, 2, 2, 1024, need, None) == 1  # misaligned perm


def test_rows_arguments_rejected_on_host():
    L = gs.lib()
    cam = gs.camera_array([scenes.pinhole(64, 48, 60.0)])
    cfg = gs.Config().c()
    lrs = (C.c_float * 6)(*([1e-3] * 6))
    p = [gs.Params(256 * (k + 1), 10, 12, 0) for k in range(4)]
    proj = gs.Projected(16, 32, 48, 64, 80, 12)
    n = C.c_size_t()
    L.gs_bwd_workspace_size(12, C.byref(n))
    rad_ok = 1024
    args = lambda rows, rad, nv, part: (C.byref(p[0]), C.byref(p[1]), C.byref(p[2]), C.byref(p[3]), rows, rad, nv,
                                        part, C.byref(lrs), 0.9, 0.999, 1e-15, 1, None, None)
    assert L.gs_adam_part(*args(4096, rad_ok, 1, 0)) == 1      # part 0 is gs_adam_rows
    assert L.gs_adam_part(*args(4096, rad_ok, 1, 3)) == 1
    assert L.gs_adam_part(*args(None, rad_ok, 1, 1)) == 1      # part 1 needs the marks
    assert L.gs_adam_part(*args(None, 1028, 1, 2)) == 1        # radii not 16-byte aligned
    assert L.gs_adam_part(*args(None, rad_ok, 0, 2)) == 1      # no view
    assert L.gs_adam_part(*args(None, None, 1, 2)) == 1        # no radii
    for rows in (None, 4098):  # no marks, misaligned marks
        assert L.gs_adam_rows(C.byref(p[0]), C.byref(p[1]), C.byref(p[2]), C.byref(p[3]), rows, C.byref(lrs), 0.9,
                              0.999, 1e-15, 1, None, None) == 1
        assert L.gs_project_bwd_rows(C.byref(p[0]), cam, 1, C.byref(cfg), C.byref(proj), 8192, n.value, None,
                                     C.byref(p[1]), None, rows, None) == 1


def test_color_jac_policy():
    """The automatic choice keeps the colour gradient exactly where its bytes, 96 per
    visible record at most (written and read back), are below the 4 (K - 11) bytes of
    SH coefficients per Gaussian that the backward then skips."""
    auto = gs.Config()
    for D in range(4):
        for views in (1, 2, 3, 16):
            # K - 11 = 3 (D + 1)^2: 12, 27, 48 coefficients at degrees 1, 2, 3
            want = (D, views) in {(2, 1), (3, 1), (3, 2)}
            assert gs.use_color_jac(auto, D, views) == want, (D, views)
            assert gs.use_color_jac(gs.Config(color_jac=True), D, views) == (D >= 1)
            assert not gs.use_color_jac(gs.Config(color_jac=False), D, views)


def test_plane_packing_roundtrip():
    s = scenes.uniform_scene(37, seed=3, sh_degree=3)
    arr = gs.pack_planes(s, gs.padded(37))
    assert arr.shape == (gs.planes(3), 64)
    back = gs.unpack_planes(arr, 37, 3)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert np.array_equal(back[k], s[k])
    # SH coefficient k of channel c sits in plane 11 + 3k + c
    assert arr[11 + 3 * 5 + 2, 7] == s["sh"][7, 5, 2]


def test_segment_workspace_sizes():
    """Split-workspace sizing: the worst case for max_pairs covers 16 items per segment of pairs, sizes grow
    with the item count, and bad arguments are refused on the host."""
    L = gs.lib()
    n = C.c_size_t()
    sizes = []
    for items in (16, 17, 1000, 65536):
        assert L.gs_segment_workspace_size_items(items, C.byref(n)) == 0
        sizes.append(n.value)
    assert sizes == sorted(sizes) and sizes[0] > 0
    assert sizes[-1] > 65536 * 1400  # about 1.4 KB per item (local state, re-run slot, checkpoint)
    assert L.gs_segment_workspace_size(1_000_000, 256, C.byref(n)) == 0
    worst = n.value
    assert L.gs_segment_workspace_size_items(16 * (1_000_000 // 256 + 2), C.byref(n)) == 0
    assert worst <= n.value
    assert L.gs_segment_workspace_size(1000, 100, C.byref(n)) == 1   # not a power of two
    assert L.gs_segment_workspace_size(1000, 16, C.byref(n)) == 1    # below 32
    assert L.gs_segment_workspace_size_items(-1, C.byref(n)) == 1


def test_init_arguments_rejected_on_host():
    """The initialisation entry points refuse bad sizes, blur widths, level tables and
    table capacities before touching the device."""
    from paper_2606_30436_b300 import spawn
    L = spawn._lib()
    n = C.c_size_t()
    assert L.gs_init_workspace_size(1280, 720, C.byref(n)) == 0 and n.value >= 4 * 1280 * 720
    assert L.gs_init_workspace_size(0, 720, C.byref(n)) == 1
    assert L.gs_init_workspace_size(1 << 16, 1 << 16, C.byref(n)) == 1  # pixel index beyond int32
    ws = C.c_void_p(256)
    big = n.value
    ok = spawn.init_config()
    args = (C.c_void_p(16), C.c_void_p(32), None, None, 64, 48)
    for bad in (spawn.init_config(sigma1=6.0),   # radius ceil(18) beyond 16
                spawn.init_config(sigma2=0.0), spawn.init_config(lam=1.5), spawn.init_config(scale=0.0)):
        assert L.gs_init_probability(*args, C.byref(bad), C.c_void_p(48), ws, big, None) == 1
    # rendered pair given halfway, misaligned output, small workspace
    assert L.gs_init_probability(C.c_void_p(16), C.c_void_p(32), C.c_void_p(64), None, 64, 48, C.byref(ok),
                                 C.c_void_p(48), ws, big, None) == 1
    assert L.gs_init_probability(*args, C.byref(ok), C.c_void_p(52), ws, big, None) == 1
    assert L.gs_init_probability(*args, C.byref(ok), C.c_void_p(48), ws, 16, None) == 1
    cam = gs.make_camera(scenes.pinhole(64, 48, 60.0))
    good_table = spawn.VoxelTable(16, 32, 48, 1024)
    anchors = spawn.AnchorSet(16, 32, 48, 64, 100)
    for table in (spawn.VoxelTable(16, 32, 48, 1000),     # not a power of two
                  spawn.VoxelTable(16, 32, 48, 512),      # below 1024
                  spawn.VoxelTable(None, 32, 48, 1024)):
        assert L.gs_init_insert(C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), C.byref(cam), C.byref(ok),
                                C.byref(table), C.byref(anchors), None, None, ws, big, None) == 1
    for cfg in (spawn.init_config(voxel=(0.1, 0.25), max_dist=(10.0, 5.0)),   # bands not increasing
                spawn.init_config(voxel=(0.0,), max_dist=(10.0,))):
        assert L.gs_init_insert(C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), C.byref(cam), C.byref(cfg),
                                C.byref(good_table), C.byref(anchors), None, None, ws, big, None) == 1
    bad_count = spawn.AnchorSet(16, 32, 48, 60, 100)  # count not 8-byte aligned
    assert L.gs_init_insert(C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), C.byref(cam), C.byref(ok),
                            C.byref(good_table), C.byref(bad_count), None, None, ws, big, None) == 1
    assert L.gs_voxel_lookup(C.byref(good_table), C.c_void_p(16), 5, 4, C.c_void_p(32), None) == 1  # ld < n
    assert L.gs_voxel_table_reset(C.byref(spawn.VoxelTable(16, 32, 48, 3000)), None) == 1


def test_stored_list_arguments_rejected_on_host():
    L = gs.lib()
    n = C.c_size_t()
    assert L.gs_list_workspace_size(-1, C.byref(n)) == 1
    assert L.gs_list_workspace_size(921600, C.byref(n)) == 0 and n.value >= 8 * (921600 // 4096 + 1)
    cam = gs.camera_array([scenes.pinhole(64, 48, 60.0)])
    cfg = gs.Config().c()
    proj = gs.Projected(16, 32, 48, 64, 80, 12)
    binning = gs.Binning(16, 64, 128, 256, 512, 1000)
    frame = gs.Frame(16, 32, 48, None, None, 0)
    ws = 256
    # offsets missing or misaligned, events without their arrays: rejected before any launch
    assert L.gs_render_fwd_lists(C.byref(proj), C.byref(binning), cam, 1, C.byref(cfg), C.byref(frame), None, 64, 80,
                                 10, ws, 1 << 20, None, None) == 1
    assert L.gs_render_fwd_lists(C.byref(proj), C.byref(binning), cam, 1, C.byref(cfg), C.byref(frame), 4, 64, 80,
                                 10, ws, 1 << 20, None, None) == 1
    assert L.gs_render_fwd_lists(C.byref(proj), C.byref(binning), cam, 1, C.byref(cfg), C.byref(frame), 64, None, None,
                                 10, ws, 1 << 20, None, None) == 1
    assert L.gs_render_fwd_lists(C.byref(proj), C.byref(binning), cam, 1, C.byref(cfg), C.byref(frame), 64, 64, 80,
                                 10, ws, 4, None, None) == 1  # scan workspace too small
    p = gs.Params(16, 10, 12, 0)
    assert L.gs_render_bwd_lists(C.byref(p), cam, 1, C.byref(cfg), C.byref(proj), C.byref(frame), None, 64, 80, 10,
                                 96, None, None, 0.1, None, 0, None, ws, 1 << 20, None) == 1
