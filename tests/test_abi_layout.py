"""The ctypes mirrors of the C structs (gs.py, spawn.py, anchors.py) have the
sizes and field offsets that a C compiler gives the declarations of
include/gs.h: a small C program built against the header prints them."""
import ctypes as C
import os
import subprocess

import pytest

from paper_2606_30436_b300 import anchors, gs, spawn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# ctypes class, C struct name, {python field: C field} where the names differ
STRUCTS = [
    (gs.Camera, "gs_camera", {}),
    (gs.RasterCfg, "gs_raster_cfg", {}),
    (gs.Params, "gs_params", {}),
    (gs.Projected, "gs_projected", {}),
    (gs.Binning, "gs_binning", {}),
    (gs.PlaneSet, "gs_plane_set", {}),
    (gs.Frame, "gs_frame", {}),
    (gs.Stats, "gs_stats", {}),
    (gs.ChunkScores, "gs_chunk_scores", {}),
    (spawn.InitCfg, "gs_init_cfg", {"lam": "lambda", "scale": "intensity_scale"}),
    (spawn.VoxelTable, "gs_voxel_table", {}),
    (spawn.AnchorSet, "gs_anchor_set", {}),
    (anchors.AnchorParams, "gs_anchor_params", {}),
]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', 'int main(void) {']
    for cls, cname, rename in STRUCTS:
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in cls._fields_:
            cf = rename.get(field, field)
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, cf))
    lines += ['  return 0;', '}']
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True)
    return dict((k, int(v)) for k, v in (ln.split() for ln in out.splitlines()))


@pytest.mark.parametrize("cls,cname,rename", STRUCTS, ids=[s[1] for s in STRUCTS])
def test_struct_layout_matches_header(c_layout, cls, cname, rename):
    assert C.sizeof(cls) == c_layout[cname], cname
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout["%s.%s" % (cname, field)], (cname, field)


def test_header_constants_match_bindings():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()

    def define(name):
        for ln in src.splitlines():
            parts = ln.split()
            if len(parts) >= 3 and parts[0] == "#define" and parts[1] == name:
                return int(parts[2])
        raise KeyError(name)

    assert define("GS_ANCHOR_K") == anchors.K
    assert define("GS_ANCHOR_FEAT") == anchors.FEAT
    assert define("GS_ANCHOR_PLANES") == anchors.PLANES
    assert define("GS_ANCHOR_WEIGHTS") == anchors.WEIGHTS
    assert define("GS_INIT_MAX_LEVELS") == spawn.GS_INIT_MAX_LEVELS
    assert define("GS_MAX_VIEWS") == gs.GS_MAX_VIEWS
