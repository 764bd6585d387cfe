"""The C ABI without a GPU: the library builds, loads and exports every entry
point include/fhv.h declares; host-only calls (memory model, sizes, level
layout, argument checks) behave as documented. No kernel is launched."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2211_15460_gb300 import fhv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def header_functions():
    text = open(os.path.join(ROOT, "include", "fhv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fhv_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    lib = fhv.lib()
    declared = header_functions()
    assert set(declared) == set(fhv.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_record_layout_matches_header():
    assert fhv.RECORD_DTYPE.itemsize == 16
    assert C.sizeof(fhv.fhv_scene) == 4 * 8 + 2 * 4 + 4 * 4 + 8  # tri_base + tail padding
    assert C.sizeof(fhv.fhv_ortho_camera) == 12 * 4 + 4 + 8 + 8


STRUCTS = ("fhv_scene", "fhv_ortho_camera", "fhv_frag_buf", "fhv_sizes", "fhv_splat_source", "fhv_view",
           "fhv_batch_config", "fhv_pofa_header")


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every field offset and struct size of the binding's ctypes structures
    equals the C compiler's for include/fhv.h."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include "fhv.h"', "int main(void) {"]
    expect = []
    for name in STRUCTS:
        st = getattr(fhv, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(C.sizeof(st))
        for field, *_ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field}));')
            expect.append(getattr(st, field).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def test_scene_tri_base_read_by_the_library():
    """The library reads tri_base where the binding writes it. With three
    setups per triangle (FHV_CAPTURE_AXIS3), 0x60000000 triangles exceed the
    2^32 setups the capture indexes: FHV_ERR_UNSUPPORTED for an accepted
    scene. Moving the same slice to tri_base = 0xA0000000 puts its ids past
    2^32 - 1, so the scene itself is rejected: FHV_ERR_INVALID_ARG. Both
    return before any launch."""
    L = fhv.lib()
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    sc.idx = sc.pos = sc.nrm = 16
    sc.n_vtx = 3
    sc.n_tri = 0x60000000

    def call():
        return L.fhv_build_pofa_direct(C.byref(sc), fhv.FHV_CAPTURE_AXIS3, None, C.c_float(1.0), 4, None, 0, 16, 16,
                                       16, 16, 1 << 20, None)

    sc.tri_base = 0
    assert call() == fhv.FHV_ERR_UNSUPPORTED
    sc.tri_base = 0xA0000000
    assert call() == fhv.FHV_ERR_INVALID_ARG
    sc.tri_base = 0x9FFFFFFE  # ids up to 0xFFFFFFFD: accepted again
    assert call() == fhv.FHV_ERR_UNSUPPORTED


def test_level_layout_is_root_first_and_aligned():
    assert fhv.fhv_level_offset(0) == 0
    assert fhv.fhv_level_offset(1) == 4
    for l in range(1, 12):
        assert fhv.fhv_level_offset(l + 1) - fhv.fhv_level_offset(l) == 8 ** l
        assert (fhv.fhv_level_offset(l) * 4) % 16 == 0


def test_memory_model_reproduces_table4():
    """Table 4 (Section 4) through the library's sizing call."""
    F = {"simple": 514479, "complex": 1685548}
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table4_memory.txt")) if l.strip() and not l.startswith("#")]
    for layout, lev, scene, mb in rows:
        if layout == "DS":
            continue
        lay = {"PPFL": fhv.FHV_LAYOUT_PPFL, "POFL": fhv.FHV_LAYOUT_POFL, "POFA": fhv.FHV_LAYOUT_POFA}[layout]
        b = fhv.fhv_memory_model(lay, 1000 * 1000, int(lev) if lev != "-" else 0, 10.0, F[scene], 48, 32)
        assert round(b / 2 ** 20) == int(mb), (layout, lev, scene)


def test_query_sizes():
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_PPFL, 1000, 640, 480, 1, 12345)
    assert s.index_bytes == 640 * 480 * 4 and s.fragment_bytes == 12345 * 20
    assert s.workspace_bytes >= 1000 * (96 + 8)
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, 10, 1, 1, 6, 0)
    assert s.n_index_entries == 8 ** 6 + fhv.fhv_level_offset(6)
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, 10, 1000)
    assert s.n_index_entries == fhv.fhv_level_offset(11)
    assert s.index_bytes == 8 * s.n_index_entries
    for depth in (0, 12):
        with pytest.raises(fhv.FhvError):
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, depth, 10)


def test_invalid_arguments_rejected_on_host():
    L = fhv.lib()
    assert L.fhv_capture_ppfl(None, None, None, None, None, 0, None) == fhv.FHV_ERR_INVALID_ARG
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    cam = fhv.fhv_ortho_camera()
    cam.pitch, cam.width, cam.height, cam.z0, cam.z1 = 1.0, 4, 4, -1.0, 1.0
    fb = fhv.fhv_frag_buf()
    # NULL device pointers / bad depth / bad pitch never reach the GPU
    assert L.fhv_capture_ppfl(C.byref(sc), C.byref(cam), None, C.byref(fb), None, 0, None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_build_pofl(C.byref(sc), 1, None, C.c_float(0.0), 3, 16, 16, C.byref(fb), 16, 1 << 20,
                            None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_build_pofl(C.byref(sc), 1, None, C.c_float(1.0), 12, 16, 16, C.byref(fb), 16, 1 << 20,
                            None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_compact_pofa(None, 10, None, 0, None, None, None, None, 0, None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_compact_pofa(16, 1 << 32, None, 5, 32, 16, 16, 16, 1 << 40, None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_render_view(None, 0, None, C.byref(sc), None, None, 0, C.byref(cam), 0, 16, 16, 16, 256,
                             None) == fhv.FHV_ERR_INVALID_ARG
    cam.z1 = -2.0
    assert L.fhv_render_view(None, 0, None, C.byref(sc), None, None, 0, C.byref(cam), 1, 16, 16, 16, 256,
                             None) == fhv.FHV_ERR_INVALID_ARG
    assert fhv.status_str(fhv.FHV_ERR_INVALID_ARG) == "invalid argument"


def test_raycast_arguments_rejected_on_host():
    L = fhv.lib()
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    cam = fhv.fhv_ortho_camera()
    cam.pitch, cam.width, cam.height, cam.z0, cam.z1 = 1.0, 4, 4, -1.0, 1.0

    def call(off=16, cnt=16, depth=3, t_stop=0.0, n_lights=0, cam_=cam):
        return L.fhv_raycast_pofa(None, 0, off, cnt, depth, C.byref(sc), None, None, C.c_float(t_stop), None, n_lights,
                                  C.byref(cam_), 16, 16, 16, 256, None)

    assert call(off=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(cnt=8) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    for depth in (0, 12):
        assert call(depth=depth) == fhv.FHV_ERR_INVALID_ARG
    for t in (-0.1, 1.0, float("nan")):
        assert call(t_stop=t) == fhv.FHV_ERR_INVALID_ARG
    assert call(n_lights=1) == fhv.FHV_ERR_INVALID_ARG  # lights missing
    cam.z1 = -2.0
    assert call() == fhv.FHV_ERR_INVALID_ARG


def test_split_render_arguments_rejected_on_host():
    L = fhv.lib()
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    cam = fhv.fhv_ortho_camera()
    cam.pitch, cam.width, cam.height, cam.z0, cam.z1 = 1.0, 4, 4, -1.0, 1.0

    def splat(n=0, base=0, k=1, vis=16, ws_bytes=256):
        return L.fhv_splat_visibility(16 if n else None, n, None, base, C.byref(sc), C.byref(cam), k, vis, 16,
                                      ws_bytes, None)

    def shade(n=0, base=0, n_lights=0, rgba=16):
        return L.fhv_shade_owned(16 if n else None, n, None, base, C.byref(sc), None, None, n_lights, C.byref(cam),
                                 16, rgba, 16, 256, None)

    assert splat(base=1 << 40) == fhv.FHV_ERR_INVALID_ARG
    assert splat(n=10, base=(1 << 40) - 5) == fhv.FHV_ERR_INVALID_ARG  # indices past 2^40
    assert splat(k=0) == fhv.FHV_ERR_INVALID_ARG
    assert splat(vis=8) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    assert splat(ws_bytes=128) == fhv.FHV_ERR_INVALID_ARG
    assert shade(n_lights=1) == fhv.FHV_ERR_INVALID_ARG  # lights missing
    assert shade(rgba=8) == fhv.FHV_ERR_INVALID_ARG
    assert shade(n=10, base=(1 << 40) - 5) == fhv.FHV_ERR_INVALID_ARG


def test_leaf_index_arguments_rejected_on_host():
    L = fhv.lib()

    def call(n=16, depth=6, m=16, ws=16, ws_bytes=None):
        wsb = fhv.FHV_LEAF_INDEX_WS_BYTES(n) if ws_bytes is None else ws_bytes
        return L.fhv_pofa_leaf_index(16, n, None, depth, 16, 16, 16, m, ws, wsb, None)

    for depth in (0, 12):
        assert call(depth=depth) == fhv.FHV_ERR_INVALID_ARG
    assert call(n=0xFFFFFFFF) == fhv.FHV_ERR_INVALID_ARG
    assert call(m=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(m=8) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    assert call(ws_bytes=fhv.FHV_LEAF_INDEX_WS_BYTES(16) - 1) == fhv.FHV_ERR_INVALID_ARG
    assert fhv.FHV_LEAF_INDEX_WS_BYTES(4097) == 16 + 12 * 2


def test_wait_probe_arguments_rejected_on_host():
    L = fhv.lib()
    for kind in (-1, 3):
        assert L.fhv_wait_probe(kind, 16, fhv.FHV_WAIT_PROBE_WS_BYTES, None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_wait_probe(0, None, fhv.FHV_WAIT_PROBE_WS_BYTES, None) == fhv.FHV_ERR_INVALID_ARG
    assert L.fhv_wait_probe(1, 8, fhv.FHV_WAIT_PROBE_WS_BYTES, None) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    assert L.fhv_wait_probe(2, 16, fhv.FHV_WAIT_PROBE_WS_BYTES - 1, None) == fhv.FHV_ERR_INVALID_ARG


def test_direct_pofa_sizes_and_arguments_rejected_on_host():
    cap, t = 100000, 5000
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_DIRECT, t, 1, 1, 8, cap)
    a = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, 8, cap)
    p = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, t, 1, 1, 8, 0)
    assert s.workspace_bytes == a.workspace_bytes + p.workspace_bytes  # capture part + compaction part
    assert s.n_index_entries == a.n_index_entries and s.fragment_bytes == cap * 16
    for depth in (0, 12):
        with pytest.raises(fhv.FhvError):
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_DIRECT, t, 1, 1, depth, cap)
    L = fhv.lib()
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    wsb = s.workspace_bytes

    def call(mode=1, pitch=1.0, depth=8, pofa=16, capacity=cap, count=16, off=16, cnt=16, ws=16, ws_bytes=wsb, scene=sc):
        return L.fhv_build_pofa_direct(C.byref(scene) if scene is not None else None, mode, None, C.c_float(pitch),
                                       depth, pofa, capacity, count, off, cnt, ws, ws_bytes, None)

    assert call(scene=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(mode=0) == fhv.FHV_ERR_INVALID_ARG  # VIEW needs a camera
    assert call(mode=3) == fhv.FHV_ERR_INVALID_ARG
    assert call(pitch=0.0) == fhv.FHV_ERR_INVALID_ARG
    for depth in (0, 12):
        assert call(depth=depth) == fhv.FHV_ERR_INVALID_ARG
    assert call(pofa=None) == fhv.FHV_ERR_INVALID_ARG  # records wanted but no output
    assert call(pofa=8) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    assert call(count=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(count=8) == fhv.FHV_ERR_INVALID_ARG
    assert call(off=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(cnt=24) == fhv.FHV_ERR_INVALID_ARG
    assert call(capacity=0xFFFFFFFF) == fhv.FHV_ERR_INVALID_ARG
    assert call(ws_bytes=wsb - 1 - (fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, t, 1, 1, 8, 0).workspace_bytes
                                    - fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, 0, 1, 1, 8, 0).workspace_bytes)) \
        == fhv.FHV_ERR_INVALID_ARG
    assert call(ws=8) == fhv.FHV_ERR_INVALID_ARG


def test_sparse_compaction_sizes_and_arguments_rejected_on_host():
    """fhv_compact_pofa_sparse: the index bound is sum over levels of
    min(8^l, n); the workspace has no term of size 8^depth; bad arguments
    are refused before anything is launched."""
    n, d = 100000, 11
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, n)
    assert s.n_index_entries == sum(min(8 ** l, n) for l in range(d + 1))
    assert s.index_bytes == 16 * s.n_index_entries and s.fragment_bytes == 16 * n
    assert s.workspace_bytes < 16 * n + 16 * 8 ** (d - 3) + (1 << 20)  # scratch + buckets, nothing of 8^d
    # many records: buckets one level finer (8^(d - 2) <= n / 2), still nothing of 8^d
    big = 300_000_000
    sb = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, big)
    assert 16 * big + 16 * 8 ** (d - 2) <= sb.workspace_bytes < 16 * big + 16 * 8 ** (d - 2) + 8 * big
    assert sb.workspace_bytes < 8 ** d
    assert fhv.OCTANT_DTYPE.itemsize == 16
    for depth in (0, 12):
        with pytest.raises(fhv.FhvError):
            fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, depth, n)
    L = fhv.lib()
    wsb = s.workspace_bytes

    def call(inp=16, n_max=n, d_n=None, depth=d, pofa=1 << 40, index=32, cap=1000, base=48, ws=64, ws_bytes=wsb):
        return L.fhv_compact_pofa_sparse(inp, n_max, d_n, depth, pofa, index, cap, base, ws, ws_bytes, None)

    for depth in (0, 12):
        assert call(depth=depth) == fhv.FHV_ERR_INVALID_ARG
    assert call(n_max=0xFFFFFFFF) == fhv.FHV_ERR_INVALID_ARG
    assert call(base=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(base=8) == fhv.FHV_ERR_INVALID_ARG  # misaligned
    assert call(index=None) == fhv.FHV_ERR_INVALID_ARG  # capacity without an array
    assert call(index=24) == fhv.FHV_ERR_INVALID_ARG
    assert call(inp=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(pofa=16) == fhv.FHV_ERR_INVALID_ARG  # overlaps the input
    assert call(d_n=8) == fhv.FHV_ERR_INVALID_ARG
    assert call(ws_bytes=wsb - 1) == fhv.FHV_ERR_INVALID_ARG
    assert call(ws=None) == fhv.FHV_ERR_INVALID_ARG


def test_capture_fragments_arguments_rejected_on_host():
    """Records-only capture: no list arrays needed (next may be NULL), but
    the scene, mode, counter and workspace are checked as for a list build."""
    L = fhv.lib()
    sc = fhv.fhv_scene()
    sc.cube_side = 1.0
    f = fhv.fhv_frag_buf()
    f.rec, f.next, f.capacity, f.d_count = 16, None, 10, 32
    wsb = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, 0, 1, 1, 6, 0).workspace_bytes

    def call(scene=sc, mode=1, pitch=1.0, frags=f, ws=64, ws_bytes=wsb):
        return L.fhv_capture_fragments(C.byref(scene) if scene is not None else None, mode, None, C.c_float(pitch),
                                       C.byref(frags) if frags is not None else None, ws, ws_bytes, None)

    assert call(scene=None) == fhv.FHV_ERR_INVALID_ARG
    assert call(mode=0) == fhv.FHV_ERR_INVALID_ARG  # VIEW needs a camera
    assert call(mode=3) == fhv.FHV_ERR_INVALID_ARG
    assert call(pitch=0.0) == fhv.FHV_ERR_INVALID_ARG
    assert call(frags=None) == fhv.FHV_ERR_INVALID_ARG
    g = fhv.fhv_frag_buf()
    g.rec, g.next, g.capacity, g.d_count = None, None, 10, 32
    assert call(frags=g) == fhv.FHV_ERR_INVALID_ARG  # capacity without records
    g.rec, g.d_count = 16, 8
    assert call(frags=g) == fhv.FHV_ERR_INVALID_ARG  # misaligned counter
    assert call(ws=8) == fhv.FHV_ERR_INVALID_ARG
    assert call(ws_bytes=200) == fhv.FHV_ERR_INVALID_ARG
    assert fhv.fhv_launch_count() >= 0
