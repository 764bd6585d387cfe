"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact on fragment records, list membership, octant occupancy, POFA
bytes and (off, cnt) of every octant, and the per-pixel visible fragment;
shaded colours within 1e-4 absolute. List order inside a slot depends on the
device's atomic order, so lists are compared in canonical form (sorted
(slot, record) pairs) after checking their structure.
"""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes
from _lists import canonical, list_owner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402
from paper_2211_15460_gb300.pipeline import PlainFHV  # noqa: E402

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
RGB_TOL = 1e-4


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def levels_gpu_to_list(arr: np.ndarray, depth: int, upto: int):
    """Per-level views of a padded level array (levels 0..upto)."""
    out = []
    for l in range(upto + 1):
        b = fhv.fhv_level_offset(l)
        out.append(arr[b: b + (1 << (3 * l))])
    return out


def levels_oracle_to_list(orc, arr, upto):
    return [arr[orc.level_base(l): orc.level_base(l) + (1 << (3 * l))] for l in range(upto + 1)]


def gpu_records(t, n):
    return fhv.records_to_numpy(t, n)


def run_ppfl(scene, cam, capacity):
    ds = fhv.DeviceScene(scene)
    head = torch.empty(cam.width * cam.height, dtype=torch.int32, device="cuda")
    fb = fhv.FragBuf(capacity)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_PPFL, scene.n_tri, cam.width, cam.height, 1, 0).workspace_bytes)
    fhv.fhv_capture_ppfl(ds, cam, head, fb, ws)
    st, n = fhv.fhv_get_count(fb)
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    stored = min(n, capacity)
    return n, head.cpu().numpy(), gpu_records(fb.rec, stored), fb.next[:stored].cpu().numpy()


def run_pofl(scene, mode, cam, pitch, depth, capacity):
    ds = fhv.DeviceScene(scene)
    leaf = torch.empty(1 << (3 * depth), dtype=torch.int32, device="cuda")
    levels = torch.empty(max(fhv.fhv_level_offset(depth), 4), dtype=torch.int32, device="cuda")
    fb = fhv.FragBuf(capacity)
    W, H = (cam.width, cam.height) if cam is not None else (1, 1)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, scene.n_tri, W, H, depth, 0).workspace_bytes)
    fhv.fhv_build_pofl(ds, mode, cam, pitch, depth, leaf, levels, fb, ws)
    st, n = fhv.fhv_get_count(fb)
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    stored = min(n, capacity)
    return (n, leaf.cpu().numpy(), levels.cpu().numpy().view(np.uint32), gpu_records(fb.rec, stored),
            fb.next[:stored].cpu().numpy(), fb)


def run_compact(rec_np, depth, n_max=None, via_counter=False):
    n = rec_np.size
    n_max = n if n_max is None else n_max
    src = torch.zeros(max(n_max, 1) * 2, dtype=torch.int64, device="cuda")
    if n:
        src[: 2 * n] = torch.from_numpy(np.ascontiguousarray(rec_np).view(np.int64)).cuda()
    out = torch.zeros_like(src)
    m = fhv.fhv_level_offset(depth + 1)
    off = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, depth, n_max).workspace_bytes)
    d_n = None
    if via_counter:
        d_n = torch.tensor([n, 0], dtype=torch.int64, device="cuda")
    fhv.fhv_compact_pofa(src, n_max if via_counter else n, d_n, depth, out, off, cnt, ws)
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    return gpu_records(out, n), off.cpu().numpy().view(np.uint32), cnt.cpu().numpy().view(np.uint32)


def run_render(rec_np, scene, cam, lights, k):
    n = rec_np.size
    ds = fhv.DeviceScene(scene)
    src = torch.zeros(max(n, 1) * 2, dtype=torch.int64, device="cuda")
    if n:
        src[: 2 * n] = torch.from_numpy(np.ascontiguousarray(rec_np).view(np.int64)).cuda()
    L = torch.from_numpy(np.ascontiguousarray(lights, np.float32).reshape(-1)).cuda()
    vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
    rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
    ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    fhv.fhv_render_view(src, n, None, ds, ds.albedo, L, lights.shape[0], cam, k, vis, rgba, ws)
    return vis.cpu().numpy().view(np.uint64), rgba.cpu().numpy().reshape(-1, 4)


def assert_pofa_equal(orc, rec_in, depth, got_rec, got_off, got_cnt):
    exp, eoff, ecnt = orc.pofa(rec_in, depth)
    assert (got_rec == exp).all(), "POFA bytes differ"
    go, gc = levels_gpu_to_list(got_off, depth, depth), levels_gpu_to_list(got_cnt, depth, depth)
    eo, ec = levels_oracle_to_list(orc, eoff, depth), levels_oracle_to_list(orc, ecnt, depth)
    for l in range(depth + 1):
        assert (gc[l] == ec[l]).all(), f"cnt differs at level {l}"
        assert (go[l] == eo[l]).all(), f"off differs at level {l}"


def assert_lists_equal(head_g, next_g, rec_g, n_g, head_o, next_o, rec_o, n_o):
    assert n_g == n_o
    own_g = list_owner(head_g, next_g, n_g)
    own_o = list_owner(head_o, next_o, n_o)
    assert (canonical(own_g, rec_g) == canonical(own_o, rec_o)).all()


def random_mesh(rng, nt, W, H, zr=1.0, spread=1.0):
    P = rng.uniform(-0.1 * W, 1.1 * W, size=(nt, 1, 2)) + rng.normal(scale=spread * rng.uniform(0.5, 6), size=(nt, 3, 2))
    z = rng.uniform(-zr, zr, size=(nt, 3, 1))
    pos = np.concatenate([P, z], axis=2).reshape(-1, 3)
    nrm = rng.normal(size=pos.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    mat = rng.integers(0, 3, size=nt).astype(np.uint32)
    return scenes.Scene(pos=pos, nrm=nrm, idx=np.arange(3 * nt).reshape(nt, 3), tri_material=mat,
                        albedo=rng.uniform(0.2, 1, size=(3, 3)))


def screen_camera(W, H, zr=4.0):
    return scenes.Camera(origin=(W / 2, H / 2, 0.0), right=(1, 0, 0), up=(0, 1, 0), fwd=(0, 0, -1), pitch=1.0,
                         width=W, height=H, z0=-zr, z1=zr)


# ------------------------------------------------------------------ tests

def test_abi_status_strings():
    assert fhv.status_str(fhv.FHV_OK) == "ok"
    assert fhv.status_str(fhv.FHV_ERR_OVERFLOW) == "fragment buffer overflow"


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_ppfl_random_tiny_meshes(orc, seed):
    rng = np.random.default_rng(100 + seed)
    W, H = int(rng.integers(7, 70)), int(rng.integers(5, 50))
    sc = random_mesh(rng, int(rng.integers(1, 300)), W, H)
    cam = screen_camera(W, H)
    n_o, head_o, rec_o, next_o = orc.ppfl(sc, cam, 1 << 18)
    n_g, head_g, rec_g, next_g = run_ppfl(sc, cam, 1 << 18)
    assert_lists_equal(head_g, next_g, rec_g, n_g, head_o, next_o[:n_o], rec_o[:n_o], n_o)


@pytest.mark.parametrize("seed,mode,depth", [(0, 0, 3), (1, 1, 1), (2, 1, 2), (3, 1, 4), (4, 0, 5), (5, 1, 6),
                                             (6, 2, 3), (7, 2, 5)])
def test_pofl_random_tiny_meshes(orc, seed, mode, depth):
    rng = np.random.default_rng(200 + seed)
    W, H = int(rng.integers(9, 60)), int(rng.integers(9, 60))
    sc = random_mesh(rng, int(rng.integers(1, 200)), W, H)
    cam = screen_camera(W, H)
    pitch = float(rng.uniform(0.3, 1.5)) * (float(sc.cube_side) / 64 if mode == 2 else 1.0)
    n_o, leaf_o, lev_o, rec_o, next_o = orc.pofl(sc, mode, cam, pitch, depth, 1 << 18)
    n_g, leaf_g, lev_g, rec_g, next_g, _ = run_pofl(sc, mode, cam, pitch, depth, 1 << 18)
    assert_lists_equal(leaf_g, next_g, rec_g, n_g, leaf_o, next_o[:n_o], rec_o[:n_o], n_o)
    for a, b in zip(levels_gpu_to_list(lev_g, depth, depth - 1), levels_oracle_to_list(orc, lev_o, depth - 1)):
        assert (a == b).all()


def test_empty_scene(orc):
    sc = scenes.Scene(pos=np.zeros((0, 3)), nrm=np.zeros((0, 3)), idx=np.zeros((0, 3)), tri_material=np.zeros(0),
                      albedo=np.ones((1, 3)))
    cam = screen_camera(16, 16)
    n, head, rec, nxt = run_ppfl(sc, cam, 64)
    assert n == 0 and (head == -1).all()
    n, leaf, lev, rec, nxt, _ = run_pofl(sc, 1, None, 0.5, 3, 64)
    assert n == 0 and (leaf == -1).all() and (lev[: fhv.fhv_level_offset(3)] == 0).all()
    r, off, cnt = run_compact(np.zeros(0, fhv.RECORD_DTYPE), 3)
    for l in range(4):
        b = fhv.fhv_level_offset(l)
        assert (off[b: b + 8 ** l] == 0).all() and (cnt[b: b + 8 ** l] == 0).all()
    vis, rgba = run_render(np.zeros(0, fhv.RECORD_DTYPE), sc, cam, scenes.directional_light((0, 0, 1))[None], 1)
    assert (vis == EMPTY).all() and (rgba == 0).all()


@pytest.mark.parametrize("cap_delta", [-1000000, -5, 0])
def test_ppfl_overflow_keeps_lists_consistent(orc, cap_delta):
    w = scenes.workload_spheres_256()
    n_o, head_o, rec_o, next_o = orc.ppfl(w.scene, w.capture, 1 << 16)
    cap = max(0, n_o + cap_delta)
    n_g, head_g, rec_g, next_g = run_ppfl(w.scene, w.capture, cap)
    assert n_g == n_o  # the counter keeps counting past capacity
    stored = min(n_g, cap)
    owner = list_owner(head_g, next_g, stored)
    # every stored record is one of the oracle's fragments of that pixel
    exp = set(zip(list_owner(head_o, next_o[:n_o], n_o).tolist(), rec_o[:n_o].tolist()))
    got = list(zip(owner.tolist(), rec_g.tolist()))
    assert all(x in exp for x in got)
    assert len(set(got)) == len(got) or stored == 0


@pytest.mark.parametrize("depth,n", [(1, 9000), (2, 20000), (3, 4097), (4, 100003), (5, 77777), (6, 1), (7, 30000),
                                     (8, 50000), (9, 2048), (3, 0)])
def test_compact_random_records(orc, depth, n):
    rng = np.random.default_rng(300 + depth + n)
    rec = np.zeros(n, fhv.RECORD_DTYPE)
    # clustered keys: a few hot octants, duplicates, and uniform keys
    k = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    hot = rng.integers(0, 1 << 63, size=8, dtype=np.uint64)
    sel = rng.random(n) < 0.5
    k[sel] = (hot[rng.integers(0, 8, size=sel.sum())] & ~np.uint64(0xFFFF)) | (k[sel] & np.uint64(0xFF))
    rec["key"] = k
    rec["tri"] = rng.integers(0, 50, size=n)
    rec["nrm"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    if n > 10:
        rec[: n // 10] = rec[n // 10: 2 * (n // 10)]  # bit-identical duplicates
    got, off, cnt = run_compact(rec, depth, n_max=n + 17, via_counter=True)
    assert_pofa_equal(orc, rec, depth, got, off, cnt)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_render_footprints(orc, k):
    w = scenes.workload_spheres_256()
    rec, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    pofa = orc.pofa_sort(rec)
    for cam in (w.views[0], w.capture):
        vis_o, rgba_o = orc.render(pofa, w.scene, cam, w.lights, k)
        vis_g, rgba_g = run_render(pofa, w.scene, cam, w.lights, k)
        assert (vis_g == vis_o).all()
        assert np.abs(rgba_g - rgba_o).max() < RGB_TOL


def test_spheres_256_full_path(orc):
    """8 UV-spheres, 256^2, depth 6: every stage of the plain path."""
    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    # PPFL (1-Pass/View)
    n_o, head_o, rec_o, next_o = orc.ppfl(w.scene, w.capture, 1 << 18)
    n_g = fhv.fhv_get_count(p.ppfl)[1]
    assert_lists_equal(p.head.cpu().numpy(), p.ppfl.next[:n_g].cpu().numpy(), gpu_records(p.ppfl.rec, n_g), n_g,
                       head_o, next_o[:n_o], rec_o[:n_o], n_o)
    # POFL (1-Pass/Normal)
    d = w.depth
    n_o, leaf_o, lev_o, prec_o, pnext_o = orc.pofl(w.scene, orc.NORMAL, None, w.normal_pitch, d, 1 << 18)
    n_g = fhv.fhv_get_count(p.pofl)[1]
    assert_lists_equal(p.leaf_head.cpu().numpy(), p.pofl.next[:n_g].cpu().numpy(), gpu_records(p.pofl.rec, n_g), n_g,
                       leaf_o, pnext_o[:n_o], prec_o[:n_o], n_o)
    lev_g = p.levels.cpu().numpy().view(np.uint32)
    for a, b in zip(levels_gpu_to_list(lev_g, d, d - 1), levels_oracle_to_list(orc, lev_o, d - 1)):
        assert (a == b).all()
    # POFA
    assert_pofa_equal(orc, prec_o[:n_o], d, gpu_records(p.pofa, n_g), p.off.cpu().numpy().view(np.uint32),
                      p.cnt.cpu().numpy().view(np.uint32))
    # novel view
    pofa_o = orc.pofa_sort(prec_o[:n_o])
    for v, cam in enumerate(w.views):
        vis_o, rgba_o = orc.render(pofa_o, w.scene, cam, w.lights, w.footprint_k)
        assert (p.vis[v].cpu().numpy().view(np.uint64) == vis_o).all()
        assert np.abs(p.rgba[v].cpu().numpy().reshape(-1, 4) - rgba_o).max() < RGB_TOL
    for ws in (p.ws_capture, p.ws_ppfl, p.ws_compact, *p.ws_views):
        assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)


def test_terrain_1080p_depth10_full_size(orc):
    """1,002,098 triangles at 1920x1080, depth 10, three views, as the
    benchmark runs it. Records, lists and visibility are compared in full;
    the dense 1.2e9-octant index is compared on every occupied octant, on
    random octants, and by invariants that hold at any size."""
    w = scenes.workload_terrain_1080p()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    d = w.depth
    # PPFL in full
    n_o, head_o, rec_o, next_o = orc.ppfl(w.scene, w.capture, 1 << 22)
    n_g = fhv.fhv_get_count(p.ppfl)[1]
    assert_lists_equal(p.head.cpu().numpy(), p.ppfl.next[:n_g].cpu().numpy(), gpu_records(p.ppfl.rec, n_g), n_g,
                       head_o, next_o[:n_o], rec_o[:n_o], n_o)
    # POFL: records and list membership; heads gathered at occupied leaves
    frag_o, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    n_g = fhv.fhv_get_count(p.pofl)[1]
    assert n_g == frag_o.size
    rec_g = gpu_records(p.pofl.rec, n_g)
    sh = np.uint64(63 - 3 * d)
    leaves = np.unique(frag_o["key"] >> sh)
    heads = p.leaf_head[torch.from_numpy(leaves.astype(np.int64)).cuda()].cpu().numpy()
    assert int((p.leaf_head != -1).sum().item()) == leaves.size
    owner = list_owner(heads, p.pofl.next[:n_g].cpu().numpy(), n_g)
    assert (leaves[owner] == (rec_g["key"] >> sh)).all()
    a = np.sort(rec_g, order=["key", "tri", "nrm"])
    b = np.sort(frag_o, order=["key", "tri", "nrm"])
    assert (a == b).all()
    # occupancy levels from the oracle's fragments
    lev_g = p.levels.cpu().numpy().view(np.uint32)
    for l in range(d):
        child = np.unique(frag_o["key"] >> np.uint64(63 - 3 * (l + 1)))
        exp = np.zeros(1 << (3 * l), np.uint32)
        np.bitwise_or.at(exp, (child >> np.uint64(3)).astype(np.int64), (1 << (child & np.uint64(7))).astype(np.uint32))
        base = fhv.fhv_level_offset(l)
        assert (lev_g[base: base + exp.size] == exp).all(), l
    # POFA bytes in full
    pofa_o = orc.pofa_sort(frag_o)
    assert (gpu_records(p.pofa, n_g) == pofa_o).all()
    # off/cnt: levels <= 7 in full, level 8..10 at occupied octants, their
    # neighbours and random octants; plus the scan invariant on every level
    for l in range(d + 1):
        base = fhv.fhv_level_offset(l)
        m = 1 << (3 * l)
        if l <= 7:
            sel = np.arange(m, dtype=np.int64)
        else:
            occ = np.unique((pofa_o["key"] >> np.uint64(63 - 3 * l)).astype(np.int64))
            rnd = np.random.default_rng(l).integers(0, m, size=200000)
            sel = np.unique(np.concatenate([occ, np.clip(occ + 1, 0, m - 1), np.clip(occ - 1, 0, m - 1), rnd, [0, m - 1]]))
        idx = torch.from_numpy(sel + base).cuda()
        go = p.off[idx].cpu().numpy().view(np.uint32)
        gc = p.cnt[idx].cpu().numpy().view(np.uint32)
        pre = (pofa_o["key"] >> np.uint64(63 - 3 * l)).astype(np.int64) if l else np.zeros(n_g, np.int64)
        eo = np.searchsorted(pre, sel, side="left")
        ec = np.searchsorted(pre, sel, side="right") - eo
        assert (go == eo).all() and (gc == ec).all(), l
        # invariant on the whole level, on the device: off[o] + cnt[o] == off[o+1], sum cnt == n
        lo = p.off[base: base + m].to(torch.int64)
        lc = p.cnt[base: base + m].to(torch.int64)
        assert int(lc.sum().item()) == n_g
        assert bool(((lo[1:] - lo[:-1]) == lc[:-1]).all().item())
        del lo, lc
    # three novel views
    for v, cam in enumerate(w.views):
        vis_o, rgba_o = orc.render(pofa_o, w.scene, cam, w.lights, w.footprint_k)
        assert (p.vis[v].cpu().numpy().view(np.uint64) == vis_o).all()
        assert np.abs(p.rgba[v].cpu().numpy().reshape(-1, 4) - rgba_o).max() < RGB_TOL
    for ws in (p.ws_capture, p.ws_ppfl, p.ws_compact, *p.ws_views):
        assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)


def test_axis3_spheres_256(orc):
    """3-Pass/1-Way POFL of the 8-sphere scene against the oracle."""
    w = scenes.workload_spheres_256()
    d = w.depth
    n_o, leaf_o, lev_o, rec_o, next_o = orc.pofl(w.scene, orc.AXIS3, None, w.normal_pitch, d, 1 << 18)
    n_g, leaf_g, lev_g, rec_g, next_g, _ = run_pofl(w.scene, fhv.FHV_CAPTURE_AXIS3, None, w.normal_pitch, d, 1 << 18)
    assert_lists_equal(leaf_g, next_g, rec_g, n_g, leaf_o, next_o[:n_o], rec_o[:n_o], n_o)
    for a, b in zip(levels_gpu_to_list(lev_g, d, d - 1), levels_oracle_to_list(orc, lev_o, d - 1)):
        assert (a == b).all()
