"""The POFA rasterised straight into octant ranges (fhv_build_pofa_direct:
Section 3.2's creation by counting per octant, scanning and rasterising
again, without lists) against the oracle.

* Tiny random meshes in every capture mode and at depths with and without
  the two-level scan: records byte for byte and (off, cnt) of every octant
  of every level equal the oracle's POFA of the oracle's fragments.
* The 256^2 sphere workload (depth 6): the same, and the same bytes as the
  list build followed by the compaction.
* Capacity: the count is the full count past a too-small capacity, the
  index is complete and no record is written; capacity 0 with no output.
* Empty scene.
* The 1080p terrain workload at depth 10: the oracle's fragment count, and
  the same POFA bytes and dense index as the list build + compaction.
"""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402
from paper_2211_15460_gb300.pipeline import PlainFHV  # noqa: E402

FILL = -7  # every index entry must be written


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def run_direct(scene, mode, cam, pitch, depth, capacity, ds=None):
    ds = ds or fhv.DeviceScene(scene)
    m = fhv.fhv_level_offset(depth + 1)
    off = torch.full((m,), FILL, dtype=torch.int32, device="cuda")
    cnt = torch.full((m,), FILL, dtype=torch.int32, device="cuda")
    pofa = torch.full((capacity * 2,), FILL, dtype=torch.int64, device="cuda") if capacity else None
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_DIRECT, scene.n_tri, 1, 1, depth,
                                           capacity).workspace_bytes)
    fhv.fhv_build_pofa_direct(ds, mode, cam, pitch, depth, pofa, capacity, count, off, cnt, ws)
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    n = int(count[0].item())
    return n, pofa, off, cnt


def assert_index_equal(orc, depth, off, cnt, eoff, ecnt):
    go, gc = off.cpu().numpy().view(np.uint32), cnt.cpu().numpy().view(np.uint32)
    for lev in range(depth + 1):
        b, e = fhv.fhv_level_offset(lev), orc.level_base(lev)
        size = 1 << (3 * lev)
        assert (gc[b: b + size] == ecnt[e: e + size]).all(), f"cnt differs at level {lev}"
        assert (go[b: b + size] == eoff[e: e + size]).all(), f"off differs at level {lev}"


def check_against_oracle(orc, sc, mode, cam, pitch, depth):
    frag_o = orc.fragments(sc, mode, cam, pitch)[0]
    exp, eoff, ecnt = orc.pofa(frag_o, depth)
    n, pofa, off, cnt = run_direct(sc, mode, cam, pitch, depth, max(frag_o.size, 1))
    assert n == frag_o.size
    assert (fhv.records_to_numpy(pofa, n) == exp).all(), "POFA bytes differ"
    assert_index_equal(orc, depth, off, cnt, eoff, ecnt)
    return n


def same_index(a, b):
    """Equal on every octant of every level (entries 1..3 pad level 1 to 16 bytes and are never written)."""
    lo = fhv.fhv_level_offset(1)
    return torch.equal(a[:1], b[:1]) and torch.equal(a[lo:], b[lo:])


def random_mesh(rng, nt, W, H):
    P = rng.uniform(-0.1 * W, 1.1 * W, size=(nt, 1, 2)) + rng.normal(scale=rng.uniform(0.5, 6), size=(nt, 3, 2))
    z = rng.uniform(-1.0, 1.0, size=(nt, 3, 1))
    pos = np.concatenate([P, z], axis=2).reshape(-1, 3)
    nrm = rng.normal(size=pos.shape)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return scenes.Scene(pos=pos, nrm=nrm, idx=np.arange(3 * nt).reshape(nt, 3),
                        tri_material=rng.integers(0, 3, size=nt).astype(np.uint32),
                        albedo=rng.uniform(0.2, 1, size=(3, 3)))


@pytest.mark.parametrize("seed,mode,depth", [(0, 0, 3), (1, 1, 1), (2, 1, 2), (3, 1, 4), (4, 0, 5), (5, 1, 6),
                                             (6, 2, 3), (7, 2, 5), (8, 1, 7)])
def test_direct_random_tiny_meshes(orc, seed, mode, depth):
    rng = np.random.default_rng(500 + seed)
    W, H = int(rng.integers(9, 60)), int(rng.integers(9, 60))
    sc = random_mesh(rng, int(rng.integers(1, 200)), W, H)
    cam = scenes.Camera(origin=(W / 2, H / 2, 0.0), right=(1, 0, 0), up=(0, 1, 0), fwd=(0, 0, -1), pitch=1.0,
                        width=W, height=H, z0=-4.0, z1=4.0)
    pitch = float(rng.uniform(0.3, 1.5)) * (float(sc.cube_side) / 64 if mode == 2 else 1.0)
    check_against_oracle(orc, sc, mode, cam, pitch, depth)


def test_direct_spheres_256(orc):
    w = scenes.workload_spheres_256()
    n = check_against_oracle(orc, w.scene, orc.NORMAL, None, w.normal_pitch, w.depth)
    p = PlainFHV(w)
    p.step()
    _, pofa, off, cnt = run_direct(w.scene, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, w.depth, n, ds=p.scene)
    assert fhv.fhv_get_count(p.pofl)[1] == n
    assert torch.equal(pofa[: 2 * n], p.pofa[: 2 * n])
    assert same_index(off, p.off) and same_index(cnt, p.cnt)


@pytest.mark.parametrize("mode", [1, 2])
def test_direct_capacity(orc, mode):
    w = scenes.workload_spheres_256()
    pitch = w.normal_pitch
    frag_o = orc.fragments(w.scene, mode, None, pitch)[0]
    _, eoff, ecnt = orc.pofa(frag_o, w.depth)
    for cap in (frag_o.size - 5, 1, 0):
        n, pofa, off, cnt = run_direct(w.scene, mode, None, pitch, w.depth, cap)
        assert n == frag_o.size, cap
        assert_index_equal(orc, w.depth, off, cnt, eoff, ecnt)
        if pofa is not None:
            assert bool((pofa == FILL).all().item()), "records written past the capacity"
    n, pofa, off, cnt = run_direct(w.scene, mode, None, pitch, w.depth, frag_o.size)  # exactly enough
    assert n == frag_o.size
    assert (fhv.records_to_numpy(pofa, n) == orc.pofa_sort(frag_o)).all()


def test_direct_empty_scene():
    sc = scenes.Scene(pos=np.zeros((0, 3)), nrm=np.zeros((0, 3)), idx=np.zeros((0, 3)), tri_material=np.zeros(0),
                      albedo=np.ones((1, 3)))
    for depth in (3, 6):
        n, pofa, off, cnt = run_direct(sc, fhv.FHV_CAPTURE_NORMAL, None, 0.5, depth, 16)
        assert n == 0
        zero = torch.zeros_like(off)
        assert same_index(off, zero) and same_index(cnt, zero)


def test_direct_terrain_1080p_depth10(orc):
    """1,002,098 triangles, tangent-space capture at depth 10 (1.2e9 octants)."""
    w = scenes.workload_terrain_1080p()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    assert n == orc.fragment_count(w.scene, orc.NORMAL, None, w.normal_pitch)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_DIRECT, w.scene.n_tri, 1, 1, w.depth,
                                           n).workspace_bytes)
    m = fhv.fhv_level_offset(w.depth + 1)
    off = torch.empty(m, dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(off)
    pofa = torch.empty(2 * n, dtype=torch.int64, device="cuda")
    count = torch.zeros(2, dtype=torch.int64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for _ in range(4):
        ev[0].record()
        fhv.fhv_build_pofa_direct(p.scene, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, w.depth, pofa, n, count, off,
                                  cnt, ws)
        ev[1].record()
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    assert int(count[0].item()) == n
    assert torch.equal(pofa, p.pofa[: 2 * n])
    assert same_index(off, p.off) and same_index(cnt, p.cnt)
    print(f"\ndirect POFA build, {n} fragments at depth 10: {min(times[1:]):.3f} ms "
          f"({n / min(times[1:]) / 1e6:.3f} Gfrag/s)")


@pytest.mark.parametrize("mode", [1, 2])
def test_direct_slice_keeps_scene_triangle_ids(orc, mode):
    """A slice of the scene's triangles (fhv_scene.tri_base) gives the
    oracle's fragments of those triangles, numbered as in the whole scene;
    the list build of the same slice stores the same records."""
    w = scenes.workload_spheres_256()
    sc, pitch, d = w.scene, w.normal_pitch, w.depth
    ds = fhv.DeviceScene(sc)
    for t0, t1 in ((0, 3001), (3001, sc.n_tri), (5000, 5000)):
        sub = scenes.Scene(pos=sc.pos, nrm=sc.nrm, idx=sc.idx[t0:t1], tri_material=sc.tri_material[t0:t1],
                           albedo=sc.albedo, cube_min=sc.cube_min, cube_side=sc.cube_side)
        frag_o = orc.fragments(sub, mode, None, pitch)[0]
        frag_o["tri"] += np.uint32(t0)
        exp, eoff, ecnt = orc.pofa(frag_o, d)
        n, pofa, off, cnt = run_direct(sub, mode, None, pitch, d, max(frag_o.size, 1), ds=ds.slice(t0, t1))
        assert n == frag_o.size
        assert (fhv.records_to_numpy(pofa, n) == exp).all()
        assert_index_equal(orc, d, off, cnt, eoff, ecnt)
        if n:
            leaf = torch.empty(1 << (3 * d), dtype=torch.int32, device="cuda")
            levels = torch.empty(fhv.fhv_level_offset(d), dtype=torch.int32, device="cuda")
            fb = fhv.FragBuf(n)
            ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, t1 - t0, 1, 1, d, 0).workspace_bytes)
            fhv.fhv_build_pofl(ds.slice(t0, t1), mode, None, pitch, d, leaf, levels, fb, ws)
            assert fhv.fhv_get_count(fb) == (fhv.FHV_OK, n)
            assert (np.sort(fhv.records_to_numpy(fb.rec, n), order=["key", "tri", "nrm"]) == exp).all()
