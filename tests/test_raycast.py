"""Ray casting through a POFA (fhv_raycast_pofa) against the oracle's
per-ray brute force over all fragments, and opaque ray casting against the
1 x 1 splat (same visibility by construction: bit-equal keys, and colours of
the same record).

Inputs of the oracle come from the oracle (fragments -> sorted POFA); the
GPU side runs its own pipeline or compacts the same records on the device.
Visibility keys are compared bit for bit, colours within 1e-4 absolute, and
with an early-out threshold t_stop within t_stop times the largest colour.
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

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
RGB_TOL = 1e-4


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


class GpuPofa:
    """A POFA on the device: records, off, cnt (from the plain pipeline or
    compacted here from host records)."""

    def __init__(self, pofa, n, off, cnt, depth):
        self.pofa, self.n, self.off, self.cnt, self.depth = pofa, n, off, cnt, depth

    @staticmethod
    def from_records(rec_np, depth):
        n = rec_np.size
        src = torch.zeros(max(n, 1) * 2, dtype=torch.int64, device="cuda")
        if n:
            src[: 2 * n] = torch.from_numpy(np.ascontiguousarray(rec_np).view(np.int64)).cuda()
        out = torch.zeros_like(src)
        m = fhv.fhv_level_offset(depth + 1)
        off = torch.empty(m, dtype=torch.int32, device="cuda")
        cnt = torch.empty(m, dtype=torch.int32, device="cuda")
        ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, depth, max(n, 1)).workspace_bytes)
        fhv.fhv_compact_pofa(src, n, None, depth, out, off, cnt, ws)
        assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
        return GpuPofa(out, n, off, cnt, depth)

    @staticmethod
    def from_pipeline(p: PlainFHV):
        return GpuPofa(p.pofa, fhv.fhv_get_count(p.pofl)[1], p.off, p.cnt, p.w.depth)


def raycast(gp: GpuPofa, scene, cam, lights, alpha=None, t_stop=0.0, ds=None, ws_bytes=None):
    ds = ds or fhv.DeviceScene(scene)
    L = torch.from_numpy(np.ascontiguousarray(lights, np.float32).reshape(-1)).cuda()
    al = None if alpha is None else torch.from_numpy(np.ascontiguousarray(alpha, np.float32)).cuda()
    vis = torch.full((cam.width * cam.height,), 5, dtype=torch.int64, device="cuda")
    rgba = torch.full((cam.width * cam.height * 4,), 7.0, dtype=torch.float32, device="cuda")
    ws = fhv.workspace(fhv.FHV_RAYCAST_WS_BYTES if ws_bytes is None else ws_bytes)
    fhv.fhv_raycast_pofa(gp.pofa, gp.n, gp.off, gp.cnt, gp.depth, ds, ds.albedo, al, t_stop, L, L.numel() // 8, cam,
                         vis, rgba, ws)
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    return vis.cpu().numpy().view(np.uint64), rgba.cpu().numpy().reshape(-1, 4)


def splat1(gp: GpuPofa, scene, cam, lights):
    ds = fhv.DeviceScene(scene)
    L = torch.from_numpy(np.ascontiguousarray(lights, np.float32).reshape(-1)).cuda()
    vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
    rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
    ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    fhv.fhv_render_view(gp.pofa, gp.n, None, ds, ds.albedo, L, L.numel() // 8, cam, 1, vis, rgba, ws)
    torch.cuda.synchronize()
    return vis.cpu().numpy().view(np.uint64), rgba.cpu().numpy().reshape(-1, 4)


def material_alpha(scene, seed, lo=0.15, hi=0.9):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, scene.albedo.shape[0]).astype(np.float32)


def max_colour(scene, lights):
    return float(scene.albedo.max()) * float(np.asarray(lights)[:, 4:7].max(axis=1).sum())


def check(orc, gp, scene, pofa_o, cam, lights, alpha=None, t_stop=0.0, ws_bytes=None):
    vis_g, rgba_g = raycast(gp, scene, cam, lights, alpha, t_stop, ws_bytes=ws_bytes)
    vis_o, rgba_o = orc.raycast(pofa_o, scene, cam, lights, alpha)
    assert (vis_g == vis_o).all()
    tol = RGB_TOL + t_stop * max(1.0, max_colour(scene, lights))
    assert np.abs(rgba_g - rgba_o).max() <= tol
    return vis_g, rgba_g, vis_o, rgba_o


# ------------------------------------------------------------------ small scenes

@pytest.fixture(scope="module")
def spheres(orc):
    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.build()
    torch.cuda.synchronize()
    frag_o, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    return w, GpuPofa.from_pipeline(p), orc.pofa_sort(frag_o), p


def spheres_cams(w):
    sc = w.scene
    return [w.capture, w.views[0], scenes.orbit_camera(sc, 200, 150, orbit_deg=123.0, elevation_deg=-40.0),
            scenes.orbit_camera(sc, 97, 61, elevation_deg=89.0), scenes.orbit_camera(sc, 64, 64, elevation_deg=0.0)]


@pytest.mark.parametrize("ci", range(5))
def test_opaque_equals_splat_and_oracle(orc, spheres, ci):
    w, gp, pofa_o, _ = spheres
    cam = spheres_cams(w)[ci]
    vis_g, rgba_g, vis_o, _ = check(orc, gp, w.scene, pofa_o, cam, w.lights)
    vis_s, rgba_s = splat1(gp, w.scene, cam, w.lights)
    assert (vis_g == vis_s).all()
    assert np.abs(rgba_g - rgba_s).max() <= 1e-6  # same record; shading differs only in FMA contraction
    assert (vis_g != EMPTY).sum() > 0.05 * vis_g.size


@pytest.mark.parametrize("ci", range(5))
def test_transparent_against_oracle(orc, spheres, ci):
    w, gp, pofa_o, _ = spheres
    cam = spheres_cams(w)[ci]
    alpha = material_alpha(w.scene, ci)
    vis_g, rgba_g, _, rgba_o = check(orc, gp, w.scene, pofa_o, cam, w.lights, alpha)
    covered = vis_g != EMPTY
    assert (rgba_g[~covered] == 0).all()
    assert (rgba_o[covered, 3] < 1.0).any()  # really translucent


@pytest.mark.parametrize("t_stop", [0.02, 0.25])
def test_early_out_within_bound(orc, spheres, t_stop):
    w, gp, pofa_o, _ = spheres
    cam = w.views[0]
    alpha = material_alpha(w.scene, 7, 0.3, 0.95)
    check(orc, gp, w.scene, pofa_o, cam, w.lights, alpha, t_stop)


def test_opaque_materials_stop_transparent_rays(orc, spheres):
    """Alpha 1 everywhere: R/T gives R's picture (T reaches 0 at the first
    fragment)."""
    w, gp, pofa_o, _ = spheres
    cam = w.views[0]
    a1 = np.ones(w.scene.albedo.shape[0], np.float32)
    vis_t, rgba_t = raycast(gp, w.scene, cam, w.lights, a1)
    vis_r, rgba_r = raycast(gp, w.scene, cam, w.lights, None)
    assert (vis_t == vis_r).all()
    assert np.abs(rgba_t - rgba_r).max() <= 1e-6


def stacked_sheets(n_sheets=14, size=8.0, gap=0.37, shift=0.23):
    """Horizontal square sheets stacked along y, each shifted a little in x and
    z, four materials: many fragments per ray (more than the ray buffer)."""
    pos, tris, mat = [], [], []
    for i in range(n_sheets):
        y = i * gap
        x0, z0 = i * shift, -i * shift * 0.5
        b = len(pos)
        pos += [(x0, y, z0), (x0, y, z0 + size), (x0 + size, y, z0 + size), (x0 + size, y, z0)]
        tris += [(b, b + 1, b + 2), (b, b + 2, b + 3)]
        mat += [i % 4, i % 4]
    albedo = np.array([(0.9, 0.2, 0.1), (0.1, 0.8, 0.3), (0.2, 0.3, 0.9), (0.7, 0.7, 0.2)], np.float32)
    return scenes.Scene(pos=np.array(pos), nrm=np.tile([0.0, 1.0, 0.0], (len(pos), 1)), idx=np.array(tris),
                        tri_material=np.array(mat), albedo=albedo)


# workspace sizes: no overflow slab (tiles with a large frontier take the
# per-pixel traversal), one slab (the others queue behind it or fall back),
# all 64 slabs
@pytest.mark.parametrize("ws_bytes", [256, 256 + 262144, None])
@pytest.mark.parametrize("depth", [3, 7])
def test_deep_rays_need_several_passes(orc, depth, ws_bytes):
    sc = stacked_sheets()
    pitch = 0.2
    frag_o, _, _ = orc.fragments(sc, orc.NORMAL, None, pitch)
    pofa_o = orc.pofa_sort(frag_o)
    gp = GpuPofa.from_records(frag_o, depth)
    lights = np.stack([scenes.directional_light((0.3, 1.0, 0.2), (0.8, 0.8, 0.8)),
                       scenes.point_light((4.0, 9.0, 4.0), (0.3, 0.3, 0.3))])
    alpha = np.array([0.08, 0.12, 0.05, 0.1], np.float32)
    cams = [scenes.orbit_camera(sc, 64, 48, elevation_deg=75.0, orbit_deg=17.0),
            scenes.orbit_camera(sc, 40, 40, elevation_deg=90.0 - 1e-3)]
    for cam in cams:
        vis_g, rgba_g, vis_o, rgba_o = check(orc, gp, sc, pofa_o, cam, lights, alpha, ws_bytes=ws_bytes)
        vis_r, _ = raycast(gp, sc, cam, lights, None, ws_bytes=ws_bytes)
        assert (vis_g == vis_r).all()
        # with every alpha <= 0.12, eight fragments give an opacity of at most
        # 1 - 0.88^8 < 0.65: these rays hold more than the 8-entry buffer
        assert (rgba_o[:, 3] > 0.65).sum() > 100


def fallback_tiles(ws):
    """Tiles cast one pixel at a time (a counter in the workspace header,
    bytes 48..51)."""
    return int(ws[48:52].view(torch.int32).item())


def test_frontier_overflow_paths(orc):
    """A deep octree over stacked sheets makes some tiles' frontier outgrow
    shared memory: with no slab they fall back to per-pixel traversal, with
    slabs they stay breadth-first; both give the oracle's image."""
    sc = stacked_sheets()
    frag_o, _, _ = orc.fragments(sc, orc.NORMAL, None, 0.2)
    pofa_o = orc.pofa_sort(frag_o)
    gp = GpuPofa.from_records(frag_o, 7)
    lights = scenes.directional_light((0.3, 1.0, 0.2))[None]
    alpha = np.array([0.08, 0.12, 0.05, 0.1], np.float32)
    cam = scenes.orbit_camera(sc, 64, 48, elevation_deg=75.0, orbit_deg=17.0)
    vis_o, rgba_o = orc.raycast(pofa_o, sc, cam, lights, alpha)
    ds = fhv.DeviceScene(sc)
    L = torch.from_numpy(lights.reshape(-1)).cuda()
    al = torch.from_numpy(alpha).cuda()
    counts = {}
    for wsb in (256, fhv.FHV_RAYCAST_WS_BYTES):
        vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
        rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
        ws = fhv.workspace(wsb)
        fhv.fhv_raycast_pofa(gp.pofa, gp.n, gp.off, gp.cnt, 7, ds, ds.albedo, al, 0.0, L, 1, cam, vis, rgba, ws)
        torch.cuda.synchronize()
        assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
        assert (vis.cpu().numpy().view(np.uint64) == vis_o).all()
        assert np.abs(rgba.cpu().numpy().reshape(-1, 4) - rgba_o).max() < RGB_TOL
        counts[wsb] = fallback_tiles(ws)
    assert counts[256] > 0
    assert counts[fhv.FHV_RAYCAST_WS_BYTES] == 0


@pytest.mark.parametrize("depth,n", [(1, 3000), (2, 20000), (5, 50000), (8, 40000)])
def test_random_records(orc, depth, n):
    """Records at random positions in the cube (any depth): R equals the
    splat, R/T equals the oracle."""
    rng = np.random.default_rng(depth * 7 + n)
    sc = scenes.spheres_scene(3, n_spheres=2, segments=8, rings=4)
    rec = np.zeros(n, fhv.RECORD_DTYPE)
    rec["key"] = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    rec["tri"] = rng.integers(0, sc.n_tri, size=n).astype(np.uint32)
    rec["nrm"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    pofa_o = orc.pofa_sort(rec)
    gp = GpuPofa.from_records(rec, depth)
    lights = scenes.directional_light((1.0, 2.0, 0.5))[None]
    cam = scenes.orbit_camera(sc, 80, 60, orbit_deg=41.0, elevation_deg=23.0)
    vis_g, rgba_g, _, _ = check(orc, gp, sc, pofa_o, cam, lights)
    vis_s, rgba_s = splat1(gp, sc, cam, lights)
    assert (vis_g == vis_s).all() and np.abs(rgba_g - rgba_s).max() <= 1e-6
    check(orc, gp, sc, pofa_o, cam, lights, material_alpha(sc, depth))


def test_edge_cases(orc, spheres):
    w, gp, pofa_o, _ = spheres
    sc = w.scene
    # empty POFA: every pixel empty
    empty = GpuPofa.from_records(np.zeros(0, fhv.RECORD_DTYPE), 4)
    vis, rgba = raycast(empty, sc, w.views[0], w.lights, material_alpha(sc, 1))
    assert (vis == EMPTY).all() and (rgba == 0).all()
    # a 1 x 1 view, and a view that looks past the cube
    cam1 = scenes.orbit_camera(sc, 1, 1)
    check(orc, gp, sc, pofa_o, cam1, w.lights)
    far = scenes.orbit_camera(sc, 32, 32)
    far.origin = far.origin + 10.0 * float(sc.cube_side) * far.right
    vis, rgba = raycast(gp, sc, far, w.lights)
    assert (vis == EMPTY).all() and (rgba == 0).all()


# ------------------------------------------------------------------ full size

def test_terrain_1080p_depth10_full_size(orc):
    """The benchmark's workload: 1,002,098 triangles, depth 10, 1920x1080
    views; every pixel against the oracle, R and R/T."""
    w = scenes.workload_terrain_1080p()
    p = PlainFHV(w)
    p.build()
    torch.cuda.synchronize()
    gp = GpuPofa.from_pipeline(p)
    frag_o, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    assert gp.n == frag_o.size
    pofa_o = orc.pofa_sort(frag_o)
    del frag_o
    ds = fhv.DeviceScene(w.scene)
    alpha = material_alpha(w.scene, 11, 0.3, 0.8)
    for v, cam in enumerate(w.views[:2]):
        vis_g, rgba_g = raycast(gp, w.scene, cam, w.lights, None, ds=ds)
        vis_o, rgba_o = orc.raycast(pofa_o, w.scene, cam, w.lights, None)
        assert (vis_g == vis_o).all()
        assert np.abs(rgba_g - rgba_o).max() < RGB_TOL
        vis_g, rgba_g = raycast(gp, w.scene, cam, w.lights, alpha, ds=ds)
        vis_o, rgba_o = orc.raycast(pofa_o, w.scene, cam, w.lights, alpha)
        assert (vis_g == vis_o).all()
        assert np.abs(rgba_g - rgba_o).max() < RGB_TOL
