"""Batched novel views (fhv_render_views) against one-call-per-view rendering
and the oracle.

Every view of a batch must get exactly the visibility fhv_render_view gives
it (bit-exact keys) and the same colours, for any work decomposition (each
splat mode: one fragment per thread, shared-memory tile, runs, the pixel
election, the per-chunk depth pre-test), for
views in any order and of different sizes, when replayed from a CUDA graph,
and a view with a bad descriptor must be skipped with FHV_DEV_BAD_VIEW.
"""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import batched, fhv  # noqa: E402

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def built():
    ws = []
    for seed, (W, H), d in ((11, (96, 64), 5), (12, (128, 128), 6)):
        sc = scenes.spheres_scene(seed, n_spheres=4, segments=16, rings=8)
        cap = scenes.orbit_camera(sc, W, H)
        ws.append(scenes.Workload(f"s{seed}", sc, cap, d, [], scenes.directional_light((1, 1, 1))[None]))
    sc = scenes.terrain_scene(13, grid=48, n_boxes=6)
    ws.append(scenes.Workload("t13", sc, scenes.orbit_camera(sc, 160, 90), 7, [], scenes.directional_light((1, 1, 1))[None]))
    return ws, batched.build_sources(ws)


def make_views(ws, order):
    per = [[] for _ in ws]
    cams = []
    for k, si in enumerate(order):
        sc = ws[si].scene
        W, H = [(64, 48), (100, 75), (37, 29)][k % 3]
        cams.append((si, scenes.orbit_camera(sc, W, H, orbit_deg=23.0 * k, elevation_deg=10.0 + 7 * k)))
    return cams


def lights():
    return np.stack([scenes.directional_light((1, 1, 1), (0.7, 0.6, 0.5)), scenes.point_light((0.5, 1.5, 0.5), (0.3, 0.3, 0.3))])


class Views(batched.BatchedViews):
    """BatchedViews over an arbitrary (source, camera) list, in that order."""

    def __init__(self, sources, cams, lights_, k):
        super().__init__(sources, [[] for _ in sources], lights_, k)
        view_structs = []
        for si, cam in cams:
            v = fhv.fhv_view()
            v.cam = fhv.camera_struct(cam)
            v.source = si
            vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
            rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
            v.d_vis, v.d_rgba = vis.data_ptr(), rgba.data_ptr()
            self.cams.append(cam)
            self.view_src.append(si)
            self.vis.append(vis)
            self.rgba.append(rgba)
            view_structs.append(v)
        self.n_views = len(view_structs)
        self.view_structs = view_structs
        self.d_views = fhv.device_structs(view_structs)
        self.ws = fhv.workspace(fhv.fhv_batch_workspace_size(self.n_views))


def reference(bv):
    """Each view rendered alone with fhv_render_view."""
    out = []
    ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    for i, cam in enumerate(bv.cams):
        s = bv.sources[bv.view_src[i]]
        vis = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
        rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
        fhv.fhv_render_view(s.records, s.n, None, s.ds, s.ds.albedo, bv.lights, bv.n_lights, cam, bv.k, vis, rgba, ws)
        out.append((vis, rgba))
    torch.cuda.synchronize()
    return out


def assert_same(bv, ref):
    for i in range(bv.n_views):
        assert torch.equal(bv.vis[i], ref[i][0]), f"view {i}: visibility differs"
        assert (bv.rgba[i] - ref[i][1]).abs().max().item() < 1e-6, f"view {i}: colour differs"


@pytest.mark.parametrize("cfg", [(8, 2048, 4096, 0), (1, 32, 256, 1), (3, 96, 512, 2), (32, 1024, 8192, 0),
                                 (8, 2048, 4096, 0, 1), (1, 32, 256, 1, 1), (3, 96, 512, 2, 1), (32, 1024, 8192, 0, 1),
                                 (8, 2048, 4096, 0, 2), (1, 32, 256, 1, 2), (3, 96, 512, 2, 2), (32, 1024, 8192, 0, 2),
                                 (8, 2048, 4096, 0, 3), (3, 96, 512, 2, 3),
                                 (8, 2048, 4096, 0, 4), (1, 32, 256, 1, 4), (3, 96, 512, 2, 4), (32, 1024, 8192, 0, 4),
                                 (8, 2048, 4096, 0, 5), (1, 32, 256, 1, 5), (3, 96, 512, 2, 5), (32, 1024, 8192, 0, 5)])
@pytest.mark.parametrize("k", [1, 2])
def test_batched_equals_single_view(built, cfg, k):
    ws, sources = built
    order = [0, 0, 0, 1, 1, 2, 2, 2, 2, 0, 1, 2, 1]  # runs and interleaved sources
    bv = Views(sources, make_views(ws, order), lights(), k)
    bv.set_config(cfg)
    bv.render()
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(bv.ws) == (fhv.FHV_OK, 0)
    assert_same(bv, reference(bv))


def test_batched_graph_replay_and_repeat(built):
    ws, sources = built
    bv = Views(sources, make_views(ws, [2, 0, 1, 2, 0, 1]), lights(), 1)
    ref = reference(bv)
    bv.capture_graph()
    for _ in range(3):
        for t in bv.vis:
            t.fill_(123)
        bv.replay()
        torch.cuda.synchronize()
        assert_same(bv, ref)


def test_batched_against_oracle(built):
    import oracle

    ws, sources = built
    bv = Views(sources, make_views(ws, [1, 2]), lights(), 1)
    bv.render()
    torch.cuda.synchronize()
    for i, (si, cam) in enumerate(zip(bv.view_src, bv.cams)):
        s = sources[si]
        rec = s.records[: 2 * s.n].cpu().numpy().view(fhv.RECORD_DTYPE)
        vis_o, rgba_o = oracle.render(rec, ws[si].scene, cam, lights(), 1)
        assert (bv.vis[i].cpu().numpy().view(np.uint64) == vis_o).all()
        assert np.abs(bv.rgba[i].cpu().numpy().reshape(-1, 4) - rgba_o).max() < 1e-4


def test_bad_view_is_skipped(built):
    ws, sources = built
    cams = make_views(ws, [0, 1, 2])
    bv = Views(sources, cams, lights(), 1)
    bad = bv.view_structs[1]
    bad.source = 7  # no such source
    bv.d_views = fhv.device_structs(bv.view_structs)
    for t in bv.vis:
        t.fill_(5)
    bv.render()
    torch.cuda.synchronize()
    st, bits = fhv.fhv_read_status(bv.ws)
    assert bits & fhv.FHV_DEV_BAD_VIEW
    assert (bv.vis[1] == 5).all()  # untouched
    ref = reference(bv)
    for i in (0, 2):
        assert torch.equal(bv.vis[i], ref[i][0])


def test_depth_pretest_matches_single_view_under_heavy_overdraw():
    """Splat mode 5 skips (chunk, view) pairs whose fragments cannot win any
    pixel. On a scene seen through many layers (spheres on a heightfield,
    three-axis capture, about 100 fragments per pixel of the small views)
    most chunks are skipped in most views; every view must still equal its
    one-call render bit for bit, and mode 0's batched render."""
    from paper_2211_15460_gb300.pipeline import PofaViews

    sc = scenes.instanced_spheres_heightfield(7, n_spheres=60, grid=256)
    views = [scenes.orbit_camera(sc, 240, 135, orbit_deg=22.5 * i) for i in range(16)] + \
        [scenes.orbit_camera(sc, 97, 61, orbit_deg=11.0, elevation_deg=60.0)]
    w = scenes.Workload("layers", sc, scenes.orbit_camera(sc, 240, 135), 7, views, lights(),
                        normal_pitch=float(sc.cube_side) / 1904)
    p = PofaViews(w)
    p.capture()
    p.compact()
    torch.cuda.synchronize()
    assert p.n > 20 * 240 * 135
    bv = p.views
    ref = reference(bv)
    for cfg in [(16, 2048, 8192, 0, 5), (8, 512, 4096, 0, 5), (3, 96, 512, 2, 5)]:
        bv.set_config(cfg)
        for t in bv.vis:
            t.fill_(7)
        bv.render()
        torch.cuda.synchronize()
        assert fhv.fhv_read_status(bv.ws) == (fhv.FHV_OK, 0)
        assert_same(bv, ref)
    bv.set_config((16, 2048, 8192, 0, 0))
    bv.render()
    torch.cuda.synchronize()
    assert_same(bv, ref)
