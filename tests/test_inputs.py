"""The seeded synthetic inputs (paper_2211_15460_gb300.scenes) against their
stated recipe: the splitmix64 stream against its published test vector,
triangle counts of every workload from their closed forms, determinism per
seed, the quantisation cube, the orbit cameras and the lights."""
import math

import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes


def test_splitmix64_published_vector():
    # splitmix64 from state 0 (the generator of Steele, Lea and Flood; its
    # first outputs are the usual check values of implementations)
    got = [int(x) for x in scenes.Rng(0).u64(5)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                   0x1B39896A51A8749B]
    r = scenes.Rng(0)
    a = r.u64(2)
    b = r.u64(3)  # consecutive calls continue the stream
    assert [int(x) for x in np.concatenate([a, b])] == got


def test_uniform_uses_top_24_bits():
    raw = scenes.Rng(9).u64(1000)
    u = scenes.Rng(9).uniform(1000, 2.0, 5.0)
    assert np.array_equal(u, 2.0 + 3.0 * (raw >> np.uint64(40)).astype(np.float64) / 2 ** 24)
    assert (u >= 2.0).all() and (u < 5.0).all()


def _uv_sphere_tris(segments, rings):
    return segments * rings * 2 - 2 * segments  # the two pole rows are fans


def test_workload_triangle_counts():
    w = scenes.workload_spheres_256()
    assert w.scene.n_tri == 8 * _uv_sphere_tris(32, 16) == 7680
    assert w.depth == 6 and (w.capture.width, w.capture.height) == (256, 256) and len(w.views) == 1
    t = scenes.workload_terrain_1080p()
    assert t.scene.n_tri == 707 * 707 * 2 + 200 * 12 == 1002098
    assert t.depth == 10 and (t.capture.width, t.capture.height) == (1920, 1080) and len(t.views) == 3
    assert t.lights.shape == (8, 8)


def test_stress_workload_recipe():
    s = scenes.workload_stress()
    assert s.scene.n_tri == 2000 * _uv_sphere_tris(64, 32) + 2047 * 2047 * 2 == 16316418
    assert s.depth == 11 and len(s.views) == 16
    assert all((v.width, v.height) == (3840, 2160) for v in s.views)
    assert math.isclose(s.normal_pitch, float(s.scene.cube_side) / scenes.STRESS_RESOLUTION, rel_tol=1e-12)


def _arrays(sc):
    return [sc.pos, sc.nrm, sc.idx, sc.tri_material, sc.albedo, sc.cube_min, np.array([sc.cube_side])]


@pytest.mark.parametrize("make", [scenes.spheres_scene, scenes.terrain_scene, scenes.boxes_scene])
def test_scenes_deterministic_per_seed(make):
    a, b, c = make(11), make(11), make(12)
    assert all(np.array_equal(x, y) for x, y in zip(_arrays(a), _arrays(b)))
    assert not np.array_equal(a.pos, c.pos)


@pytest.mark.parametrize("make", [scenes.spheres_scene, scenes.terrain_scene, scenes.boxes_scene])
def test_scene_well_formed(make):
    sc = make()
    assert sc.idx.max() < sc.n_vtx and sc.tri_material.max() < sc.albedo.shape[0]
    n = np.linalg.norm(sc.nrm.astype(np.float64), axis=1)
    assert np.abs(n - 1.0).max() < 1e-5
    lo = sc.pos.astype(np.float64).min(axis=0)
    hi = sc.pos.astype(np.float64).max(axis=0)
    ext = float((hi - lo).max())
    assert np.array_equal(sc.cube_min, lo.astype(np.float32))
    assert math.isclose(float(sc.cube_side), ext * (1 + 2 ** -10), rel_tol=1e-6)
    assert (sc.pos < sc.cube_min + sc.cube_side).all()  # every vertex strictly inside the cube
    assert ((sc.albedo >= 0.2) & (sc.albedo <= 1.0)).all()


def test_orbit_cameras():
    w = scenes.workload_terrain_1080p()
    R = 0.5 * math.sqrt(3.0) * float(w.scene.cube_side)
    for cam in [w.capture] + list(w.views):
        f, r, u = (np.asarray(v, np.float64) for v in (cam.fwd, cam.right, cam.up))
        frame = np.stack([r, u, f])
        assert np.abs(frame @ frame.T - np.eye(3)).max() < 1e-6  # orthonormal
        assert np.allclose(np.cross(r, u), -f, atol=1e-6)  # right-handed with the eye looking along fwd
        assert math.isclose(float(cam.pitch), 2 * R / min(cam.width, cam.height), rel_tol=1e-6)
        assert math.isclose(float(cam.z0), -R, rel_tol=1e-6) and math.isclose(float(cam.z1), R, rel_tol=1e-6)
        assert np.allclose(cam.origin, w.scene.center, atol=1e-6)
        assert math.isclose(-f[1], math.sin(math.radians(30.0)), abs_tol=1e-6)  # elevation 30 degrees
    f0 = np.asarray(w.views[0].fwd, np.float64)
    for view, deg in zip(w.views, (0.0, 30.0, 60.0)):
        f = np.asarray(view.fwd, np.float64)
        h0, h = f0[[0, 2]] / np.linalg.norm(f0[[0, 2]]), f[[0, 2]] / np.linalg.norm(f[[0, 2]])
        assert math.isclose(float(h0 @ h), math.cos(math.radians(deg)), abs_tol=1e-6)  # orbit about +y


def test_lights():
    w = scenes.workload_terrain_1080p()
    L = w.lights
    assert (L[:, 0] == 1.0).all()  # point lights
    assert ((L[:, 1] >= 0) & (L[:, 1] < 1) & (L[:, 3] >= 0) & (L[:, 3] < 1)).all()
    assert ((L[:, 2] >= 0.5) & (L[:, 2] < 1.0)).all()
    assert np.allclose(L[:, 4:7], 0.125)
    d = scenes.workload_spheres_256().lights
    assert d.shape == (1, 8) and d[0, 0] == 0.0
    assert np.allclose(d[0, 1:4], np.ones(3) / math.sqrt(3.0), atol=1e-7)


def test_batched_workloads_recipe():
    from paper_2211_15460_gb300 import batched

    ws = batched.batched_workloads()
    assert len(ws) == 16
    n = [w.scene.n_tri for w in ws]
    assert n[0] == 9600 and n[-1] == 1999680  # 10k .. 2M, rounded to whole meshes
    assert all(b > a for a, b in zip(n, n[1:]))  # geometric growth
    for w in ws:
        assert len(w.views) == 64 and (w.capture.width, w.capture.height) == (1280, 720)
        assert w.depth == (10 if w.scene.n_tri > 500_000 else 9)
    again = batched.batched_workloads()
    assert all(np.array_equal(a.scene.pos, b.scene.pos) for a, b in zip(ws, again))
