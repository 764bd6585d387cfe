"""The sharded build and render (one scene's records split over ranks).

On CPU: gloo ranks run the orchestration of paper_2211_15460_gb300.sharded
with the oracle as every rank's local compaction / splat / shade; the
owners' slices, concatenated in rank order, must be the oracle's POFA of all
records byte for byte, and the visibility and image must equal the oracle's
render of that POFA exactly. On the GPU: the same with the library's kernels,
two processes sharing one device (no kernel waits on another: the exchange
runs through gloo on the host), against the single-process result.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2211_15460_gb300 import sharded  # noqa: E402

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
MASK = np.uint64((1 << 40) - 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


# ------------------------------------------------------------ host logic

def test_balanced_bounds():
    b = sharded.balanced_bounds(np.ones(64, np.int64), 4)
    assert b.tolist() == [0, 16, 32, 48, 64]
    b = sharded.balanced_bounds(np.array([0, 0, 100, 0]), 2)  # all in one octant: one rank takes it
    assert b[0] == 0 and b[-1] == 4 and (np.diff(b) >= 0).all()
    counts = [int(np.array([0, 0, 100, 0])[b[r]:b[r + 1]].sum()) for r in range(2)]
    assert sorted(counts) == [0, 100]
    b = sharded.balanced_bounds(np.zeros(8, np.int64), 3)
    assert b[0] == 0 and b[-1] == 8 and (np.diff(b) >= 0).all()
    b = sharded.balanced_bounds(np.array([5, 1]), 5)  # more ranks than octants
    assert b[0] == 0 and b[-1] == 2 and (np.diff(b) >= 0).all()
    rng = np.random.default_rng(3)
    for world in (2, 3, 7):
        h = rng.integers(0, 50, 512)
        b = sharded.balanced_bounds(h, world)
        per = np.array([h[b[r]:b[r + 1]].sum() for r in range(world)])
        assert per.sum() == h.sum() and (np.diff(b) >= 0).all()
        assert per.max() <= h.sum() / world + h.max()  # within one octant of an even split
    # fractional weights are not truncated: 1.4 + 0.6 per pair of tiny triangles
    w = np.tile([1.4, 0.6], 8)
    b = sharded.balanced_bounds(w, 2)
    assert abs(w[:b[1]].sum() - 8.0) < 1e-9
    w = np.array([0.9, 0.9, 0.9, 0.1, 0.1, 0.1])  # truncated to 1s these would split 3 | 3
    b = sharded.balanced_bounds(w, 2)
    assert b.tolist() == [0, 2, 6]


def test_sample_weights_closed_form():
    from paper_2211_15460_gb300 import fhv, scenes

    # triangle 0: right triangle of legs 1 in the xy plane (area 1/2, normal +z);
    # triangle 1: the same tilted into the plane x = z (area 1/2 * sqrt(2), normal (1, 0, -1) / sqrt(2))
    pos = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0], [1, 0, 1], [0, 1, 0]], np.float64)
    sc = scenes.Scene(pos=pos, nrm=np.tile([0.0, 0.0, 1.0], (6, 1)), idx=np.arange(6).reshape(2, 3),
                      tri_material=np.zeros(2), albedo=np.ones((1, 3)))
    h = 0.5
    w = sharded.sample_weights(sc, fhv.FHV_CAPTURE_NORMAL, h)
    assert np.allclose(w, [0.5 / h ** 2 + 1, 0.5 * np.sqrt(2) / h ** 2 + 1])
    w = sharded.sample_weights(sc, fhv.FHV_CAPTURE_AXIS3, h)  # |Ax| + |Ay| + |Az| of the area vectors
    assert np.allclose(w, [0.5 / h ** 2 + 1, 1.0 / h ** 2 + 1])
    cam = scenes.Camera(origin=(0, 0, 0), right=(1, 0, 0), up=(0, 1, 0), fwd=(0, 0, -1), pitch=0.25, width=8,
                        height=8, z0=-1, z1=1)
    w = sharded.sample_weights(sc, fhv.FHV_CAPTURE_VIEW, 0.0, cam)  # area projected on the view plane
    assert np.allclose(w, [0.5 / 0.0625 + 1, 0.5 / 0.0625 + 1])


@pytest.mark.parametrize("mode", [1, 2])
def test_triangle_ranges_balance_fragments(oracle_mod, mode):
    """The estimate behind the triangle ranges predicts the capture's work:
    over 4 ranks the oracle's fragment counts per range stay within 30 % of
    their mean (measured: 1.05-1.13 max / mean for the sphere workload,
    about 1.27 for the terrain workload)."""
    from paper_2211_15460_gb300 import scenes

    w = scenes.workload_spheres_256()
    sc = w.scene
    b = sharded.balanced_bounds(sharded.sample_weights(sc, mode, w.normal_pitch), 4)
    counts = []
    for r in range(4):
        sub = scenes.Scene(pos=sc.pos, nrm=sc.nrm, idx=sc.idx[b[r]:b[r + 1]], tri_material=sc.tri_material[b[r]:b[r + 1]],
                           albedo=sc.albedo, cube_min=sc.cube_min, cube_side=sc.cube_side)
        counts.append(oracle_mod.fragment_count(sub, mode, None, w.normal_pitch))
    c = np.array(counts, np.float64)
    assert c.sum() == oracle_mod.fragment_count(sc, mode, None, w.normal_pitch)
    assert c.max() / c.mean() < 1.3 and c.min() / c.mean() > 0.7


# ------------------------------------------------------- CPU ranks (oracle)

class OracleOps:
    """Each rank's local steps by the oracle (test infrastructure)."""

    def __init__(self, depth):
        self.depth = depth

    @staticmethod
    def _records(t):
        from paper_2211_15460_gb300.fhv import RECORD_DTYPE

        return np.ascontiguousarray(t.numpy()).view(RECORD_DTYPE).reshape(-1)

    def compact(self, rec):
        import oracle

        out, off, cnt = oracle.pofa(self._records(rec), self.depth)
        return sharded.LocalPofa(torch.from_numpy(out.view(np.int64).reshape(-1, 2).copy()),
                                 torch.from_numpy(off.astype(np.int64)), torch.from_numpy(cnt.astype(np.int64)),
                                 oracle.level_base)

    def capture(self, scene, t0, t1, mode, cam, pitch):
        """The oracle's fragments of triangles [t0, t1) with the whole scene's ids, compacted."""
        import oracle
        from paper_2211_15460_gb300 import scenes

        sub = scenes.Scene(pos=scene.pos, nrm=scene.nrm, idx=scene.idx[t0:t1], tri_material=scene.tri_material[t0:t1],
                           albedo=scene.albedo, cube_min=scene.cube_min, cube_side=scene.cube_side)
        rec = oracle.fragments(sub, mode, cam, pitch)[0]
        rec["tri"] += np.uint32(t0)
        return self.compact(torch.from_numpy(np.ascontiguousarray(rec).view(np.int64).reshape(-1, 2).copy()))

    def splat(self, rec, base, scene, cam, k):
        import oracle

        vis = oracle.splat_visibility(self._records(rec), scene, cam, k)
        vis = np.where(vis != EMPTY, vis + np.uint64(base), EMPTY)
        return torch.from_numpy(vis.view(np.int64).copy())

    def shade(self, rec, base, scene, albedo, lights, n_lights, cam, vis):
        import oracle

        v = vis.numpy().view(np.uint64)
        idx = v & MASK
        own = (v != EMPTY) & (idx >= np.uint64(base)) & (idx < np.uint64(base + rec.shape[0]))
        v = np.where(own, v - np.uint64(base), EMPTY)
        return torch.from_numpy(oracle.shade(v, self._records(rec), scene, albedo, lights, cam).reshape(-1).copy())


def _split(rec, world, how):
    if how == "interleaved":
        return [rec[r::world] for r in range(world)]
    cut = [0, rec.size // 2, rec.size] + [rec.size] * (world - 2)  # ranks past the second get nothing
    return [rec[cut[r]:cut[r + 1]] for r in range(world)]


def _cpu_worker(rank, world, port, how, out, k=None):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2211_15460_gb300 import scenes

        w = scenes.workload_spheres_256()
        rec = oracle.fragments(w.scene, oracle.NORMAL, None, w.normal_pitch)[0]
        mine = _split(rec, world, how)[rank]
        comm = sharded.Comm()
        ops = OracleOps(w.depth)
        local = torch.from_numpy(np.ascontiguousarray(mine).view(np.int64).reshape(-1, 2).copy())
        sp = sharded.build_pofa(local, w.depth, comm, ops)
        vis, rgba = sharded.render(sp, w.scene, w.scene.albedo, w.lights, w.lights.shape[0], w.views[0],
                                   k or w.footprint_k, comm, ops)
        out[rank] = (sp.rec.numpy().copy(), sp.base, sp.total, vis.numpy().copy(), rgba.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,how,k", [(2, "interleaved", 1), (3, "halves", 1), (2, "halves", 2)])
def test_sharded_matches_single_rank_oracle(oracle_mod, world, how, k):
    from paper_2211_15460_gb300 import scenes

    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_cpu_worker, args=(world, _free_port(), how, out, k), nprocs=world, join=True)
    w = scenes.workload_spheres_256()
    rec = oracle_mod.fragments(w.scene, oracle_mod.NORMAL, None, w.normal_pitch)[0]
    ref = oracle_mod.pofa(rec, w.depth)[0]
    parts = [out[r] for r in range(world)]
    assert [p[1] for p in parts] == list(np.cumsum([0] + [p[0].shape[0] for p in parts])[:-1])
    assert all(p[2] == rec.size for p in parts)
    got = np.concatenate([p[0] for p in parts]).reshape(-1)
    assert got.tobytes() == ref.view(np.int64).tobytes()  # byte-identical POFA
    assert max(p[0].shape[0] for p in parts) < rec.size  # the work is split
    vis_ref, rgba_ref = oracle_mod.render(ref, w.scene, w.views[0], w.lights, k)
    for p in parts:
        assert np.array_equal(p[3].view(np.uint64), vis_ref)
        assert np.array_equal(p[4].reshape(-1, 4), rgba_ref)


def _cpu_capture_worker(rank, world, port, mode, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2211_15460_gb300 import scenes

        w = scenes.workload_spheres_256()
        comm = sharded.Comm()
        ops = OracleOps(w.depth)
        sp = sharded.capture_pofa(w.scene, w.scene, mode, None, w.normal_pitch, w.depth, comm, ops)
        vis, rgba = sharded.render(sp, w.scene, w.scene.albedo, w.lights, w.lights.shape[0], w.views[0],
                                   w.footprint_k, comm, ops)
        out[rank] = (sp.rec.numpy().copy(), sp.base, sp.total, vis.numpy().copy(), rgba.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,mode", [(2, 1), (3, 2)])
def test_sharded_capture_matches_single_rank_oracle(oracle_mod, world, mode):
    """Every rank captures its range of triangles (about equal estimated
    samples); the owners' slices are the oracle's POFA of the whole scene."""
    from paper_2211_15460_gb300 import scenes

    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_cpu_capture_worker, args=(world, _free_port(), mode, out), nprocs=world, join=True)
    w = scenes.workload_spheres_256()
    rec = oracle_mod.fragments(w.scene, mode, None, w.normal_pitch)[0]
    ref = oracle_mod.pofa(rec, w.depth)[0]
    parts = [out[r] for r in range(world)]
    assert all(p[2] == rec.size for p in parts)
    got = np.concatenate([p[0] for p in parts]).reshape(-1)
    assert got.tobytes() == ref.view(np.int64).tobytes()
    vis_ref, rgba_ref = oracle_mod.render(ref, w.scene, w.views[0], w.lights, w.footprint_k)
    for p in parts:
        assert np.array_equal(p[3].view(np.uint64), vis_ref)
        assert np.array_equal(p[4].reshape(-1, 4), rgba_ref)


# ------------------------------------------------------------- GPU ranks

def _gpu_worker(rank, world, port, rec_np, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2211_15460_gb300 import fhv, scenes

        w = scenes.workload_spheres_256()
        scene = fhv.DeviceScene(w.scene, "cuda")
        lights = torch.from_numpy(np.ascontiguousarray(w.lights, np.float32).reshape(-1)).cuda()
        mine = torch.from_numpy(rec_np[rank::world].copy()).cuda()
        comm = sharded.Comm()
        ops = sharded.DeviceOps(w.depth)
        sp = sharded.build_pofa(mine, w.depth, comm, ops)
        vis, rgba = sharded.render(sp, scene, scene.albedo, lights, w.lights.shape[0], w.views[0], w.footprint_k,
                                   comm, ops)
        torch.cuda.synchronize()
        out[rank] = (sp.rec.cpu().numpy().copy(), sp.base, vis.cpu().numpy().copy(), rgba.cpu().numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_on_device_matches_single_process():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_15460_gb300 import fhv, scenes
    from paper_2211_15460_gb300.pipeline import PlainFHV

    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    ref_pofa = p.pofa[: 2 * n].view(-1, 2).cpu().numpy().copy()
    ref_vis, ref_rgba = p.vis[0].cpu().numpy().copy(), p.rgba[0].cpu().numpy().copy()
    rec = p.pofl.rec[: 2 * n].view(-1, 2).cpu().numpy().copy()  # the captured records, in capture order
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_gpu_worker, args=(world, _free_port(), rec, out), nprocs=world, join=True)
    parts = [out[r] for r in range(world)]
    got = np.concatenate([q[0] for q in parts])
    assert got.tobytes() == ref_pofa.tobytes()
    assert parts[1][1] == parts[0][0].shape[0]
    for q in parts:
        assert np.array_equal(q[2], ref_vis)
        assert np.array_equal(q[3], ref_rgba)


def _gpu_capture_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2211_15460_gb300 import fhv, scenes

        w = scenes.workload_spheres_256()
        ds = fhv.DeviceScene(w.scene, "cuda")
        comm = sharded.Comm()
        ops = sharded.DeviceOps(w.depth)
        sp = sharded.capture_pofa(w.scene, ds, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, w.depth, comm, ops)
        torch.cuda.synchronize()
        out[rank] = (sp.rec.cpu().numpy().copy(), sp.base, sp.total)
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_capture_on_device_matches_single_process():
    """Two processes each build the POFA of their range of triangles
    (fhv_build_pofa_direct on a slice), then exchange: the slices are the
    single-process POFA byte for byte."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_15460_gb300 import fhv, scenes
    from paper_2211_15460_gb300.pipeline import PlainFHV

    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    ref_pofa = p.pofa[: 2 * n].view(-1, 2).cpu().numpy().copy()
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_gpu_capture_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    parts = [out[r] for r in range(world)]
    assert all(q[2] == n for q in parts)
    assert parts[1][1] == parts[0][0].shape[0]
    assert np.concatenate([q[0] for q in parts]).tobytes() == ref_pofa.tobytes()


@pytest.mark.gpu
def test_split_render_entries_match_render_view():
    """fhv_splat_visibility + fhv_shade_owned over two slices of one POFA
    (unsigned minimum of the visibility, sum of the images) give exactly what
    fhv_render_view gives for the whole POFA."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_15460_gb300 import fhv, scenes
    from paper_2211_15460_gb300.pipeline import PlainFHV

    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    pofa = p.pofa[: 2 * n].view(-1, 2)
    cam = w.views[0]
    ws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    ref2_vis = torch.empty_like(p.vis[0])
    ref2_rgba = torch.empty_like(p.rgba[0])
    fhv.fhv_render_view(pofa, n, None, p.scene, p.scene.albedo, p.lights, p.n_lights, cam, 2, ref2_vis, ref2_rgba, ws)
    refs = {1: (p.vis[0], p.rgba[0]), 2: (ref2_vis, ref2_rgba)}
    for fk, cut in ((1, 0), (1, n // 3), (1, n), (2, n // 2)):
        slices = [(pofa[:cut], 0), (pofa[cut:], cut)]
        vis = []
        for rec, base in slices:
            v = torch.empty(cam.width * cam.height, dtype=torch.int64, device="cuda")
            fhv.fhv_splat_visibility(rec if rec.shape[0] else None, rec.shape[0], None, base, p.scene, cam, fk, v,
                                     ws)
            vis.append(v.cpu().numpy().view(np.uint64))
        merged = np.minimum(vis[0], vis[1])
        assert np.array_equal(merged, refs[fk][0].cpu().numpy().view(np.uint64))
        vis_t = torch.from_numpy(merged.view(np.int64).copy()).cuda()
        imgs = []
        for rec, base in slices:
            rgba = torch.empty(cam.width * cam.height * 4, dtype=torch.float32, device="cuda")
            fhv.fhv_shade_owned(rec if rec.shape[0] else None, rec.shape[0], None, base, p.scene, p.scene.albedo,
                                p.lights, p.n_lights, cam, vis_t, rgba, ws)
            imgs.append(rgba.cpu().numpy().reshape(-1, 4))
        assert np.array_equal(imgs[0] + imgs[1], refs[fk][1].cpu().numpy().reshape(-1, 4))
        idx = merged & MASK
        owned_a = (merged != EMPTY) & (idx < np.uint64(cut))
        assert (imgs[1][owned_a] == 0).all() and (imgs[0][~owned_a] == 0).all()
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
