"""The stress configuration at full size on the GPU: 16,316,418 triangles
captured along the three axes into one POFA at depth 11 (about 5e8 records of
16 bytes; the dense octree index has 9.8e9 octants) and 16 novel views at
3840 x 2160 rendered by one batched call.

The oracle cannot redo all of it in a test's time, so it checks what it can
compute by parts, and the rest is checked by properties that hold at any
size:
* oracle: the total fragment count; every fragment of 256 random triangles
  (a sub-scene of them, same vertices and quantisation cube); the
  visibility and image of one whole view from all records;
* the POFA is the POFL's records in (key, tri, nrm) order: sorted, and equal
  to them as a multiset (sums of fields and of two mixing functions);
* offsets and counts: levels 0..7 in full against the sorted keys, levels
  8..11 at random and occupied octants, and off[o] + cnt[o] = off[o + 1],
  sum cnt = n on every level; the sparse leaf index equals them on every
  occupied leaf; the sparse-index compaction gives the same records, and on
  every level exactly the octants with cnt > 0, with their off and cnt;
* the other 15 views against one fhv_render_view call each (visibility
  bit-identical, colours within 1e-6);
* opaque ray casting of view 0 through the depth-11 octree, with and without
  overflow slabs, gives the splat's visibility.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import batched, fhv, scenes  # noqa: E402

RGB_TOL = 1e-4
C1, C2 = np.uint64(0x9E3779B97F4A7C15), np.uint64(0xBF58476D1CE4E5B9)


def mixes(r):
    k, t, m = r["key"], r["tri"].astype(np.uint64), r["nrm"].astype(np.uint64)
    with np.errstate(over="ignore"):
        h1 = k * C1 + (t << np.uint64(32) | m) * C2
        h2 = (k ^ (k >> np.uint64(29))) * C2 + t * C1 + m
        return [int(x.sum(dtype=np.uint64)) for x in (k, t, m, h1, h2)]


def test_stress_depth11_full_size(oracle_mod):
    orc = oracle_mod
    w = scenes.workload_stress()
    sc, d, pitch = w.scene, w.depth, w.normal_pitch
    ds = fhv.DeviceScene(sc, "cuda")
    leaf = torch.empty(1 << (3 * d), dtype=torch.int32, device="cuda")
    levels = torch.empty(fhv.fhv_level_offset(d), dtype=torch.int32, device="cuda")
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, sc.n_tri, 1, 1, d, 0).workspace_bytes)
    probe = fhv.FragBuf(1, "cuda")  # counts past capacity: learns the size
    fhv.fhv_build_pofl(ds, fhv.FHV_CAPTURE_AXIS3, w.capture, pitch, d, leaf, levels, probe, ws)
    st, n = fhv.fhv_get_count(probe)
    assert st == fhv.FHV_ERR_OVERFLOW and 4e8 < n < 6e8, n
    del probe
    fb = fhv.FragBuf(n, "cuda")
    off = torch.empty(fhv.fhv_level_offset(d + 1), dtype=torch.int32, device="cuda")
    cnt = torch.empty_like(off)
    pofa = torch.empty(2 * n, dtype=torch.int64, device="cuda")
    wsc = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, d, n).workspace_bytes)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    fhv.fhv_build_pofl(ds, fhv.FHV_CAPTURE_AXIS3, w.capture, pitch, d, leaf, levels, fb, ws)
    ev[1].record()
    fhv.fhv_compact_pofa(fb.rec, n, fb.count, d, pofa, off, cnt, wsc)
    ev[2].record()
    bv = batched.BatchedViews([batched.BuiltSource(sc, pofa, n, ds)], [w.views], w.lights, w.footprint_k)
    bv.render()  # first call: kernel attributes
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t0.record()
    bv.render()
    ev[3].record()
    torch.cuda.synchronize()
    assert fhv.fhv_get_count(fb) == (fhv.FHV_OK, n)
    for x in (ws, wsc, bv.ws):
        assert fhv.fhv_read_status(x) == (fhv.FHV_OK, 0)
    print(f"\nstress: {n} fragments; build {ev[0].elapsed_time(ev[1]):.2f} ms, compact "
          f"{ev[1].elapsed_time(ev[2]):.2f} ms, 16 views at 3840x2160 {t0.elapsed_time(ev[3]):.2f} ms")

    # the total against the oracle
    assert orc.fragment_count(sc, orc.AXIS3, None, pitch) == n

    # POFA = POFL records sorted by (key, tri, nrm)
    P = pofa.view(-1, 2).cpu().numpy().view(fhv.RECORD_DTYPE).reshape(-1)
    L = fb.rec[: 2 * n].view(-1, 2).cpu().numpy().view(fhv.RECORD_DTYPE).reshape(-1)
    assert mixes(P) == mixes(L)
    del L
    k = P["key"]
    assert bool((k[1:] >= k[:-1]).all())
    eq = np.flatnonzero(k[1:] == k[:-1])
    t, m = P["tri"], P["nrm"]
    assert bool(((t[eq + 1] > t[eq]) | ((t[eq + 1] == t[eq]) & (m[eq + 1] >= m[eq]))).all())
    del eq

    # every fragment of 256 random triangles, against the oracle
    sel = np.sort(np.random.default_rng(11).choice(sc.n_tri, 256, replace=False))
    sub = scenes.Scene(pos=sc.pos, nrm=sc.nrm, idx=sc.idx[sel], tri_material=sc.tri_material[sel], albedo=sc.albedo,
                       cube_min=sc.cube_min, cube_side=sc.cube_side)
    ro = orc.fragments(sub, orc.AXIS3, None, pitch)[0]
    ro["tri"] = sel[ro["tri"]].astype(np.uint32)
    flag = np.zeros(sc.n_tri, bool)
    flag[sel] = True
    rg = P[flag[t]]
    assert ro.size == rg.size > 0
    assert (np.sort(ro, order=["key", "tri", "nrm"]) == rg).all()  # rg is already in that order
    del flag, rg

    # offsets and counts
    rng = np.random.default_rng(12)
    for lev in range(d + 1):
        base = fhv.fhv_level_offset(lev)
        size = 1 << (3 * lev)
        pre = (k >> np.uint64(63 - 3 * lev)).astype(np.int64) if lev else np.zeros(n, np.int64)
        if lev <= 7:
            octs = np.arange(size, dtype=np.int64)
        else:
            occ = pre[rng.integers(0, n, 100000)]
            octs = np.unique(np.concatenate([occ, np.clip(occ + 1, 0, size - 1), rng.integers(0, size, 100000),
                                             [0, size - 1]]))
        idx = torch.from_numpy(octs + base).cuda()
        go = off[idx].cpu().numpy().view(np.uint32)
        gc = cnt[idx].cpu().numpy().view(np.uint32)
        eo = np.searchsorted(pre, octs, side="left")
        ec = np.searchsorted(pre, octs, side="right") - eo
        assert (go == eo).all() and (gc == ec).all(), lev
        del pre
        total, step = 0, 1 << 28
        for c0 in range(0, size, step):  # scan identity in chunks (the leaf level has 8.6e9 octants)
            c1 = min(size, c0 + step)
            lo = off[base + c0: base + c1 + (1 if c1 < size else 0)].to(torch.int64)
            lc = cnt[base + c0: base + c1].to(torch.int64)
            total += int(lc.sum().item())
            if c1 < size:
                assert bool(((lo[1:] - lo[:-1]) == lc).all().item()), lev
            else:
                assert bool(((lo[1:] - lo[:-1]) == lc[:-1]).all().item()), lev
                assert int(lo[-1].item()) + int(lc[-1].item()) == n
            del lo, lc
        assert total == n, lev

    # the sparse leaf index equals the dense offsets and counts on every occupied leaf
    leaf_ids = torch.empty(n, dtype=torch.int64, device="cuda")
    loff = torch.empty(n, dtype=torch.int32, device="cuda")
    lcnt = torch.empty(n, dtype=torch.int32, device="cuda")
    mdev = torch.zeros(2, dtype=torch.int64, device="cuda")
    lws = fhv.workspace(fhv.FHV_LEAF_INDEX_WS_BYTES(n))
    fhv.fhv_pofa_leaf_index(pofa, n, None, d, leaf_ids, loff, lcnt, mdev, lws)
    mm = int(mdev[0].item())
    assert 0 < mm <= n
    assert mm == int((cnt[fhv.fhv_level_offset(d): fhv.fhv_level_offset(d + 1)] != 0).sum().item())
    # ids in range before they index anything on the device
    assert bool(((leaf_ids[:mm] >= 0) & (leaf_ids[:mm] < (1 << (3 * d)))).all().item())
    sel = leaf_ids[:mm] + fhv.fhv_level_offset(d)
    assert torch.equal(off[sel], loff[:mm]) and torch.equal(cnt[sel], lcnt[:mm])
    assert bool((leaf_ids[1:mm] > leaf_ids[: mm - 1]).all().item())
    print(f"sparse leaf index: {mm} occupied leaves of {1 << (3 * d)}")
    del leaf_ids, loff, lcnt, sel

    # the sparse-index compaction (no array of 8^11 entries): the same records, and every level's entries
    # are exactly the octants with cnt > 0 in the dense arrays, with their off and cnt
    del leaf
    torch.cuda.empty_cache()
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, n)
    spofa = torch.empty_like(pofa)
    base = torch.zeros(d + 4, dtype=torch.int64, device="cuda")
    sws = fhv.workspace(s.workspace_bytes)
    fhv.fhv_compact_pofa_sparse(fb.rec, n, fb.count, d, spofa, None, 0, base, sws)  # learns the index size
    need = int(base[d + 1].item())
    assert fhv.fhv_read_status(sws)[1] & fhv.FHV_DEV_INDEX_OVERFLOW
    index = torch.empty(2 * need, dtype=torch.int64, device="cuda")
    t2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t2[0].record()
    fhv.fhv_compact_pofa_sparse(fb.rec, n, fb.count, d, spofa, index, need, base, sws)
    t2[1].record()
    torch.cuda.synchronize()
    assert fhv.fhv_read_status(sws) == (fhv.FHV_OK, 0)
    assert torch.equal(spofa, pofa)
    lb = base[: d + 2].cpu().numpy()
    ent = index.view(-1, 2)
    for lev in range(d + 1):
        e = ent[lb[lev]: lb[lev + 1]]
        b0, size = fhv.fhv_level_offset(lev), 1 << (3 * lev)
        occupied = int((cnt[b0: b0 + size] != 0).sum().item()) if size < (1 << 31) else sum(
            int((cnt[b0 + c0: b0 + min(size, c0 + (1 << 30))] != 0).sum().item()) for c0 in range(0, size, 1 << 30))
        assert e.shape[0] == occupied, lev
        octs = e[:, 0]
        assert bool(((octs >= 0) & (octs < size)).all().item()), lev
        if octs.numel() > 1:
            assert bool((octs[1:] > octs[:-1]).all().item()), lev
        sel = octs + b0
        assert torch.equal((e[:, 1] & 0xFFFFFFFF), off[sel].to(torch.int64) & 0xFFFFFFFF), lev
        assert torch.equal((e[:, 1] >> 32) & 0xFFFFFFFF, cnt[sel].to(torch.int64) & 0xFFFFFFFF), lev
    print(f"sparse index: {need} occupied octants over {d + 1} levels ({16 * need / 1e9:.3f} GB), "
          f"compaction {t2[0].elapsed_time(t2[1]):.2f} ms")
    del spofa, index, sws, ent
    torch.cuda.empty_cache()

    # views: batched == one call each; view 0 against the oracle
    lights = torch.from_numpy(np.ascontiguousarray(w.lights, np.float32).reshape(-1)).cuda()
    one_vis = torch.empty_like(bv.vis[0])
    one_rgba = torch.empty_like(bv.rgba[0])
    rws = fhv.workspace(fhv.FHV_RENDER_WS_BYTES)
    for i, cam in enumerate(w.views):
        fhv.fhv_render_view(pofa, n, None, ds, ds.albedo, lights, w.lights.shape[0], cam, w.footprint_k, one_vis,
                            one_rgba, rws)
        assert torch.equal(one_vis, bv.vis[i]), i
        assert (one_rgba - bv.rgba[i]).abs().max().item() < 1e-6, i  # same winner; contraction may differ
    t1 = time.time()
    vis_o = orc.splat_visibility(P, sc, w.views[0], w.footprint_k)
    assert (bv.vis[0].cpu().numpy().view(np.uint64) == vis_o).all()
    rgba_o = orc.shade(vis_o, P, sc, sc.albedo, w.lights, w.views[0])
    assert np.abs(bv.rgba[0].cpu().numpy().reshape(-1, 4) - rgba_o).max() < RGB_TOL
    print(f"oracle view: {time.time() - t1:.1f} s")
    assert fhv.fhv_read_status(rws) == (fhv.FHV_OK, 0)

    # opaque ray casting through the depth-11 octree equals the splat's visibility (a property of the
    # method the oracle pins), with overflow slabs and without them (tiles whose frontier does not fit
    # on chip then cast their rays depth first)
    cam = w.views[0]
    for ws_bytes in (fhv.FHV_RAYCAST_WS_BYTES, fhv.FHV_RENDER_WS_BYTES):
        cws = fhv.workspace(ws_bytes)
        fhv.fhv_raycast_pofa(pofa, n, off, cnt, d, ds, ds.albedo, None, 0.0, lights, w.lights.shape[0], cam, one_vis,
                             one_rgba, cws)
        torch.cuda.synchronize()
        assert torch.equal(one_vis, bv.vis[0]), ws_bytes
        assert fhv.fhv_read_status(cws) == (fhv.FHV_OK, 0)
        fallback = int(cws[48:52].cpu().numpy().view(np.uint32)[0])
        print(f"ray cast, workspace {ws_bytes} bytes: {fallback} tiles cast depth first")
