"""FHV_POFA with a sparse octree index (fhv_compact_pofa_sparse) through the
C ABI: the records equal the dense compaction's (the unique sorted array),
and every level's entries are exactly the occupied octants in Morton order
with the offset and count the definition gives them (the first record with
that prefix, the number of records with it), checked against brute force
on random records and against the oracle's octant ranges and the dense
arrays on the benchmark scene."""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402


def random_records(rng, n, depth, clustered=False):
    """Random records with bit-identical duplicates; `clustered` packs them
    into few leaves (long leaf ranges: shared-memory and merge sorts);
    "bucketed" gives buckets (octants of level depth - 3) of about 300
    records whose keys repeat (whole-range sorts through packed keys, with
    runs of equal keys ordered by triangle and normal)."""
    rec = np.zeros(n, fhv.RECORD_DTYPE)
    key = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    if clustered == "bucketed":
        gsh = np.uint64(63 - 3 * (depth - 3))
        bucket = rng.integers(0, max(1, n // 300), size=n, dtype=np.uint64) * np.uint64(7919) % (np.uint64(1) << np.uint64(3 * (depth - 3)))
        key = (bucket << gsh) | rng.integers(0, 1000, size=n, dtype=np.uint64)
    elif clustered:
        key = key >> np.uint64(3 * depth) | (rng.integers(0, 5, size=n, dtype=np.uint64) << np.uint64(63 - 3 * depth))
    rec["key"] = key
    rec["tri"] = rng.integers(0, 50, size=n)
    rec["nrm"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    if n >= 16:
        rec[: n // 8] = rec[n // 8: 2 * (n // 8)]
    return rec


def brute_levels(sorted_rec, depth):
    """Per level: (octants, off, cnt) of the occupied octants, from the sorted keys."""
    k = sorted_rec["key"]
    out = []
    for l in range(depth + 1):
        pre = (k >> np.uint64(63 - 3 * l)) if l else np.zeros(k.size, np.uint64)
        octs, first, counts = np.unique(pre, return_index=True, return_counts=True)
        out.append((octs, first, counts))
    return out


def run_sparse(rec, depth, n_max=None, d_n=None, capacity=None):
    n = rec.size
    n_max = n if n_max is None else n_max
    src = torch.zeros(2 * max(n_max, 1), dtype=torch.int64, device="cuda")
    if n:
        src[: 2 * n] = torch.from_numpy(rec.view(np.int64)).cuda()
    pofa = torch.full_like(src, -1)
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, depth, n_max)
    cap = s.n_index_entries if capacity is None else capacity
    index = torch.full((2 * max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    base = torch.full((depth + 2 + 2,), -1, dtype=torch.int64, device="cuda")
    ws = fhv.workspace(s.workspace_bytes)
    fhv.fhv_compact_pofa_sparse(src, n_max, d_n, depth, pofa, index, cap, base, ws)
    st = fhv.fhv_read_status(ws)[1]
    return pofa, index, base, st


def check_index(index, base, depth, expect):
    levels = fhv.sparse_levels(index, base, depth)
    for l, ((octs, first, counts), got) in enumerate(zip(expect, levels)):
        assert got.size == octs.size, l
        assert (got["octant"] == octs).all(), l
        assert (got["off"] == first).all(), l
        assert (got["cnt"] == counts).all(), l


@pytest.mark.parametrize("depth,n,clustered", [(1, 50_000, False), (2, 20_000, True), (4, 100_000, False),
                                               (5, 70_000, True), (6, 30_000, False), (10, 300_000, False),
                                               (11, 200_000, False), (11, 40_000, True), (3, 1, False),
                                               (10, 200_000, "bucketed"), (11, 150_000, "bucketed")])
def test_sparse_compaction_against_brute_force(depth, n, clustered):
    rng = np.random.default_rng(depth * 1000 + n)
    rec = random_records(rng, n, depth, clustered)
    pofa, index, base, st = run_sparse(rec, depth)
    assert st == 0
    srt = np.sort(rec, order=["key", "tri", "nrm"])
    assert (fhv.records_to_numpy(pofa, n) == srt).all()
    check_index(index, base, depth, brute_levels(srt, depth))
    assert int(base[depth + 1].item()) == sum(e[0].size for e in brute_levels(srt, depth))


def test_sparse_compaction_counter_and_empty():
    rng = np.random.default_rng(7)
    rec = random_records(rng, 5000, 8)
    d_n = torch.tensor([3000, 0], dtype=torch.int64, device="cuda")  # only the first 3000 count
    pofa, index, base, st = run_sparse(rec, 8, n_max=5000, d_n=d_n)
    assert st == 0
    srt = np.sort(rec[:3000], order=["key", "tri", "nrm"])
    assert (fhv.records_to_numpy(pofa, 3000) == srt).all()
    check_index(index, base, 8, brute_levels(srt, 8))
    d_n.zero_()
    pofa, index, base, st = run_sparse(rec, 8, n_max=5000, d_n=d_n)
    assert st == 0 and (base[: 8 + 2] == 0).all()


def test_sparse_index_overflow_reports_the_size():
    """An index too small for the occupied octants: entries up to the
    capacity are written, the status word says so, and the level bases give
    the size to re-allocate (Section 3.1's rule for undersized buffers)."""
    rng = np.random.default_rng(8)
    rec = random_records(rng, 20_000, 10)
    srt = np.sort(rec, order=["key", "tri", "nrm"])
    expect = brute_levels(srt, 10)
    need = sum(e[0].size for e in expect)
    cap = need // 3
    pofa, index, base, st = run_sparse(rec, 10, capacity=cap)
    assert st & fhv.FHV_DEV_INDEX_OVERFLOW
    assert int(base[11].item()) == need
    assert (fhv.records_to_numpy(pofa, rec.size) == srt).all()
    flat = np.concatenate([np.stack([o.astype(np.uint64), f.astype(np.uint64), c.astype(np.uint64)], 1)
                           for o, f, c in expect])
    got = index[: 2 * cap].cpu().numpy().view(fhv.OCTANT_DTYPE).reshape(-1)
    lb = base[:12].cpu().numpy()
    # entries whose successor on the same level was written carry their count too
    for k in range(cap):
        assert got["octant"][k] == flat[k, 0] and got["off"][k] == flat[k, 1]
        l = int(np.searchsorted(lb, k, side="right") - 1)
        if k + 1 < cap or k + 1 == lb[l + 1]:
            assert got["cnt"][k] == flat[k, 2]


@pytest.fixture(scope="module")
def terrain_records():
    w = scenes.workload_terrain_1080p()
    ds = fhv.DeviceScene(w.scene)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, w.scene.n_tri, 1, 1, w.depth, 0).workspace_bytes)
    probe = fhv.FragBuf(0, links=False)
    fhv.fhv_capture_fragments(ds, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, probe, ws)
    n = fhv.fhv_get_count(probe)[1]
    fb = fhv.FragBuf(n, links=False)
    fhv.fhv_capture_fragments(ds, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, fb, ws)
    assert fhv.fhv_get_count(fb) == (fhv.FHV_OK, n)
    return w, fb, n


def test_sparse_equals_dense_on_terrain_depth10(oracle_mod, terrain_records):
    """The 1M-triangle terrain at depth 10: the sparse compaction's records
    equal the dense one's byte for byte; every occupied octant of every
    level equals the dense arrays' off / cnt, the levels hold exactly the
    octants with cnt > 0, and sampled octants equal the oracle's range."""
    w, fb, n = terrain_records
    d = w.depth
    m = fhv.fhv_level_offset(d + 1)
    off = torch.empty(m, dtype=torch.int32, device="cuda")
    cnt = torch.empty(m, dtype=torch.int32, device="cuda")
    dense = torch.empty(2 * n, dtype=torch.int64, device="cuda")
    wsd = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, d, n).workspace_bytes)
    fhv.fhv_compact_pofa(fb.rec, n, fb.count, d, dense, off, cnt, wsd)
    s = fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA_SPARSE, 0, 1, 1, d, n)
    pofa = torch.empty(2 * n, dtype=torch.int64, device="cuda")
    index = torch.empty(2 * s.n_index_entries, dtype=torch.int64, device="cuda")
    base = torch.empty(d + 2 + 2, dtype=torch.int64, device="cuda")
    ws = fhv.workspace(s.workspace_bytes)
    fhv.fhv_compact_pofa_sparse(fb.rec, n, fb.count, d, pofa, index, s.n_index_entries, base, ws)
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    assert torch.equal(pofa, dense)
    lb = base[: d + 2].cpu().numpy()
    ent = index.view(-1, 2)
    total_occ = 0
    for l in range(d + 1):
        e = ent[lb[l]: lb[l + 1]]
        octs = e[:, 0]
        offcnt = e[:, 1]
        lo_ = (offcnt & 0xFFFFFFFF).to(torch.int64)
        hi_ = (offcnt >> 32) & 0xFFFFFFFF
        dl = slice(fhv.fhv_level_offset(l), fhv.fhv_level_offset(l) + (1 << (3 * l)))
        occupied = torch.nonzero(cnt[dl] != 0).flatten()
        assert torch.equal(octs, occupied), l
        assert torch.equal(lo_, off[dl][occupied].to(torch.int64) & 0xFFFFFFFF), l
        assert torch.equal(hi_, cnt[dl][occupied].to(torch.int64) & 0xFFFFFFFF), l
        total_occ += occupied.numel()
    assert int(lb[d + 1]) == total_occ
    # the oracle's octant ranges on sampled occupied octants of every level
    srt = fhv.records_to_numpy(pofa, n)
    levels = fhv.sparse_levels(index, base, d)
    rng = np.random.default_rng(3)
    for l in range(d + 1):
        e = levels[l]
        pick = rng.choice(e.size, min(e.size, 300), replace=False)
        for k in pick:
            assert oracle_mod.octant_range(srt, l, int(e["octant"][k])) == (int(e["off"][k]), int(e["cnt"][k])), l
    print(f"\nterrain depth 10: {n} records, {total_occ} occupied octants over 11 levels "
          f"({int(lb[d + 1] - lb[d])} leaves)")
