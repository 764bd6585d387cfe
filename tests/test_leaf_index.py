"""The sparse leaf index of a POFA (fhv_pofa_leaf_index) against its
definition on the oracle's POFA (distinct leaves of the sorted keys, the
index of each one's first record, its record count) and against the dense
offsets and counts of fhv_compact_pofa on every occupied leaf."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402


def random_records(rng, n):
    rec = np.zeros(n, fhv.RECORD_DTYPE)
    k = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    hot = rng.integers(0, 1 << 63, size=8, dtype=np.uint64)
    sel = rng.random(n) < 0.5
    k[sel] = (hot[rng.integers(0, 8, size=sel.sum())] & ~np.uint64(0xFFFF)) | (k[sel] & np.uint64(0xFF))
    rec["key"] = k
    rec["tri"] = rng.integers(0, 50, size=n)
    rec["nrm"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    if n > 10:
        rec[: n // 10] = rec[n // 10: 2 * (n // 10)]  # bit-identical duplicates
    return rec


def to_dev(rec):
    return torch.from_numpy(rec.view(np.int64).copy()).cuda()


@pytest.mark.parametrize("depth,n", [(1, 5000), (3, 4095), (3, 4096), (6, 4097), (6, 1), (9, 100003), (9, 0),
                                     (4, 20000)])
def test_leaf_index(oracle_mod, depth, n):
    rng = np.random.default_rng(700 + depth + n)
    rec = random_records(rng, n)
    m_oct = fhv.fhv_level_offset(depth + 1)
    off = torch.empty(m_oct, dtype=torch.int32, device="cuda")
    cnt = torch.empty(m_oct, dtype=torch.int32, device="cuda")
    pofa = torch.empty(max(n, 1) * 2, dtype=torch.int64, device="cuda")
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, depth, max(n, 1)).workspace_bytes)
    fhv.fhv_compact_pofa(to_dev(rec) if n else pofa, n, None, depth, pofa, off, cnt, ws)
    cap = n + 7  # the device counter path: n_max above n
    count = torch.tensor([n, 0], dtype=torch.int64, device="cuda")
    src = torch.zeros(cap * 2, dtype=torch.int64, device="cuda")
    src[: 2 * n] = pofa[: 2 * n]
    leaf = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    loff = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    lcnt = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    m = torch.zeros(2, dtype=torch.int64, device="cuda")
    lws = fhv.workspace(fhv.FHV_LEAF_INDEX_WS_BYTES(cap))
    fhv.fhv_pofa_leaf_index(src, cap, count, depth, leaf, loff, lcnt, m, lws)
    torch.cuda.synchronize()
    # the definition, on the oracle's POFA
    ref = oracle_mod.pofa(rec, depth)[0]
    lv = (ref["key"] >> np.uint64(63 - 3 * depth)).astype(np.int64)
    ul, first, counts = np.unique(lv, return_index=True, return_counts=True)
    mm = int(m[0].item())
    assert mm == ul.size
    assert np.array_equal(leaf[:mm].cpu().numpy(), ul)
    assert np.array_equal(loff[:mm].cpu().numpy().view(np.uint32), first.astype(np.uint32))
    assert np.array_equal(lcnt[:mm].cpu().numpy().view(np.uint32), counts.astype(np.uint32))
    # and the dense arrays agree on every occupied leaf
    if mm:
        idx = leaf[:mm] + fhv.fhv_level_offset(depth)
        assert torch.equal(off[idx], loff[:mm]) and torch.equal(cnt[idx], lcnt[:mm])
