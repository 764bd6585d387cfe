"""Saving and loading a built POFA (host side, no GPU): the file round-trips
the records and either index layout byte for byte, and damaged files or
small buffers are refused."""
import os

import numpy as np
import pytest

from paper_2211_15460_gb300 import fhv, scenes


def sparse_index(sorted_rec, depth):
    """Occupied octants of every level of sorted records (OCTANT_DTYPE) and the level bases."""
    k = sorted_rec["key"]
    parts, base = [], [0]
    for l in range(depth + 1):
        pre = (k >> np.uint64(63 - 3 * l)) if l else np.zeros(k.size, np.uint64)
        octs, first, counts = np.unique(pre, return_index=True, return_counts=True)
        e = np.zeros(octs.size, fhv.OCTANT_DTYPE)
        e["octant"], e["off"], e["cnt"] = octs, first, counts
        parts.append(e)
        base.append(base[-1] + octs.size)
    return np.concatenate(parts), np.array(base, np.uint64)


@pytest.fixture(scope="module")
def built(oracle_mod):
    w = scenes.workload_spheres_256()
    rec = oracle_mod.fragments(w.scene, oracle_mod.NORMAL, None, w.normal_pitch)[0]
    pofa, off, cnt = oracle_mod.pofa(rec, w.depth)
    return w.depth, pofa, off.astype(np.uint32), cnt.astype(np.uint32)


def test_dense_round_trip(tmp_path, built):
    depth, pofa, off, cnt = built
    m = fhv.fhv_level_offset(depth + 1)
    off_p = np.zeros(m, np.uint32)
    cnt_p = np.zeros(m, np.uint32)
    for l in range(depth + 1):  # the oracle's root-first levels into the library's padded layout
        import oracle

        b, s = oracle.level_base(l), 8 ** l
        off_p[fhv.fhv_level_offset(l): fhv.fhv_level_offset(l) + s] = off[b: b + s]
        cnt_p[fhv.fhv_level_offset(l): fhv.fhv_level_offset(l) + s] = cnt[b: b + s]
    path = str(tmp_path / "dense.fhv")
    fhv.fhv_pofa_save(path, depth, pofa, off=off_p, cnt=cnt_p)
    h = fhv.fhv_pofa_load_header(path)
    assert (h.depth, h.index_kind, h.n_records, h.n_index_entries) == (depth, 0, pofa.size, m)
    d, rec, (o, c) = fhv.fhv_pofa_load(path)
    assert d == depth and rec.tobytes() == pofa.tobytes()
    assert np.array_equal(o, off_p) and np.array_equal(c, cnt_p)
    assert os.path.getsize(path) == 8 + 64 + 16 * pofa.size + 8 * m


def test_sparse_round_trip_and_refusals(tmp_path, built):
    depth, pofa, _, _ = built
    ent, base = sparse_index(pofa, depth)
    path = str(tmp_path / "sparse.fhv")
    fhv.fhv_pofa_save(path, depth, pofa, index=ent, level_base=base)
    d, rec, (e, b) = fhv.fhv_pofa_load(path)
    assert d == depth and rec.tobytes() == pofa.tobytes()
    assert e.tobytes() == ent.tobytes() and np.array_equal(b, base)
    L = fhv.lib()
    # a record buffer too small: nothing read
    small = np.zeros(10, fhv.RECORD_DTYPE)
    eb = np.zeros(ent.size, fhv.OCTANT_DTYPE)
    bb = np.zeros(depth + 2, np.uint64)
    st = L.fhv_pofa_load(path.encode(), fhv._np_ptr(small), 10, None, None, fhv._np_ptr(eb), ent.size, fhv._np_ptr(bb))
    assert st == fhv.FHV_ERR_OVERFLOW
    # both or neither index, bad depth
    with pytest.raises(fhv.FhvError):
        fhv.fhv_pofa_save(str(tmp_path / "x"), depth, pofa)
    with pytest.raises(fhv.FhvError):
        fhv.fhv_pofa_save(str(tmp_path / "x"), 12, pofa, index=ent, level_base=base)
    # a damaged magic and a truncated file
    raw = open(path, "rb").read()
    bad = tmp_path / "bad.fhv"
    bad.write_bytes(b"XX" + raw[2:])
    with pytest.raises(fhv.FhvError):
        fhv.fhv_pofa_load_header(str(bad))
    bad.write_bytes(raw[: len(raw) - 17])
    with pytest.raises(fhv.FhvError):
        fhv.fhv_pofa_load(str(bad))
    with pytest.raises(fhv.FhvError):
        fhv.fhv_pofa_load_header(str(tmp_path / "missing.fhv"))
