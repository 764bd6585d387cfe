"""The allocation-free POFA compaction entry point against the regular one.

fhv_compact_pofa_static serves callers that cannot allocate device memory
(plug-ins handed device pointers by a host application, real-time loops that
must not call cudaMalloc): its scratch is a fixed array inside the library.
Two calls in a row, through the C ABI, must give the same POFA records and
(off, cnt) arrays as fhv_compact_pofa with a caller-owned workspace. The
first call uses a shallow octree so that octant ranges exceed the shared-memory
sort and the merge scratch inside the fixed array is used; the second a deep
one, so the tile look-back states in the array are reused after the first
call left them dirty.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402


def _records(rng, n):
    rec = np.zeros(n, fhv.RECORD_DTYPE)
    rec["key"] = rng.integers(0, 1 << 63, size=n, dtype=np.uint64)
    rec["tri"] = rng.integers(0, 1000, size=n)
    rec["nrm"] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)
    rec[: n // 8] = rec[n // 8: 2 * (n // 8)]  # bit-identical duplicates
    return rec


def _device(rec, n_max):
    t = torch.zeros(2 * n_max, dtype=torch.int64, device="cuda")
    t[: 2 * rec.size] = torch.from_numpy(rec.view(np.int64)).cuda()
    return t


def test_static_workspace_compaction_matches_regular_entry_point():
    L = fhv.lib()
    rng = np.random.default_rng(2024)
    for depth, n in ((1, 100_000), (10, 300_000)):
        rec = _records(rng, n)
        n_max = n + 5
        src = _device(rec, n_max)
        d_n = torch.tensor([n, 0], dtype=torch.int64, device="cuda")
        m = fhv.fhv_level_offset(depth + 1)
        # regular entry point, caller-owned workspace
        ref_out = torch.zeros_like(src)
        ref_off = torch.zeros(m, dtype=torch.int32, device="cuda")
        ref_cnt = torch.zeros(m, dtype=torch.int32, device="cuda")
        ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFA, 0, 1, 1, depth, n_max).workspace_bytes)
        fhv.fhv_compact_pofa(src, n_max, d_n, depth, ref_out, ref_off, ref_cnt, ws)
        # allocation-free entry point, called directly through the C ABI
        out = torch.full_like(src, -1)
        off = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        st = L.fhv_compact_pofa_static(src.data_ptr(), n_max, d_n.data_ptr(), depth, out.data_ptr(), off.data_ptr(),
                                       cnt.data_ptr(), stream)
        assert st == fhv.FHV_OK, fhv.status_str(st)
        # the call's device status word (bounded waits, octant ranges) is clean
        word = C.c_uint32(7)
        st = L.fhv_read_static_status(C.byref(word), stream)
        assert st == fhv.FHV_OK and word.value == 0, (fhv.status_str(st), word.value)
        torch.cuda.synchronize()
        assert torch.equal(out[: 2 * n], ref_out[: 2 * n])
        # every octant of every level (entries 1..3 after the root are unused padding)
        defined = [slice(0, 1), slice(fhv.fhv_level_offset(1), m)]
        for sl in defined:
            assert torch.equal(off[sl], ref_off[sl])
            assert torch.equal(cnt[sl], ref_cnt[sl])
        # and the result is the sorted record array
        got = out[: 2 * n].cpu().numpy().view(fhv.RECORD_DTYPE)
        assert (got == np.sort(rec, order=["key", "tri", "nrm"])).all()
        del ref_off, ref_cnt, off, cnt
        torch.cuda.empty_cache()


def test_static_workspace_rejects_oversized_input():
    L = fhv.lib()
    st = L.fhv_compact_pofa_static(None, fhv.FHV_STATIC_MAX_RECORDS + 1, None, 6, None, None, None, None)
    assert st == fhv.FHV_ERR_UNSUPPORTED
