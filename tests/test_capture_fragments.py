"""Records-only capture (fhv_capture_fragments) against the oracle: the
global fragment list of every capture mode holds exactly the oracle's
fragments (bit-exact records, compared as sorted multisets because the
append order follows the device's atomics), and the overflow rule of
Section 3.1 holds without any list arrays."""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402


@pytest.fixture(scope="module")
def orc():
    import oracle

    oracle.build()
    return oracle


def _capture(scene, mode, cam, pitch, capacity):
    ds = fhv.DeviceScene(scene)
    fb = fhv.FragBuf(capacity, links=False)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, scene.n_tri, 1, 1, 1, 0).workspace_bytes)
    fhv.fhv_capture_fragments(ds, mode, cam, pitch, fb, ws)
    st, n = fhv.fhv_get_count(fb)
    assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
    return st, n, fhv.records_to_numpy(fb.rec, min(n, capacity))


def _sorted(rec):
    return np.sort(rec, order=["key", "tri", "nrm"])


@pytest.mark.parametrize("mode", ["view", "normal", "axis3"])
def test_capture_fragments_matches_oracle(orc, mode):
    w = scenes.workload_spheres_256()
    if mode == "view":
        args = (fhv.FHV_CAPTURE_VIEW, w.capture, 0.0)
        ref, _, _ = orc.fragments(w.scene, orc.VIEW, w.capture, 0.0)
    else:
        m = fhv.FHV_CAPTURE_NORMAL if mode == "normal" else fhv.FHV_CAPTURE_AXIS3
        args = (m, None, w.normal_pitch)
        ref, _, _ = orc.fragments(w.scene, orc.NORMAL if mode == "normal" else orc.AXIS3, None, w.normal_pitch)
    st, n, got = _capture(w.scene, *args, capacity=ref.size + 100)
    assert st == fhv.FHV_OK and n == ref.size
    assert (_sorted(got) == _sorted(ref)).all()


def test_capture_fragments_terrain_normal(orc):
    """The benchmark scene at 1080p pitch (1.5M fragments, many tiles of the sample space)."""
    w = scenes.workload_terrain_1080p()
    ref, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    st, n, got = _capture(w.scene, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, ref.size)
    assert st == fhv.FHV_OK and n == ref.size
    assert (_sorted(got) == _sorted(ref)).all()


@pytest.mark.parametrize("capacity", [0, 5, 10_000])
def test_capture_fragments_overflow(orc, capacity):
    """Past capacity the counter keeps counting and nothing is stored; the
    stored prefix is a sub-multiset of the oracle's fragments."""
    w = scenes.workload_spheres_256()
    ref, _, _ = orc.fragments(w.scene, orc.NORMAL, None, w.normal_pitch)
    st, n, got = _capture(w.scene, fhv.FHV_CAPTURE_NORMAL, None, w.normal_pitch, capacity)
    assert n == ref.size and st == fhv.FHV_ERR_OVERFLOW
    assert got.size == min(capacity, n)
    if got.size:
        pool = {}
        for r in ref.tolist():
            pool[r] = pool.get(r, 0) + 1
        for r in got.tolist():
            assert pool.get(r, 0) > 0
            pool[r] -= 1
