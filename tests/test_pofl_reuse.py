"""POFL builds into the previous build's lists (fhv_build_pofl_reuse): the
lists must equal a fresh build's, across changes of scene and of fragment
count, and the rest of the head array must stay -1."""
import numpy as np
import pytest

from paper_2211_15460_gb300 import scenes
from _lists import canonical, list_owner

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv  # noqa: E402
from paper_2211_15460_gb300.pipeline import PlainFHV  # noqa: E402


def lists_of(leaf_head, nxt, rec, n):
    """Canonical (slot, record) rows after checking the list structure."""
    owner = list_owner(leaf_head.cpu().numpy(), nxt[:n].cpu().numpy(), n)
    return canonical(owner, fhv.records_to_numpy(rec, n))


def build(fn, sc_dev, sc, depth, head, levels, fb, ws, pitch):
    fn(sc_dev, fhv.FHV_CAPTURE_NORMAL, None, pitch, depth, head, levels, fb, ws)
    torch.cuda.synchronize()
    return fhv.fhv_get_count(fb)[1]


def test_reuse_equals_fresh_build_across_scenes():
    depth = 6
    scs = [scenes.spheres_scene(s, n_spheres=n) for s, n in ((1, 8), (2, 3), (3, 12), (1, 8))]
    # one cube and pitch for all, so that every scene fits the same octree
    cube_min = np.min([s.cube_min for s in scs], axis=0)
    side = max(float(s.cube_side) for s in scs) * 1.5
    for s in scs:
        s.cube_min, s.cube_side = cube_min.astype(np.float32), np.float32(side)
    pitch = side / 256
    cap = 1 << 20
    head = torch.empty(1 << (3 * depth), dtype=torch.int32, device="cuda")
    levels = torch.empty(fhv.fhv_level_offset(depth), dtype=torch.int32, device="cuda")
    fb = fhv.FragBuf(cap)
    T = max(s.n_tri for s in scs)
    ws = fhv.workspace(fhv.fhv_query_sizes(fhv.FHV_LAYOUT_POFL, T, 1, 1, depth, 0).workspace_bytes)
    # fresh builds for reference, in their own buffers
    ref = []
    for s in scs:
        h2 = torch.empty_like(head)
        l2 = torch.empty_like(levels)
        f2 = fhv.FragBuf(cap)
        ds = fhv.DeviceScene(s)
        n2 = build(fhv.fhv_build_pofl, ds, s, depth, h2, l2, f2, ws, pitch)
        ref.append((lists_of(h2, f2.next, f2.rec, n2), l2.cpu().numpy(), int((h2 != -1).sum().item())))
    for i, s in enumerate(scs):
        fn = fhv.fhv_build_pofl if i == 0 else fhv.fhv_build_pofl_reuse
        n = build(fn, fhv.DeviceScene(s), s, depth, head, levels, fb, ws, pitch)
        assert fhv.fhv_read_status(ws) == (fhv.FHV_OK, 0)
        got = lists_of(head, fb.next, fb.rec, n)
        assert got.size == ref[i][0].size and (got == ref[i][0]).all(), i
        assert (levels.cpu().numpy() == ref[i][1]).all(), i
        assert int((head != -1).sum().item()) == ref[i][2], i  # every other head is -1


def test_pipeline_steps_reuse_the_lists():
    """The plain pipeline rebuilds in place from its second step on; every
    step gives the first step's POFA."""
    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    first = (fhv.records_to_numpy(p.pofa, n).copy(), p.off.clone(), p.cnt.clone(), p.vis[0].clone())
    for _ in range(3):
        p.step()
    torch.cuda.synchronize()
    assert fhv.fhv_get_count(p.pofl)[1] == n
    assert (fhv.records_to_numpy(p.pofa, n) == first[0]).all()
    assert torch.equal(p.off, first[1]) and torch.equal(p.cnt, first[2]) and torch.equal(p.vis[0], first[3])
