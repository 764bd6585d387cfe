"""Repeated end-to-end steps with the read-back of one step overlapping the
next (pipeline.StreamingSteps): every step's images and fragment count reach
host memory and equal a plain step's."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv, scenes  # noqa: E402
from paper_2211_15460_gb300.pipeline import PlainFHV, StreamingSteps  # noqa: E402


def test_streaming_steps_match_a_plain_step():
    w = scenes.workload_spheres_256()
    p = PlainFHV(w)
    p.step()
    torch.cuda.synchronize()
    ref = [t.cpu().clone() for t in p.rgba]
    n = fhv.fhv_get_count(p.pofl)[1]
    ss = StreamingSteps(p)
    assert ss.h2d_bytes > 0 and ss.d2h_bytes == sum(t.numel() * 4 for t in ref) + 16
    slots = [ss.step() for _ in range(5)]
    ss.finish()
    torch.cuda.synchronize()
    assert slots == [0, 1, 0, 1, 0]
    for s in (0, 1):
        for h, r in zip(ss.host_out[s], ref):
            assert torch.equal(h, r)
        assert int(ss.count_host[s][0]) == n


def test_streaming_pofa_steps_match_a_plain_step(oracle_mod):
    """The headline pipeline (records-only capture, POFA compaction, every view
    in one batched call) on the sphere workload captured along three axes:
    one plain step's images equal the oracle's render of its POFA, and
    streaming steps (scene uploaded, images read back, alternating device
    sets) give the same images and fragment count."""
    import numpy as np

    from paper_2211_15460_gb300.pipeline import PofaViews, StreamingPofaSteps

    w = scenes.workload_spheres_256()
    w.views = [scenes.orbit_camera(w.scene, 96, 64, orbit_deg=d) for d in (0.0, 40.0, 200.0)]
    p = PofaViews(w)
    p.step()
    torch.cuda.synchronize()
    ref = [t.cpu().clone() for t in p.views.rgba]
    rec = oracle_mod.fragments(w.scene, oracle_mod.AXIS3, None, w.normal_pitch)[0]
    assert p.n == rec.size
    pofa = oracle_mod.pofa_sort(rec)
    assert (fhv.records_to_numpy(p.pofa, p.n) == pofa).all()
    for cam, r in zip(w.views, ref):
        vis_o, rgba_o = oracle_mod.render(pofa, w.scene, cam, w.lights, w.footprint_k)
        assert np.abs(r.numpy().reshape(-1, 4) - rgba_o).max() < 1e-4
    ss = StreamingPofaSteps(p)
    assert ss.h2d_bytes > 0 and ss.d2h_bytes == sum(t.numel() * 4 for t in ref) + 16
    slots = [ss.step() for _ in range(4)]
    ss.finish()
    torch.cuda.synchronize()
    assert slots == [0, 1, 0, 1]
    for s in (0, 1):
        for h, r in zip(ss.host_out[s], ref):
            assert torch.equal(h, r)
        assert int(ss.count_host[s][0]) == p.n
