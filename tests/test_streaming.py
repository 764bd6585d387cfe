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
