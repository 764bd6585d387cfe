"""Failure detection without a fault: every kind of bounded device wait the
library uses (the scans' decoupled look-back, the bulk copies' mbarrier wait,
the tensor-core kernels' mbarrier wait) is run on a condition that nothing
satisfies. Each must give up within its bound, report FHV_DEV_TIMEOUT
through the workspace status (fhv_read_status -> FHV_ERR_TIMEOUT), and leave
the context usable: a normal build and render after it still match the
results taken before it."""
import time

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2211_15460_gb300 import fhv, scenes  # noqa: E402
from paper_2211_15460_gb300.pipeline import PlainFHV  # noqa: E402


def _step(p):
    p.step()
    torch.cuda.synchronize()
    n = fhv.fhv_get_count(p.pofl)[1]
    return n, p.pofa[: 2 * n].clone(), p.vis[0].clone(), p.rgba[0].clone()


def test_bounded_waits_time_out_and_context_stays_usable():
    p = PlainFHV(scenes.workload_spheres_256())
    before = _step(p)
    ws = fhv.workspace(fhv.FHV_WAIT_PROBE_WS_BYTES)
    for kind in (0, 1, 2):
        t0 = time.time()
        fhv.fhv_wait_probe(kind, ws)
        st, bits = fhv.fhv_read_status(ws)
        dt = time.time() - t0
        assert st == fhv.FHV_ERR_TIMEOUT and bits & fhv.FHV_DEV_TIMEOUT, (kind, st, bits)
        assert dt < 30.0, (kind, dt)
        print(f"\nwait kind {kind}: gave up after {dt * 1e3:.1f} ms")
    after = _step(p)
    assert after[0] == before[0]
    for a, b in zip(after[1:], before[1:]):
        assert torch.equal(a, b)
