"""cmrt_diagnostics_noalloc: diagnostics of caller-owned device populations
with no allocation (for callers recording a CUDA graph, running under a
device-memory cap, or that must not let cudaMalloc synchronise the device).

Called through the C ABI and checked against the context-based
cmrt_diagnostics on the same state, on two calls in a row.  This file sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402


def _agree(a, b):
    # same FP32 values reduced in FP64: masses and momentum to round-off, max |u| exactly
    assert abs(a[0] - b[0]) <= 1e-12 * abs(b[0])
    assert abs(a[1] - b[1]) <= 1e-12 * abs(b[1])
    assert abs(a[2] - b[2]) <= 1e-9 * abs(b[0])
    assert abs(a[3] - b[3]) <= 1e-9 * abs(b[0])
    assert abs(a[4] - b[4]) <= 1e-7 * max(abs(b[4]), 1e-12)
    assert a[5] == b[5] == 0


@pytest.mark.parametrize("wall", [False, True])
def test_noalloc_diagnostics_match_context_diagnostics_twice(wall):
    d, rn, u = I.static_drop(n=96, radius=20.0)
    d["wall_y"] = wall
    d["g_acc"] = (2e-5, -1e-5)
    lat = cm.Lattice(d, rn, u)
    params = cm.make_params(d)
    stream = torch.cuda.current_stream().cuda_stream
    for nsteps in (5, 7):  # two calls in a row, on two different states
        lat.step(nsteps)
        pops = lat.populations()
        ref = cm.cmrt_diagnostics(lat.ctx)
        got = cm.cmrt_diagnostics_noalloc(params, pops.data_ptr(), stream)
        _agree(got, ref)
    lat.close()


def test_noalloc_rejects_host_memory():
    d, _, _ = I.static_drop(n=16, radius=4.0)
    params = cm.make_params(d)
    host = np.zeros((2, 9, 16, 16), dtype=np.float32)
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_diagnostics_noalloc(params, host.ctypes.data)
    assert ei.value.status == cm.CMRT_EINVAL
