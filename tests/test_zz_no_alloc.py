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


def _device_pops(n=16):
    return torch.zeros((2, 9, n, n), dtype=torch.float32, device="cuda")


def test_noalloc_rejects_misaligned_pointer():
    """nx a multiple of 4: the pass copies 16-byte chunks, so a base address
    4 bytes into a tensor is refused on the host, before any launch."""
    d, _, _ = I.static_drop(n=16, radius=4.0)
    params = cm.make_params(d)
    buf = torch.zeros(2 * 9 * 16 * 16 + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_diagnostics_noalloc(params, buf.data_ptr() + 4)
    assert ei.value.status == cm.CMRT_EINVAL
    assert "aligned" in str(ei.value)


def test_noalloc_rejects_lattice_wider_than_scratch():
    """983,041 columns need 8193 column strips, one more than the scratch area
    holds: refused before the launch (the pointer is never read)."""
    d = I.base_params(983_041, 1)
    params = cm.make_params(d)
    pops = _device_pops()
    with pytest.raises(cm.CmrtError) as ei:
        cm.cmrt_diagnostics_noalloc(params, pops.data_ptr())
    assert ei.value.status == cm.CMRT_EINVAL
    assert "strips" in str(ei.value)
    # the widest accepted lattice passes the same checks (one row, 983,040 columns)
    d = I.base_params(983_040, 1)
    d["wall_y"] = False
    wide = torch.zeros((2, 9, 1, 983_040), dtype=torch.float32, device="cuda")
    wide[0, 0] = 1.0
    wide[1, 0] = 0.1
    out = cm.cmrt_diagnostics_noalloc(cm.make_params(d), wide.data_ptr())
    assert out[0] == pytest.approx(983_040.0)
    assert out[1] == pytest.approx(98_304.0)


def test_noalloc_rejects_capturing_stream():
    """The call waits for its stream, which a stream recording a CUDA graph
    does not allow: it is refused with nothing enqueued, and the caller's
    capture ends normally."""
    d, _, _ = I.static_drop(n=16, radius=4.0)
    params = cm.make_params(d)
    pops = _device_pops()
    x = torch.zeros(4, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        with pytest.raises(cm.CmrtError) as ei:
            cm.cmrt_diagnostics_noalloc(params, pops.data_ptr(), side.cuda_stream)
    assert ei.value.status == cm.CMRT_EINVAL
    assert "capturing" in str(ei.value)
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
