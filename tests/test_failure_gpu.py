"""Failure paths that are visible on the host only: an allocation that the
device cannot satisfy (CMRT_ENOMEM) and the state of the library after it.
No GPU fault is provoked."""
import ctypes

import pytest

from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()


def test_init_too_large_for_the_device_returns_enomem():
    """A lattice whose two state buffers exceed the device memory: cmrt_init
    returns CMRT_ENOMEM, hands back no context and frees what it took (the
    failure is an ordinary cudaMalloc error, visible on the host only)."""
    free0, total = torch.cuda.mem_get_info()
    side = int((2 * total / 72) ** 0.5) + 1  # one state buffer alone is larger than the device
    d = I.base_params(side, side)
    params = cm.make_params(d)
    h = ctypes.c_void_p(1)
    st = cm.load().cmrt_init(ctypes.byref(params), None, None, None, ctypes.byref(h))
    assert st == cm.CMRT_ENOMEM
    assert h.value is None
    assert "cudaMalloc" in cm.load().cmrt_last_error(None).decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)
    # the device stays usable: a small lattice initialises and steps
    d, rn, u = I.static_drop(n=16, radius=4.0)
    lat = cm.Lattice(d, rn, u)
    lat.step(2)
    lat.close()
