"""Host-memory transfers (cmrt_init inputs, cmrt_fields outputs, population
export and import) stage through the state buffer that does not hold the
current state.  These tests check that doing so never changes the state:
a run interleaved with host transfers equals an uninterrupted one, bit for
bit, for single lattices in FP32 and FP16 storage and for batch members."""

import numpy as np
import pytest

from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("graph_steps", [0, 4])
def test_host_transfers_leave_the_state_alone(precision, graph_steps):
    d, rn, u = I.static_drop(n=40, radius=10.0)
    d = dict(d, precision=precision)
    a = cm.Lattice(d, rn, u)  # host inputs
    b = cm.Lattice(d, torch.tensor(rn, dtype=torch.float32, device="cuda"),
                   torch.tensor(u, dtype=torch.float32, device="cuda"))
    for lat in (a, b):
        lat.set_graph_steps(graph_steps)
    assert torch.equal(a.populations(), b.populations())
    a.step(5)
    b.step(5)
    host = a.fields_host()
    dev = {k: v.cpu().numpy() for k, v in b.fields().items()}
    for k in dev:
        assert np.array_equal(host[k], dev[k]), k
    a.step(3)
    pops = np.empty((2, 9, d["ny"], d["nx"]), dtype=np.float32)
    cm.cmrt_get_populations(a.ctx, pops.ctypes.data)  # host destination
    a.step(4)
    b.step(7)
    assert torch.equal(a.populations(), b.populations())
    a.set_populations(pops)  # host source: back to time 8's populations
    b.set_populations(torch.from_numpy(pops).cuda())
    a.step(9)
    b.step(9)
    assert torch.equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_member_host_fields_leave_the_batch_alone():
    members = []
    for k, side in enumerate((32, 48)):
        d = I.base_params(side, side, rho0_r=1.0, rho0_b=0.2)
        rn = I.drops_field(side, side, [(side / 2.0, side / 2.0)], [side / 4.0])
        members.append((d, rn, I.velocity_noise(side, side, 1e-4, 30 + k)))
    a = cm.Batch(members)
    b = cm.Batch(members)
    a.step(3)
    b.step(3)
    host = a.member(1).fields_host()
    dev = {k: v.cpu().numpy() for k, v in b.member(1).fields().items()}
    for k in dev:
        assert np.array_equal(host[k], dev[k]), k
    a.step(5)
    b.step(5)
    for k in range(2):
        assert torch.equal(a.member(k).populations(), b.member(k).populations()), k
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pinned_host_buffers_are_read_and_written_in_place(precision):
    """Page-locked host memory is accessed by the kernels directly (no
    staging copy); the results equal the device-buffer path bit for bit."""
    d, rn, u = I.static_drop(n=48, radius=12.0)
    d = dict(d, precision=precision)
    h_rn = torch.tensor(rn, dtype=torch.float32).pin_memory()
    h_u = torch.tensor(u, dtype=torch.float32).pin_memory()
    a = cm.Lattice(d, h_rn, h_u)
    b = cm.Lattice(d, h_rn.cuda(), h_u.cuda())
    assert torch.equal(a.populations(), b.populations())
    a.step(6)
    b.step(6)
    outs = [torch.empty((d["ny"], d["nx"]), dtype=torch.float32).pin_memory() for _ in range(5)]
    cm.cmrt_fields(a.ctx, *(o.data_ptr() for o in outs))
    ref = b.fields()
    for o, k in zip(outs, ("rho_r", "rho_b", "ux", "uy", "p")):
        assert torch.equal(o, ref[k].cpu()), k
    pops = torch.empty((2, 9, d["ny"], d["nx"]), dtype=torch.float32).pin_memory()
    cm.cmrt_get_populations(a.ctx, pops.data_ptr())
    assert torch.equal(pops, b.populations().cpu())
    a.step(3)
    cm.cmrt_set_populations(a.ctx, pops.data_ptr())  # back to time 6
    b.set_populations(pops.cuda())  # (16-bit storage re-encodes: not the identity)
    a.step(5)
    b.step(5)
    assert torch.equal(a.populations(), b.populations())
    a.close()
    b.close()

