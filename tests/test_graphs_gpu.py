"""Steps replayed from recorded CUDA graphs (cmrt_set_graph_steps, default
32 steps per graph) against steps launched one by one: the same kernels on the same buffers, so every
result must be bit-identical -- populations, time, launch counts, the
non-finite check at diag_every boundaries and the adjoint's forward run."""
import numpy as np
import pytest

from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()


def _cases():
    d0, rn0, u0 = I.static_drop(n=32, radius=8.0)
    d1, rn1, u1 = I.layered_channel(nx=40, ny=24)
    d2, rn2, u2 = I.layered_channel(nx=30, ny=20)
    d2 = dict(d2, stencil_order=6)
    d3, rn3, u3 = I.static_drop(n=36, radius=9.0)
    d3 = dict(d3, precision=2)
    return [("periodic", d0, rn0, u0), ("walls", d1, rn1, u1), ("order6_walls", d2, rn2, u2),
            ("fp16", d3, rn3, u3)]


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("graph_steps", [2, 4, 32])
def test_graph_steps_bit_identical(case, graph_steps):
    name, d, rn, u = case
    d = dict(d, diag_every=10)
    a = cm.Lattice(d, rn, u)
    a.set_graph_steps(0)
    b = cm.Lattice(d, rn, u)
    b.set_graph_steps(graph_steps)
    assert b.graph_steps == graph_steps
    for n in (1, 37, 6, 64):  # odd counts change the buffer parity between calls
        a.step(n)
        b.step(n)
        assert a.time == b.time
        assert a.launches == b.launches
        assert torch.equal(a.populations(), b.populations()), (name, n)
    a.close()
    b.close()


def test_graph_steps_rejects_odd_and_negative_counts():
    d, rn, u = I.static_drop(n=32, radius=8.0)
    lat = cm.Lattice(d, rn, u)
    for bad in (3, -2):
        with pytest.raises(cm.CmrtError) as ei:
            lat.set_graph_steps(bad)
        assert ei.value.status == cm.CMRT_EINVAL
    assert lat.graph_steps == 32  # the default stays
    lat.step(2)  # the context stays usable
    lat.close()


def test_nonfinite_state_is_reported_through_graphs():
    d, rn, u = I.static_drop(n=32, radius=8.0)
    d["diag_every"] = 8
    lat = cm.Lattice(d, rn, u)
    lat.set_graph_steps(4)
    pops = lat.populations().cpu().numpy()
    pops[1, 3, 7, 9] = np.nan
    lat.set_populations(pops)
    with pytest.raises(cm.CmrtError) as ei:
        lat.step(16)
    assert ei.value.status == cm.CMRT_ENONFINITE
    assert lat.time == 8  # the check after the first two graphs caught it
    lat.close()


def test_adjoint_forward_run_through_graphs_is_identical():
    n = 32
    d = I.base_params(n, n, rho0_r=1.0, rho0_b=0.1, g_acc=(0.0, -1e-5))
    rn = I.drops_field(n, n, [(16.0, 16.0)], [8.0], dtype=np.float32)
    t = cm.Lattice(dict(d, sigma=1.05 * d["sigma"]), rn, None)
    t.step(30)
    f = t.fields()
    a_, b_ = f["rho_r"] / d["rho0_r"], f["rho_b"] / d["rho0_b"]
    target = ((a_ - b_) / (a_ + b_)).contiguous()
    t.close()
    out = []
    for gs in (0, 4):
        lat = cm.Lattice(d, rn, None)
        lat.set_graph_steps(gs)
        J, g, grn = lat.adjoint(30, target, ckpt_every=10, want_rho_n0=True)
        out.append((J, g, grn.cpu(), lat.launches, lat.populations().cpu()))
        lat.close()
    (J0, g0, r0, l0, p0), (J1, g1, r1, l1, p1) = out
    assert J0 == J1 and g0 == g1 and l0 == l1
    assert torch.equal(r0, r1) and torch.equal(p0, p1)
