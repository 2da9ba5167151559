"""App. B's order-6 gradient stencil (stencil_order = 6) on the GPU against the
FP64 oracle, whose order-6 gradient is pinned by tests/golden/app_b_stencil.txt
and the polynomial-exactness tests of tests/test_oracle_identities.py.

The order-6 step runs as plane passes (cmrt_planes.cu); the bars are those of
the compact step: populations element by element at 2e-6 of the largest after
3 steps, fields at 1e-5 after 100 steps, colour-mass drift 1e-6.
"""
import zlib

import numpy as np
import pytest

from oracle import cmrt_adjoint as A
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()

CASES = [
    ("periodic40x32", 40, 32, False, {}),
    ("walls37x29_gravity", 37, 29, True, {"g_acc": (2e-5, -1e-5)}),
    ("walls130x3", 130, 3, True, {}),
    ("tiny5x4", 5, 4, False, {}),
    ("visc_eta_walls", 48, 20, True, {"visc_mode": 1, "eta": 0.2}),
    ("lambda100", 64, 24, False, {"rho0_b": 0.01, "sigma": 0.02}),
]


@pytest.mark.parametrize("name,nx,ny,wall,extra", CASES, ids=[c[0] for c in CASES])
def test_order6_steps_match_oracle_elementwise(name, nx, ny, wall, extra):
    rn, u = I.random_state_fields(nx, ny, seed=zlib.crc32(name.encode()) % 1000)
    extra = dict(extra)
    rho0_b = extra.pop("rho0_b", 0.1)
    d = I.base_params(nx, ny, rho0_r=1.0, rho0_b=rho0_b, wall_y=wall, stencil_order=6, **extra)
    p = O.Params(**d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 3)
    lat = cm.Lattice(d, rn, u)
    lat.step(3)
    got = lat.populations().double().cpu().numpy()
    lat.close()
    ref = np.stack([R, B])
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


def test_order6_differs_from_compact():
    """Guards against the compact stencil running in place of App. B's."""
    d, rn, u = I.static_drop(n=32, radius=8.0)
    a = cm.Lattice(d, rn, u)
    b = cm.Lattice(dict(d, stencil_order=6), rn, u)
    a.step(5)
    b.step(5)
    diff = (a.populations() - b.populations()).abs().max().item()
    a.close()
    b.close()
    assert diff > 1e-5, diff


def test_order6_static_drop_100_steps_parity_bar():
    d, rn, u = I.static_drop()
    d["stencil_order"] = 6
    p = O.Params(**d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 100)
    lat = cm.Lattice(d, rn, u)
    d0 = lat.diagnostics()
    lat.step(100)
    g = {k: v.double().cpu().numpy() for k, v in lat.fields().items()}
    d1 = lat.diagnostics()
    lat.close()
    f = O.fields(R, B, p)
    for k in ("rho_r", "rho_b", "p"):
        assert np.abs(g[k] - f[k]).max() / np.abs(f[k]).max() <= 1e-5, k
    uref = max(np.abs(np.stack([f["ux"], f["uy"]])).max(), 0.01)
    for k in ("ux", "uy"):
        assert np.abs(g[k] - f[k]).max() / uref <= 1e-5, k
    assert abs(d1["mass_r"] - d0["mass_r"]) / d0["mass_r"] <= 1e-6
    assert abs(d1["mass_b"] - d0["mass_b"]) / d0["mass_b"] <= 1e-6
    ref = O.diagnostics(R, B, p)
    assert abs(d1["umax"] - ref["umax"]) <= 1e-5 * max(ref["umax"], 0.01)


def test_order6_step_vjp_matches_oracle():
    nx, ny = 36, 22
    d = I.base_params(nx, ny, sigma=0.01, wall_y=True, g_acc=(1e-4, -2e-4), stencil_order=6)
    p = O.Params(**d)
    rng = np.random.default_rng(3)
    rn = I.drops_field(nx, ny, [(nx / 2 + 0.3, ny / 2 - 0.2)], [6.5], periodic_y=False)
    u = rng.uniform(-0.02, 0.02, size=(2, ny, nx))
    R, B = O.step(*O.init_state(rn, u[0], u[1], p), p)
    R, B = R.astype(np.float32), B.astype(np.float32)
    lat = cm.Lattice(d, None, None)
    lat.set_populations(np.stack([R, B]))
    lam_next = rng.standard_normal((2, 9, ny, nx)).astype(np.float32)
    got, g = lat.step_vjp(lam_next)
    lat.close()
    lR, lB, gref = A.step_vjp(R.astype(np.float64), B.astype(np.float64), lam_next[0].astype(np.float64),
                              lam_next[1].astype(np.float64), p)
    ref = np.stack([lR, lB])
    err = np.abs(got.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 2e-5, err
    gmax = max(abs(v) for v in gref.values())
    for k, name in enumerate(cm.ADJOINT_PARAMS):
        assert abs(g[k] - gref[name]) <= 1e-4 * abs(gref[name]) + 1e-6 * gmax, (name, g[k], gref[name])
