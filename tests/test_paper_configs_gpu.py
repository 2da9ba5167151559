"""The paper's own validation configurations on the CUDA path.

- Steady stratified channel (the Ba test; Sec. 4, App. D): walls, the heavy
  fluid in the middle half, Lambda = 8 (alpha_B = 0.2, alpha_R = 0.9),
  nu = 0.333, pressure-driven, App. B's order-6 colour gradient.  The GPU
  path matches the FP64 oracle on this configuration, and its steady state
  is compared with App. D's Simpson-rule solution for the density profile
  the lattice carries (Eq. equ_integral).
- Micro-currents of a static red drop (Sec. 4.2, Tables tab_micro1 and
  tab_micro2): radius 60 on 200 x 200, Lambda from 1e-3 to 1e3, curvature
  computed (K = div n-hat) or fixed (K = 1/R).  The GPU path matches the
  oracle on a 64 x 64 replica at the extreme density ratios; the full-size
  table is produced on the GPU as context (the paper does not print sigma,
  beta or nu for it).

Full-size results are written as JSON to the files named by the environment
variables CMRT_BA_JSON and CMRT_MICRO_JSON, if set.
"""
import json
import os

import numpy as np
import pytest

from oracle import analytic as A
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()


def _errs(g, f):
    out = {}
    for k in ("rho_r", "rho_b"):
        out[k] = np.abs(g[k] - f[k]).max() / np.abs(f[k]).max()
    uref = max(np.abs(np.stack([f["ux"], f["uy"]])).max(), 0.01)
    for k in ("ux", "uy"):
        out[k] = np.abs(g[k] - f[k]).max() / uref
    return out


def _parity(d, rn, u, nsteps=100):
    """GPU against the FP64 oracle after nsteps, in the parity-bar norms, with
    the bar: 1e-5, or for u five times the FP32 storage floor where that is
    higher.  The floor is the oracle's own error when its state is rounded to
    FP32 after every step; a light fluid's velocity is resolved only to the
    FP32 spacing of its populations over its density, which in the light
    phases of these configurations (rho = 0.125, and 0.001 at Lambda = 1000)
    puts the floor at 2.4e-6 .. 6.2e-6, and the kernel's FP32 arithmetic adds
    rounding of the same order (2.4 to 4.4 times the floor, measured; the
    static drop's 6.3e-6 is 2.4 times its 2.6e-6)."""
    p = O.Params(**d)
    R0, B0 = O.init_state(rn, u[0], u[1], p)
    R, B = O.run(R0, B0, p, nsteps)
    to32 = lambda X: X.astype(np.float32).astype(np.float64)
    Rq, Bq = to32(R0), to32(B0)
    for _ in range(nsteps):
        Rq, Bq = O.step(Rq, Bq, p)
        Rq, Bq = to32(Rq), to32(Bq)
    ref = O.fields(R, B, p)
    floor = _errs(O.fields(Rq, Bq, p), ref)
    lat = cm.Lattice(d, rn, u)
    lat.step(nsteps)
    got = _errs({k: v.double().cpu().numpy() for k, v in lat.fields().items()}, ref)
    lat.close()
    for k in ("rho_r", "rho_b"):
        assert got[k] <= 1e-5, (k, got[k])
    ubar = max(1e-5, 5.0 * max(floor["ux"], floor["uy"]))
    for k in ("ux", "uy"):
        assert got[k] <= ubar, (k, got[k], ubar)


def _ba_start(d, rn):
    """The channel starts from App. D's profile for its initial density, so that
    the run only has to relax the interfaces' diffuse structure."""
    rho = d["rho0_r"] * (1 + rn[:, 0]) / 2 + d["rho0_b"] * (1 - rn[:, 0]) / 2
    nu = A.nu_of_lambda3(d["lambda3_r"])
    ux = A.app_d_steady(rho, nu, d["g_vol"][0])
    u = np.zeros((2,) + rn.shape)
    u[0] = ux[:, None]
    return u


@pytest.mark.parametrize("order", [6, 2])
def test_ba_channel_matches_oracle(order):
    d, rn, _ = I.ba_channel(stencil_order=order)
    _parity(d, rn, _ba_start(d, rn))


@pytest.mark.slow
def test_ba_channel_steady_state_against_app_d():
    """80k steps (over six e-folding times nu pi^2 / H^2 of the slowest mode):
    the velocity profile against App. D's solution for the simulated density.
    Sec. 4 reports agreement from a figure only; the bound is the error this
    scheme reaches (5.1 % of the peak velocity with App. B's stencil and
    beta = 0.67, against 12.7 % with the compact stencil, measured), and App.
    B's stencil must beat the compact one, as Sec. 4 found it necessary here."""
    out = {}
    for order in (6, 2):
        d, rn, _ = I.ba_channel(stencil_order=order)
        u = _ba_start(d, rn)
        lat = cm.Lattice(d, rn, u)
        lat.step(80_000)
        f = {k: v.double().cpu().numpy() for k, v in lat.fields().items()}
        lat.close()
        rho = (f["rho_r"] + f["rho_b"])[:, 0]
        ref = A.app_d_steady(rho, A.nu_of_lambda3(d["lambda3_r"]), d["g_vol"][0])
        ux = f["ux"][:, 0]
        err = float(np.abs(ux - ref).max() / ref.max())
        out[order] = {"max_rel_err": err, "u_peak": float(ref.max()),
                      "asymmetry": float(np.abs(ux - ux[::-1]).max() / ref.max())}
        assert np.isfinite(err)
    path = os.environ.get("CMRT_BA_JSON")
    if path:
        with open(path, "w") as fh:
            json.dump({"workload": "Ba channel H = 200, Lambda = 8, nu = 0.333, 80k steps", "orders": out}, fh,
                      indent=1)
    assert out[6]["max_rel_err"] <= 0.06
    assert out[6]["max_rel_err"] < out[2]["max_rel_err"]
    assert out[6]["asymmetry"] <= 1e-3


@pytest.mark.parametrize("Lam", I.MICRO_CURRENT_LAMBDAS)
@pytest.mark.parametrize("fixed", [False, True], ids=["computed_K", "fixed_K"])
def test_micro_current_replica_matches_oracle(Lam, fixed):
    """64 x 64 replica of the micro-current drop (radius 0.3 of the box, as
    60 / 200), 100 steps, at every density ratio of the tables.  The centre
    sits off the lattice nodes: at a drop centred on a node the colour
    gradient there is zero in exact arithmetic, so the FP64 oracle leaves n
    at 0 (below the threshold of the unit normal) while FP32 rounding leaves
    a gradient of a few ulps whose direction is noise, and the two runs part
    at that node by more than rounding (u 9.4e-5 at Lambda = 100 against
    6.8e-6 off the node)."""
    d, rn, u = I.micro_current_drop(Lam, n=64, radius=19.2, fixed_K=fixed, centre=(32.3, 31.8))
    _parity(d, rn, u)


@pytest.mark.slow
def test_micro_current_table():
    """Sec. 4.2's study on the GPU: |u|_max after 200k steps (over 30 e-folding
    times of the box's slowest shear mode, so that the initial transient has
    died out) for each Lambda of
    the tables, with K computed and with K = 1/R.  Context, not a target: the
    paper's sigma, beta and nu are not printed.  Checked: every run stays
    finite and the fixed curvature lowers the micro-current wherever the
    curvature error dominates it (Lambda = 0.1 and 10), the signature the
    paper reports."""
    table = {}
    for Lam in I.MICRO_CURRENT_LAMBDAS:
        row = {}
        for fixed in (False, True):
            d, rn, u = I.micro_current_drop(Lam, fixed_K=fixed)
            lat = cm.Lattice(d, rn, u)
            lat.step(200_000)
            f = lat.fields()
            umax = float(torch.sqrt(f["ux"] ** 2 + f["uy"] ** 2).max())
            lat.close()
            assert np.isfinite(umax), (Lam, fixed)
            row["fixed_K" if fixed else "computed_K"] = umax
        table[str(Lam)] = row
    path = os.environ.get("CMRT_MICRO_JSON")
    if path:
        with open(path, "w") as fh:
            json.dump({"workload": "red drop R = 60, 200 x 200 periodic, sigma 0.005, beta 0.67, nu 1/6, "
                                   "200k steps; |u|_max", "table": table}, fh, indent=1)
    for Lam in ("0.1", "10.0"):
        assert table[Lam]["fixed_K"] < table[Lam]["computed_K"], (Lam, table[Lam])
