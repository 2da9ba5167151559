"""16-bit population storage (BF16 / FP16 deviations from rho_C psi_i, FP32
arithmetic) against the FP64 oracle and the FP32 path.

Reference psi_i: phi_i of Eq. eq_phi at the node's own mixture
(precision_reference 0, the default), the lattice weights w_i (1) or phi_i of
the pure colour (2).  Bars (relative field error, u normalised by
max(|u_ref|, 0.01)):

- FP16 with the mixture reference: 1e-3 in rho_R and rho_B, the target the
  storage form is held to; u has a floor of ~1.5e-3: the recolour term of
  Eq. eq_re_color makes the minority colour's populations anisotropic by
  beta phi_i rho_maj / rho (tens of percent of their own size), which no
  isotropic reference removes, and FP16 rounds that part to 2^-12 every
  step.  u is held to 3e-3.
- BF16 (8-bit significand) reaches ~1e-2 at best and is held to 3e-2: it
  cannot meet 1e-3 with any of the three references.
"""
import numpy as np
import pytest

from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

BF16, FP16 = 1, 2
MIX, WREF, PURE = 0, 1, 2
RHO_BAR = {FP16: 1e-3, BF16: 3e-2}
U_BAR = {FP16: 3e-3, BF16: 3e-2}


def _check(errs, prec):
    for k in ("rho_r", "rho_b"):
        assert errs[k] <= RHO_BAR[prec], (k, errs[k])
    for k in ("ux", "uy"):
        assert errs[k] <= U_BAR[prec], (k, errs[k])


def _field_errs(lat, p, R, B):
    g = {k: v.double().cpu().numpy() for k, v in lat.fields().items()}
    f = O.fields(R, B, p)
    out = {}
    for k in ("rho_r", "rho_b"):
        out[k] = np.abs(g[k] - f[k]).max() / np.abs(f[k]).max()
    uref = max(np.abs(np.stack([f["ux"], f["uy"]])).max(), 0.01)
    for k in ("ux", "uy"):
        out[k] = np.abs(g[k] - f[k]).max() / uref
    return out


@pytest.mark.parametrize("prec", [FP16, BF16])
@pytest.mark.parametrize("ref", [MIX, WREF, PURE])
def test_encode_decode_round_trip(prec, ref):
    nx, ny = 72, 40
    d = I.base_params(nx, ny, precision=prec, precision_reference=ref)
    rn, u = I.random_state_fields(nx, ny, seed=3, amplitude=0.02)
    p = O.Params(**{k: v for k, v in d.items() if k not in ("precision", "precision_reference")})
    R, B = O.init_state(rn, u[0], u[1], p)
    pops = np.stack([R, B]).astype(np.float32)
    lat = cm.Lattice(d)
    lat.set_populations(pops)
    back = lat.populations().cpu().numpy()
    lat.close()
    eps = 2.0 ** -11 if prec == FP16 else 2.0 ** -8
    # the error is a rounding of the deviation from rho_C psi_i, far below the population
    assert np.abs(back - pops).max() <= 2 * eps * np.abs(pops).max()


def _oracle_params(d):
    return O.Params(**{k: v for k, v in d.items() if k not in ("precision", "precision_reference")})


@pytest.mark.parametrize("prec", [FP16, BF16])
def test_static_drop_100_steps(prec):
    d, rn, u = I.static_drop()
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 100)
    lat = cm.Lattice(dict(d, precision=prec), rn, u)
    m0 = lat.diagnostics()
    lat.step(100)
    errs = _field_errs(lat, p, R, B)
    m1 = lat.diagnostics()
    lat.close()
    _check(errs, prec)
    # the stored densities absorb the deviations' rounding: colour mass drifts
    # only at the FP32 level, as with FP32 storage
    assert abs(m1["mass_r"] - m0["mass_r"]) / m0["mass_r"] <= 1e-6
    assert abs(m1["mass_b"] - m0["mass_b"]) / m0["mass_b"] <= 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("prec", [FP16, BF16])
def test_buoyant_replica_2000_steps(prec):
    d, rn, u = I.buoyant_replica(side=128)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 2000)
    lat = cm.Lattice(dict(d, precision=prec), rn, u)
    lat.step(2000)
    errs = _field_errs(lat, p, R, B)
    lat.close()
    _check(errs, prec)


@pytest.mark.slow
def test_fp16_buoyant_replica_512_2000_steps():
    """The 512 x 512 replica of the 16384 x 8192 buoyant field (same seeded
    generator, drop count scaled by area), 2000 steps of FP16 storage against
    the FP64 oracle; the oracle cannot run the full 10k steps within a test.
    The errors are written as JSON to the file named by CMRT_ACCURACY512_JSON,
    if set."""
    d, rn, u = I.buoyant_replica(side=512)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 2000)
    lat = cm.Lattice(dict(d, precision=FP16), rn, u)
    m0 = lat.diagnostics()
    lat.step(2000)
    errs = _field_errs(lat, p, R, B)
    m1 = lat.diagnostics()
    lat.close()
    drift = {"mass_r": abs(m1["mass_r"] - m0["mass_r"]) / m0["mass_r"],
             "mass_b": abs(m1["mass_b"] - m0["mass_b"]) / m0["mass_b"]}
    import json
    import os
    out = os.environ.get("CMRT_ACCURACY512_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump({"workload": "buoyant replica 512x512, walls, g = 1e-6, 2000 steps, FP16 storage",
                       "errors": errs, "mass_drift": drift}, fh, indent=1)
    _check(errs, FP16)
    assert drift["mass_r"] <= 1e-5 and drift["mass_b"] <= 1e-5


def test_fp16_close_to_fp32_on_full_size_field():
    """The reduced-precision form tracks the (oracle-checked) FP32 path on the
    16384 x 8192 buoyant field over 50 steps, within the FP16 bar."""
    d, rn, u = I.buoyant_drops()
    a = cm.Lattice(d, rn, u)
    b = cm.Lattice(dict(d, precision=FP16), rn, u)
    a.step(50)
    b.step(50)
    fa, fb = a.fields(), b.fields()
    a.close()
    b.close()
    for k in ("rho_r", "rho_b"):
        assert float((fa[k] - fb[k]).abs().max() / fa[k].abs().max()) <= RHO_BAR[FP16]
    uref = max(float(torch.stack([fa["ux"], fa["uy"]]).abs().max()), 0.01)
    for k in ("ux", "uy"):
        assert float((fa[k] - fb[k]).abs().max()) / uref <= U_BAR[FP16]


@pytest.mark.slow
def test_accuracy_table_buoyant_replica():
    """Per-field error of every storage form against the FP64 oracle on a
    128 x 128 replica of the buoyant-drops field after 2000 steps (the oracle
    cannot run the 512^2 x 10k replica within a test).  Written as JSON to
    the file named by the environment variable CMRT_ACCURACY_JSON, if set."""
    import json
    import os
    d, rn, u = I.buoyant_replica(side=128)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 2000)
    table = {}
    for name, prec, ref in (("fp32", 0, MIX), ("fp16", FP16, MIX), ("bf16", BF16, MIX), ("fp16_pure", FP16, PURE),
                            ("bf16_pure", BF16, PURE), ("fp16_wref", FP16, WREF), ("bf16_wref", BF16, WREF)):
        lat = cm.Lattice(dict(d, precision=prec, precision_reference=ref), rn, u)
        lat.step(2000)
        table[name] = _field_errs(lat, p, R, B)
        lat.close()
    assert max(table["fp32"].values()) <= 1e-4
    _check(table["fp16"], FP16)
    _check(table["bf16"], BF16)
    # the mixture reference is the most accurate of the three
    for prec in ("fp16", "bf16"):
        assert max(table[prec].values()) <= max(table[prec + "_pure"].values())
        assert max(table[prec].values()) <= max(table[prec + "_wref"].values())
    out = os.environ.get("CMRT_ACCURACY_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump({"workload": "buoyant replica 128x128, 1 drop, walls, g = 1e-6, 2000 steps",
                       "errors": table}, fh, indent=1)
