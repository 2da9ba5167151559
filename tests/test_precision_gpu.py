"""16-bit population storage (BF16 / FP16 deviations, FP32 arithmetic)
against the FP64 oracle and the FP32 path.

A record keeps rho_R, rho_B and the rest populations R_0, B_0 in FP32, four
16-bit reference dipoles per colour -- the equilibrium's velocity term and
the recolour's segregation term per link direction -- and the deviations
C_i - rho_C psi_i -/+ D_C of the moving links in 16 bits, so that for a
state the step wrote they are only the non-equilibrium and second-order
parts of the populations.  Reference psi_i: phi_i of Eq. eq_phi at the
node's own mixture (precision_reference 0, the default), the lattice
weights w_i (1) or phi_i of the pure colour (2).  Bars (relative field
error, u normalised by max(|u_ref|, 0.01)), FP16 and BF16 with the mixture
reference: 1e-4 in rho_R and rho_B and 3e-4 in u, ten and three times
tighter than the target of 1e-3 and within three times of the FP32 path's
own error on the 512^2 replica (1.0e-4 in u after 2000 steps).
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
RHO_BAR = {FP16: 1e-4, BF16: 1e-4}
U_BAR = {FP16: 3e-4, BF16: 3e-4}


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


@pytest.mark.parametrize("prec", [FP16, BF16])
@pytest.mark.parametrize("nx,ny,wall", [(130, 140, True), (33, 17, False), (250, 36, False)],
                         ids=["walls130x140", "ragged33x17", "ragged250x36"])
def test_ragged_lattices_100_steps(prec, nx, ny, wall):
    """Widths that are not a multiple of 4 (each thread copies its own column
    of every plane, no 16-byte chunks), strips that end inside a window, and
    walls: a drop with a velocity field, 100 steps against the FP64 oracle at
    the 16-bit bars."""
    d = I.base_params(nx, ny, rho0_r=1.0, rho0_b=0.1, sigma=0.01, wall_y=wall, g_acc=(1e-5, -1e-5))
    r = max(3.0, min(nx, ny) / 4.0)
    rn = I.drops_field(nx, ny, [(nx / 2.0 + 0.3, ny / 2.0 - 0.2)], [r], periodic_y=not wall)
    u = I.velocity_noise(nx, ny, 1e-3, 21)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 100)
    lat = cm.Lattice(dict(d, precision=prec), rn, u)
    lat.step(100)
    errs = _field_errs(lat, p, R, B)
    lat.close()
    _check(errs, prec)


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
def test_buoyant_replica_512_2000_steps():
    """The 512 x 512 replica of the 16384 x 8192 buoyant field (same seeded
    generator, drop count scaled by area), 2000 steps of FP32, FP16 and BF16
    storage against the FP64 oracle; the oracle cannot run the full 10k
    steps within a test.  The errors (FP32 as the floor the 16-bit forms sit
    on) are written as JSON to the file named by CMRT_ACCURACY512_JSON, if
    set."""
    d, rn, u = I.buoyant_replica(side=512)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 2000)
    table, drift = {}, {}
    for name, prec in (("fp32", 0), ("fp16", FP16), ("bf16", BF16)):
        lat = cm.Lattice(dict(d, precision=prec), rn, u)
        m0 = lat.diagnostics()
        lat.step(2000)
        table[name] = _field_errs(lat, p, R, B)
        m1 = lat.diagnostics()
        lat.close()
        drift[name] = {"mass_r": abs(m1["mass_r"] - m0["mass_r"]) / m0["mass_r"],
                       "mass_b": abs(m1["mass_b"] - m0["mass_b"]) / m0["mass_b"]}
    import json
    import os
    out = os.environ.get("CMRT_ACCURACY512_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump({"workload": "buoyant replica 512x512, walls, g = 1e-6, 2000 steps",
                       "errors": table, "mass_drift": drift}, fh, indent=1)
    for name, prec in (("fp16", FP16), ("bf16", BF16)):
        _check(table[name], prec)
        assert drift[name]["mass_r"] <= 1e-5 and drift[name]["mass_b"] <= 1e-5


@pytest.mark.slow
@pytest.mark.skipif(not __import__("os").environ.get("CMRT_LONG"),
                    reason="the FP64 oracle needs about 11 minutes for 10k steps at 512^2; set CMRT_LONG=1")
def test_buoyant_replica_512_10k_steps():
    """The 16384 x 8192 buoyant field's error measure as the target statement
    puts it: 10k steps on the 512 x 512 replica against the FP64 oracle, for
    FP32, FP16 and BF16 storage.  Held to the target's 1e-3 for the 16-bit
    forms; the errors are written as JSON to the file named by
    CMRT_ACCURACY10K_JSON, if set."""
    d, rn, u = I.buoyant_replica(side=512)
    p = _oracle_params(d)
    R, B = O.run(*O.init_state(rn, u[0], u[1], p), p, 10_000)
    table = {}
    for name, prec in (("fp32", 0), ("fp16", FP16), ("bf16", BF16)):
        lat = cm.Lattice(dict(d, precision=prec), rn, u)
        m0 = lat.diagnostics()
        lat.step(10_000)
        table[name] = _field_errs(lat, p, R, B)
        m1 = lat.diagnostics()
        lat.close()
        table[name]["mass_drift_r"] = abs(m1["mass_r"] - m0["mass_r"]) / m0["mass_r"]
        table[name]["mass_drift_b"] = abs(m1["mass_b"] - m0["mass_b"]) / m0["mass_b"]
    import json
    import os
    out = os.environ.get("CMRT_ACCURACY10K_JSON")
    if out:
        with open(out, "w") as fh:
            json.dump({"workload": "buoyant replica 512x512, walls, g = 1e-6, 10k steps", "errors": table}, fh,
                      indent=1)
    for name in ("fp16", "bf16"):
        for k in ("rho_r", "rho_b", "ux", "uy"):
            assert table[name][k] <= 1e-3, (name, k, table[name][k])


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
