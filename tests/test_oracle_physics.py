"""Physics pins of the whole oracle step against what the paper and
continuum mechanics fix: conservation (Sec. 2, Eq. eq_re_color; App. A),
the Laplace law (Sec. 4.2), curvature of a circle, single-phase reductions
(shear-wave decay, Poiseuille flow, sound damping), the stationary flat
interface profile (Sec. 2, Eq. equ_rhoN) and the layered flows of App. C and
App. D, each within the error bound the paper states (Sec. 4.1: below 1 %).
"""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I


def _drop_state(n=64, radius=16.0, Lambda=10.0, noise=1e-6, seed=1, **kw):
    d, rn, u = I.static_drop(n=n, radius=radius, Lambda=Lambda, noise=noise, seed=seed)
    d.update(kw)
    p = O.Params(**d)
    R, B = O.init_state(rn, u[0], u[1], p)
    return p, R, B


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("wall", [False, True])
def test_colour_mass_conserved_to_roundoff(wall):
    """Collision conserves rho (lambda_0 = 0, S^(0) = 0), recolour conserves each
    colour (Sec. 2), streaming and bounce-back move populations: each colour
    mass is invariant, to FP64 round-off over 300 steps."""
    p, R, B = _drop_state(n=32, radius=8.0, g_acc=(0.0, -1e-5), wall_y=wall)
    d0 = O.diagnostics(R, B, p)
    R, B = O.run(R, B, p, 300)
    d1 = O.diagnostics(R, B, p)
    assert abs(d1["mass_r"] - d0["mass_r"]) <= 1e-13 * d0["mass_r"]
    assert abs(d1["mass_b"] - d0["mass_b"]) <= 1e-13 * d0["mass_b"]


def test_momentum_budget_equals_total_force():
    """App. A, Eq. moev: (rho u)+ = rho u + G (n = 1), recolour keeps f+, periodic
    streaming moves momentum: P(t+1) - P(t) = sum_r G(r, t) every step."""
    p, R, B = _drop_state(n=32, radius=8.0, g_acc=(3e-5, -1e-5), g_vol=(1e-6, 2e-6))
    for _ in range(5):
        d = O.macroscopic(R, B, p)
        P0 = np.array([d.jx.sum(), d.jy.sum()])
        Gsum = np.array([d.Gx.sum(), d.Gy.sum()])
        R, B = O.step(R, B, p)
        d1 = O.macroscopic(R, B, p)
        P1 = np.array([d1.jx.sum(), d1.jy.sum()])
        np.testing.assert_allclose(P1 - P0, Gsum, rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------- curvature, Laplace
def test_curvature_of_tanh_drop():
    """K = div n-hat (Sec. 2) of a radial profile is 1/r; at the interface of a
    drop of radius 16 the compact stencil gives 1/R within 5 %."""
    n, R0 = 64, 16.0
    p = O.Params(nx=n, ny=n)
    rn = I.drops_field(n, n, [(32.0, 32.0)], [R0])
    gx, gy = O.gradient(rn, p)
    nx_, ny_ = O.unit_normal(gx, gy, p)
    K = O.curvature(nx_, ny_, p)
    y, x = np.mgrid[0:n, 0:n]
    r = np.sqrt((x - 32.0) ** 2 + (y - 32.0) ** 2)
    ring = np.abs(r - R0) < 1.0
    np.testing.assert_allclose(K[ring].mean(), 1.0 / R0, rtol=0.05)
    # n-hat points outward for a red drop
    assert np.all((nx_ * (x - 32.0) + ny_ * (y - 32.0))[ring] > 0)


@pytest.mark.slow
def test_laplace_law_static_drop():
    """Sec. 4.2: the pressure step across a drop follows the Laplace law,
    in 2D dp = sigma / R.  Static drop, 64^2 periodic, Lambda = 10, 2000 steps;
    p = 3/5[(1-a_R) rho_R + (1-a_B) rho_B]; R from the area where rho^N > 0."""
    p, R, B = _drop_state()
    R, B = O.run(R, B, p, 2000)
    f = O.fields(R, B, p)
    rn = O.colour_index(f["rho_r"], f["rho_b"], p)
    Rm = np.sqrt((rn > 0).sum() / np.pi)
    y, x = np.mgrid[0:64, 0:64]
    d = np.sqrt((x - 32.0) ** 2 + (y - 32.0) ** 2)
    dp = f["p"][d < Rm - 4].mean() - f["p"][d > Rm + 4].mean()
    np.testing.assert_allclose(dp, p.sigma / Rm, rtol=0.05)


# ---------------------------------------------------------------- single-phase reductions
def _single_phase(nx, ny, alpha, lam3, **kw):
    return O.Params(nx=nx, ny=ny, rho0_r=1.0, rho0_b=1.0, alpha_r=alpha, alpha_b=alpha, sigma=0.0,
                    lambda3_r=lam3, lambda3_b=lam3, **kw)


@pytest.mark.parametrize("alpha,lam3", [(4 / 9, 1.0), (0.95, 1.0), (0.95, 1.4)])
def test_shear_wave_decay(alpha, lam3):
    """A shear wave decays as exp(-nu k^2 t) with nu = (2/lambda_3 - 1)/6 (App. A,
    after Eq. Correction), with or without the density-contrast equilibrium."""
    ny, U, n = 64, 1e-3, 800
    p = _single_phase(4, ny, alpha, lam3)
    k = 2 * np.pi / ny
    y = np.arange(ny)[:, None] * np.ones((1, 4))
    R, B = O.init_state(np.ones((ny, 4)), U * np.sin(k * y), 0 * y, p)
    R, B = O.run(R, B, p, n)
    ux = O.fields(R, B, p)["ux"][:, 0]
    s = np.sin(k * y[:, 0])
    amp = (ux * s).sum() / (s * s).sum()
    np.testing.assert_allclose(amp / U, A.shear_wave_amplitude(A.nu_of_lambda3(lam3), k, n), rtol=2e-3)


@pytest.mark.parametrize("lam3", [1.0, 1.5])
def test_poiseuille_half_way_bounce_back(lam3):
    """Body-force Poiseuille flow between half-way bounce-back walls matches the
    parabola u = f/(2 eta) s (H - s) (walls at y = -1/2 and ny - 1/2)."""
    ny, g = 32, 1e-6
    p = _single_phase(4, ny, 0.95, lam3, g_acc=(g, 0.0), wall_y=True)
    ref = A.poiseuille(ny, g, A.nu_of_lambda3(lam3))
    R, B = O.init_state(np.ones((ny, 4)), np.broadcast_to(ref[:, None], (ny, 4)), np.zeros((ny, 4)), p)
    R, B = O.run(R, B, p, 1500)
    f = O.fields(R, B, p)
    assert np.abs(f["ux"][:, 0] - ref).max() / ref.max() < 1.5e-3
    assert np.abs(f["uy"]).max() < 1e-14


@pytest.mark.parametrize("alpha", [4 / 9, 0.95])
def test_poiseuille_exact_with_tuned_ghost_rate(alpha):
    """With half-way bounce-back, a two-rate collision reproduces the Poiseuille
    parabola exactly when (1/lambda_even - 1/2)(1/lambda_odd - 1/2) = 3/16
    (Ginzburg's "magic" combination).  Here lambda_3 plays the even (stress)
    rate and Dellar's lambda_7 (J_x, J_y; App. A) the odd one: the discrete
    steady state must then equal f/(2 eta) s (H - s) to round-off.  This pins
    the force source (n = 1), the force-adjusted velocity u = (sum f c + G/2)/rho
    (m = 1/2, Eq. equ_constants), nu(lambda_3) and the bounce-back geometry."""
    ny, g, lam3 = 16, 1e-5, 0.7
    lam7 = 1.0 / (3.0 / 16.0 / (1.0 / lam3 - 0.5) + 0.5)
    p = _single_phase(4, ny, alpha, lam3, lambda7=lam7, g_acc=(g, 0.0), wall_y=True)
    ref = A.poiseuille(ny, g, A.nu_of_lambda3(lam3))
    R, B = O.init_state(np.ones((ny, 4)), np.broadcast_to(ref[:, None], (ny, 4)), np.zeros((ny, 4)), p)
    R, B = O.run(R, B, p, 2000)
    ux = O.fields(R, B, p)["ux"][:, 0]
    assert np.abs(ux - ref).max() / ref.max() < 1e-10


@pytest.mark.parametrize("alpha", [4 / 9, 0.95])
def test_sound_damping_of_printed_scheme(alpha):
    """Effect of the isotropic (1/3) rho div u term of Eqs. equ_T_identity and
    Correction, implemented as printed.  A Chapman-Enskog expansion of the
    scheme as printed (linear, single phase, c^2 = 3/5 (1 - alpha)) gives the
    viscous stress 2 rho nu S - 3 nu c^2 rho (div u) delta, so a sound wave of
    wavenumber k decays at rate nu k^2 (1 - 3 c^2 / 2): half the textbook LBM
    rate when alpha = 4/9, 0.955 of it when alpha = 0.95."""
    N = 64
    lam3 = 1.0
    p = _single_phase(N, 4, alpha, lam3)
    x = np.arange(N)[None, :] * np.ones((4, 1))
    k = 2 * np.pi / N
    rho_r = 1 + 1e-4 * np.cos(k * x)
    f0 = O.equilibrium(rho_r, 0 * rho_r, 0 * x, 0 * x, p)
    R, B = f0, 0 * f0
    c2 = 0.6 * (1 - alpha)
    n = 1500 if alpha < 0.5 else 3000
    amps = []
    cx = np.cos(k * x[0])
    for _ in range(n):
        rr = R.sum(0)[0]
        amps.append(((rr - 1) * cx).sum() / (cx * cx).sum())
        R, B = O.step(R, B, p)
    amps = np.abs(np.array(amps))
    pk = [i for i in range(1, n - 1) if amps[i] >= amps[i - 1] and amps[i] >= amps[i + 1]]
    rate = -np.polyfit(np.array(pk, float), np.log(amps[pk]), 1)[0]
    expect = A.nu_of_lambda3(lam3) * k * k * (1 - 1.5 * c2)
    np.testing.assert_allclose(rate, expect, rtol=0.015)


# ---------------------------------------------------------------- flat interface
@pytest.mark.parametrize("Lambda", [1.0, 10.0])
def test_flat_interface_stationary_profile(Lambda):
    """Sec. 2, Eq. equ_rhoN: a flat interface at rest is stationary with
    rho^N = tanh(beta' y).  At leading order the recolour flux with unit link
    vectors c-hat_i gives beta' = beta (2 + 1/sqrt 2)/3 (the diagonals carry
    1/sqrt 2); the paper's analysis, which neglects that factor, gives beta."""
    H, beta = 64, 0.3
    d = I.base_params(4, H, rho0_r=1.0, rho0_b=1.0 / Lambda, beta=beta, wall_y=True)
    p = O.Params(**d)
    y = np.arange(H)[:, None] * np.ones((1, 4))
    rn = np.tanh((H / 2 - 0.5 - y) / 2.0)
    R, B = O.init_state(rn, 0 * y, 0 * y, p)
    R, B = O.run(R, B, p, 2000)
    f = O.fields(R, B, p)
    rN = O.colour_index(f["rho_r"], f["rho_b"], p)[:, 0]
    k = np.where((rN[:-1] > 0) & (rN[1:] <= 0))[0][0]
    yc = k + rN[k] / (rN[k] - rN[k + 1])
    assert abs(yc - (H / 2 - 0.5)) < 0.05
    m = np.abs(rN) < 0.9
    slope = -np.polyfit(np.arange(H)[m], np.arctanh(rN[m]), 1)[0]
    np.testing.assert_allclose(slope, beta * (2 + 1 / np.sqrt(2)) / 3, rtol=0.02)


@pytest.mark.slow
def test_layered_steady_flow_app_d():
    """App. D generalised: steady flow through a continuous density profile,
    d/dy(eta du/dy) = -rho g, walls in y.  Lambda = 10, equal kinematic
    viscosities, beta = 0.3, App. B's high-order stencil (Sec. 4.1 found it
    necessary for this test).  Error below 1.5 % of max u."""
    H, g = 64, 1e-6
    d, rn, _ = I.layered_channel(nx=4, ny=H, Lambda=10.0, visc_ratio=1.0, g=g)
    d.update(beta=0.3, stencil_order=6)
    p = O.Params(**d)
    nu = A.nu_of_lambda3(p.lambda3_r)
    rho0 = p.rho0_r * (1 + rn[:, 0]) / 2 + p.rho0_b * (1 - rn[:, 0]) / 2
    start = A.layered_steady(rho0, np.full(H, nu), g_acc=g)
    R, B = O.init_state(rn, np.broadcast_to(start[:, None], rn.shape), 0 * rn, p)
    R, B = O.run(R, B, p, 2000)
    f = O.fields(R, B, p)
    rho = (f["rho_r"] + f["rho_b"])[:, 0]
    ref = A.layered_steady(rho, np.full(H, nu), g_acc=g)
    assert np.abs(f["ux"][:, 0] - ref).max() / ref.max() < 0.015


@pytest.mark.slow
@pytest.mark.parametrize("order,bound", [(6, 0.003), (2, 0.01)])
def test_layered_transient_app_c(order, bound):
    """App. C, flat interface: impulsively sheared two-layer flow, constant shear
    viscosity eta = 0.166, beta = 0.5, Lambda = 10, heavy fluid above; lattice
    relative error epsilon(t) of Eq. equ_aps_defn below the paper's 1 % bound
    at T = 1000 (Sec. 4.1) against the same PDE solved with the diffuse density
    profile the lattice carries."""
    H, T, eta, u0, Lam, beta = 400, 1000, 0.166, 1e-3, 10.0, 0.5
    d = I.base_params(4, H, rho0_r=1.0, rho0_b=1.0 / Lam, sigma=0.0, beta=beta, wall_y=True,
                      visc_mode=1, eta=eta, stencil_order=order)
    p = O.Params(**d)
    y = np.arange(H)[:, None] * np.ones((1, 4))
    h = H / 2.0 - 0.5
    rn = -I.layer_field(4, H, h, width=1.0 / beta)
    ux0 = np.where(y < h, u0, -u0)
    R, B = O.init_state(rn, ux0, 0 * y, p)
    f0 = O.fields(R, B, p)
    R, B = O.run(R, B, p, T)
    f = O.fields(R, B, p)
    rho = 0.5 * ((f0["rho_r"] + f0["rho_b"]) + (f["rho_r"] + f["rho_b"]))[:, 0]
    ua = A.layered_transient(rho, np.full(H, eta), ux0[:, 0], float(T))
    us = f["ux"][:, 0]
    eps = ((ua - us) ** 2).sum() / np.abs(us).max() ** 2
    assert eps < bound


def test_transient_references_agree():
    """The two independent App. C solutions (Sturm-Liouville series with the
    sharp interface; eigen-expansion of a fine discretisation) agree for a
    sharp profile, and the series reproduces App. C's single-fluid limit."""
    H, h = 200.0, 99.5
    s = np.arange(200) + 0.5
    rho = np.where(np.arange(200) < 100, 0.1, 1.0)
    u_init = np.where(np.arange(200) < 100, 1.0, -1.0)
    series = A.two_layer_transient(H, h + 0.5, 0.1, 1.0, 0.166, 0.166, 1.0, -1.0, s, 500.0, nmodes=300)
    fine = A.layered_transient(rho, np.full(200, 0.166), u_init, 500.0, refine=4)
    assert np.abs(series - fine).max() < 0.02
    # equal fluids: the series is the Fourier solution of the heat equation
    one = A.two_layer_transient(H, h + 0.5, 1.0, 1.0, 0.2, 0.2, 1.0, 1.0, s, 300.0, nmodes=300)
    ks = (2 * np.arange(300) + 1) * np.pi / H
    four = sum(4 / (np.pi * (2 * m + 1)) * np.exp(-0.2 * ks[m] ** 2 * 300.0) * np.sin(ks[m] * s) for m in range(300))
    assert np.abs(one - four).max() < 1e-6


# ---------------------------------------------------------------- FP32 floor (parity tolerance)
def test_fp32_storage_floor_within_parity_bar():
    """The parity bar for the FP32 GPU path (max relative error 1e-5 in rho_R,
    rho_B and u after 100 steps, u normalised by max(|u_ref|_inf, 0.01)) is
    attainable with FP32 population storage: FP64 arithmetic whose state is
    rounded to FP32 after every step stays within it on the static drop.
    (Naive FP32 arithmetic that rebuilds f+ from all nine modes does not: it
    loses ~2.5e-5; a kernel must keep its rounding near the storage level.)"""
    d, rn, u = I.static_drop()
    p = O.Params(**d)
    R0, B0 = O.init_state(rn, u[0], u[1], p)
    R64, B64 = O.run(R0, B0, p, 100)
    to32 = lambda X: X.astype(np.float32).astype(np.float64)
    R, B = to32(R0), to32(B0)
    for _ in range(100):
        R, B = O.step(R, B, p)
        R, B = to32(R), to32(B)
    f64 = O.fields(R64, B64, p)
    f32 = O.fields(R, B, p)
    for k in ("rho_r", "rho_b"):
        assert np.abs(f32[k] - f64[k]).max() / np.abs(f64[k]).max() < 1e-5
    uref = max(np.abs(np.stack([f64["ux"], f64["uy"]])).max(), 0.01)
    for k in ("ux", "uy"):
        assert np.abs(f32[k] - f64[k]).max() / uref < 1e-5


def test_app_d_simpson_solution():
    """App. D's Simpson-rule solution of the stratified channel (Eq.
    equ_integral) reduces to plane Poiseuille flow for a uniform density and
    agrees with the independent trapezoid integration of the general steady
    problem for the symmetric three-layer profile of the Ba test."""
    H, nu, G = 200, 0.333, 1e-8
    u = A.app_d_steady(np.full(H, 0.5), nu, G)
    np.testing.assert_allclose(u, A.poiseuille(H, G, 0.5 * nu), rtol=1e-12)
    _, rn, _ = I.ba_channel(H=H)
    rho = 1.0 * (1 + rn[:, 0]) / 2 + 0.125 * (1 - rn[:, 0]) / 2
    ref = A.layered_steady(rho, np.full(H, nu), g_vol=G)
    np.testing.assert_allclose(A.app_d_steady(rho, nu, G), ref, rtol=1e-6)
