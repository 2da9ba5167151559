"""Exact and brute-force pins of the oracle's local definitions.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code: lattice isotropy (App. A,
Eq. equ_moments), h.k = delta (App. A), moments of the equilibrium (App. A,
Eq. eq_appb1), moments of the sources (Eqs. equ_source1-2 vs Eq. Correction),
the modal/direct equivalence of the collision (Sec. 3, Eq. equ_temp1),
recolour mass conservation (Sec. 2), stencil exactness on polynomials
(App. B), and the streaming/bounce-back geometry.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import cmrt_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(**kw):
    base = dict(nx=8, ny=8)
    base.update(kw)
    return O.Params(**base)


# ---------------------------------------------------------------- lattice
def test_lattice_isotropy_exact():
    """App. A, Eq. equ_moments: sum w = 1, odd moments vanish,
    sum w c_a c_b = delta/3, sum w c_a c_b c_g c_d = (dd + dd + dd)/9."""
    W = O.W_FRAC
    c = [(int(O.CX[i]), int(O.CY[i])) for i in range(9)]
    assert sum(W) == 1
    d = lambda a, b: Fraction(int(a == b))
    for a in range(2):
        assert sum(W[i] * c[i][a] for i in range(9)) == 0
        for b in range(2):
            assert sum(W[i] * c[i][a] * c[i][b] for i in range(9)) == Fraction(1, 3) * d(a, b)
            for g in range(2):
                assert sum(W[i] * c[i][a] * c[i][b] * c[i][g] for i in range(9)) == 0
                for e in range(2):
                    lhs = sum(W[i] * c[i][a] * c[i][b] * c[i][g] * c[i][e] for i in range(9))
                    rhs = Fraction(1, 9) * (d(a, b) * d(g, e) + d(a, g) * d(b, e) + d(a, e) * d(b, g))
                    assert lhs == rhs
    # odd i are the longer (diagonal) links, weights 1/36; even i axis links 1/9
    for i in range(1, 9):
        assert (abs(c[i][0]) + abs(c[i][1]) == 2) == (i % 2 == 1)
        assert W[i] == (Fraction(1, 36) if i % 2 else Fraction(1, 9))
    # opposite links
    for i in range(9):
        j = int(O.OPPOSITE[i])
        assert c[j] == (-c[i][0], -c[i][1])


def test_projector_inverse_identity_exact():
    """App. A: h^(p) . k^(p') = delta_pp', hence M^{-1} = (k^(0) ... k^(8))."""
    h = O.projector_rows_exact()
    k = O.inverse_columns_exact()
    for p in range(9):
        for q in range(9):
            s = sum(h[p][i] * k[q][i] for i in range(9))
            assert s == (1 if p == q else 0), (p, q, s)
    np.testing.assert_allclose(O.M @ O.MINV, np.eye(9), atol=1e-15)
    np.testing.assert_allclose(O.MINV @ O.M, np.eye(9), atol=1e-15)


def test_ghost_rows_are_dellars_basis():
    """App. A: g_0 = 1, g_odd = 4, g_even = -2; rows 6..8 of M are g, g c_x, g c_y."""
    assert list(O.GHOST) == [1, 4, -2, 4, -2, 4, -2, 4, -2]
    np.testing.assert_array_equal(O.M[6], O.GHOST)
    np.testing.assert_array_equal(O.M[7], O.GHOST * O.CX)
    np.testing.assert_array_equal(O.M[8], O.GHOST * O.CY)


# ---------------------------------------------------------------- equilibrium
@pytest.fixture
def rand_local():
    rng = np.random.default_rng(11)
    n = 64
    rho_r = rng.uniform(0.01, 1.2, n)
    rho_b = rng.uniform(0.01, 0.3, n)
    ux = rng.uniform(-0.1, 0.1, n)
    uy = rng.uniform(-0.1, 0.1, n)
    return rho_r, rho_b, ux, uy


@pytest.mark.parametrize("alphas", [(0.95, 0.5), (0.9, 0.2), (4 / 9, 4 / 9), (0.5, 0.9995)])
def test_phi_and_equilibrium_moments(rand_local, alphas):
    """Eq. eq_phi: sum phi_i = 1.  App. A, Eq. eq_appb1:
    sum (1, c, cc) f^(0) = (rho, rho u, 3/5[(1-a_R) rho_R + (1-a_B) rho_B] delta + rho u u)."""
    rho_r, rho_b, ux, uy = rand_local
    p = _params(alpha_r=alphas[0], alpha_b=alphas[1])
    phi = O.phi_weights(rho_r, rho_b, p)
    np.testing.assert_allclose(phi.sum(0), 1.0, rtol=0, atol=1e-15)
    f0 = O.equilibrium(rho_r, rho_b, ux, uy, p)
    rho = rho_r + rho_b
    cx = O.CX[:, None].astype(float)
    cy = O.CY[:, None].astype(float)
    np.testing.assert_allclose(f0.sum(0), rho, rtol=1e-14)
    np.testing.assert_allclose((cx * f0).sum(0), rho * ux, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose((cy * f0).sum(0), rho * uy, rtol=1e-13, atol=1e-16)
    ceff = 0.6 * ((1 - alphas[0]) * rho_r + (1 - alphas[1]) * rho_b)
    np.testing.assert_allclose((cx * cx * f0).sum(0), ceff + rho * ux * ux, rtol=1e-13)
    np.testing.assert_allclose((cy * cy * f0).sum(0), ceff + rho * uy * uy, rtol=1e-13)
    np.testing.assert_allclose((cx * cy * f0).sum(0), rho * ux * uy, rtol=1e-12, atol=1e-17)


def test_phi_prime_is_pressure_deviation(rand_local):
    """App. A: Phi' is the deviation of the isotropic equilibrium stress from
    the colour-blind rho/3, i.e. sum c_x^2 f^(0) - rho u_x^2 - rho/3."""
    rho_r, rho_b, ux, uy = rand_local
    p = _params(alpha_r=0.95, alpha_b=0.5, rho0_r=1.0, rho0_b=0.1)
    f0 = O.equilibrium(rho_r, rho_b, ux, uy, p)
    rho = rho_r + rho_b
    pxx = (O.CX[:, None] ** 2 * f0).sum(0)
    np.testing.assert_allclose(O.phi_prime(rho_r, rho_b, p), pxx - rho * ux * ux - rho / 3, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(O.pressure(rho_r, rho_b, p), pxx - rho * ux * ux, rtol=1e-13)


@pytest.mark.parametrize("alphas", [(0.95, 0.5), (4 / 9, 4 / 9), (0.6, 0.3)])
def test_modal_equilibrium_is_projection(rand_local, alphas):
    """App. A lists h^(p).f^(0); check them against a brute-force M f^(0)."""
    rho_r, rho_b, ux, uy = rand_local
    p = _params(alpha_r=alphas[0], alpha_b=alphas[1])
    f0 = O.equilibrium(rho_r, rho_b, ux, uy, p)
    np.testing.assert_allclose(O.modal_equilibrium(rho_r, rho_b, ux, uy, p), O.M @ f0, rtol=1e-12, atol=1e-15)
    # the table's N^(0) = 0 agrees with the projection only when alpha_R = alpha_B = 4/9
    p1 = _params(alpha_r=alphas[0], alpha_b=alphas[1], ghost_N_mode=1)
    m1 = O.modal_equilibrium(rho_r, rho_b, ux, uy, p1)
    same = np.allclose(m1[6], (O.M @ f0)[6], atol=1e-14)
    assert same == (alphas == (4 / 9, 4 / 9))


# ---------------------------------------------------------------- sources
@pytest.fixture
def rand_source_inputs():
    rng = np.random.default_rng(5)
    n = 64
    vals = {k: rng.uniform(-1e-2, 1e-2, n) for k in ("ux", "uy", "Gx", "Gy", "dPx", "dPy", "divu")}
    vals["rho"] = rng.uniform(0.1, 1.1, n)
    vals["lam3"] = rng.uniform(0.3, 1.9, n)
    return vals


def test_source_moments_match_correction_tensor(rand_source_inputs):
    """sum_i (1, c, cc)(F_1 + F_2) = (0, G, C) with F_1, F_2 from Eqs.
    equ_source1, equ_source2, equ_T_identity and C from Eq. Correction.
    (Eq. equ_Fis writes C + C^T; the explicit sources give C, as App. A's
    S^(3..5) list has it.)"""
    v = rand_source_inputs
    p = _params()
    F = O.source_F1(v["ux"], v["uy"], v["dPx"], v["dPy"], v["divu"], v["rho"], v["lam3"], p) \
        + O.source_F2(v["ux"], v["uy"], v["Gx"], v["Gy"], v["lam3"], p)
    cxx, cyy, cxy = O.correction_tensor(v["ux"], v["uy"], v["Gx"], v["Gy"], v["dPx"], v["dPy"],
                                        v["divu"], v["rho"], v["lam3"], p)
    cx = O.CX[:, None].astype(float)
    cy = O.CY[:, None].astype(float)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-17)
    np.testing.assert_allclose((cx * F).sum(0), v["Gx"], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose((cy * F).sum(0), v["Gy"], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose((cx * cx * F).sum(0), cxx, rtol=1e-11, atol=1e-18)
    np.testing.assert_allclose((cy * cy * F).sum(0), cyy, rtol=1e-11, atol=1e-18)
    np.testing.assert_allclose((cx * cy * F).sum(0), cxy, rtol=1e-11, atol=1e-18)
    # full modal projection: S = M F, including S^(6) = S^(7) = S^(8) = 0
    S = O.modal_sources(v["Gx"], v["Gy"], cxx, cyy, cxy, p)
    np.testing.assert_allclose(O.M @ F, S, rtol=1e-11, atol=1e-17)
    np.testing.assert_allclose((O.M @ F)[6:], 0.0, atol=1e-17)


def test_direct_collision_equals_modal(rand_local, rand_source_inputs):
    """Sec. 3, Eq. equ_temp1: f+ = f - A (f - f^(0)) + F with
    A = M^{-1} diag(lambda) M equals the modal route M^{-1} m+."""
    rho_r, rho_b, ux, uy = rand_local
    v = rand_source_inputs
    p = _params(alpha_r=0.95, alpha_b=0.5, lambda6=1.3, lambda7=0.8)
    n = rho_r.size
    rng = np.random.default_rng(9)
    f0 = O.equilibrium(rho_r, rho_b, ux, uy, p)
    f = f0 * (1 + rng.uniform(-0.05, 0.05, f0.shape))
    lam3 = v["lam3"][:n]
    F = O.source_F1(ux, uy, v["dPx"], v["dPy"], v["divu"], rho_r + rho_b, lam3, p) \
        + O.source_F2(ux, uy, v["Gx"], v["Gy"], lam3, p)
    direct = np.empty_like(f)
    for j in range(n):
        lam = np.diag([0, 0, 0, lam3[j], lam3[j], lam3[j], p.lambda6, p.lambda7, p.lambda7])
        A = O.MINV @ lam @ O.M
        direct[:, j] = f[:, j] - A @ (f[:, j] - f0[:, j]) + F[:, j]
    cxx, cyy, cxy = O.correction_tensor(ux, uy, v["Gx"], v["Gy"], v["dPx"], v["dPy"], v["divu"],
                                        rho_r + rho_b, lam3, p)
    m = O.modes(f, p)
    meq = O.modal_equilibrium(rho_r, rho_b, ux, uy, p)
    S = O.modal_sources(v["Gx"], v["Gy"], cxx, cyy, cxy, p)
    modal = O.reconstruct(O.relax(m, meq, S, lam3, p), p)
    np.testing.assert_allclose(modal, direct, rtol=1e-12, atol=1e-15)


def test_equilibrium_is_collision_fixed_point(rand_local):
    """P3: a uniform state at equilibrium (no gradients, no force) collides to itself
    for any relaxation rates; the recolour then only splits it by rho_C / rho."""
    rho_r, rho_b, ux, uy = rand_local
    for lam3, l6, l7 in [(1.0, 1.0, 1.0), (1.7, 0.4, 1.9), (0.3, 1.5, 0.2)]:
        p = O.Params(nx=4, ny=3, alpha_r=0.95, alpha_b=0.5, lambda3_r=lam3, lambda3_b=lam3,
                     lambda6=l6, lambda7=l7, sigma=0.01)
        j = 7
        shape = (3, 4)
        rr = np.full(shape, rho_r[j]); rb = np.full(shape, rho_b[j])
        u_x = np.full(shape, ux[j]); u_y = np.full(shape, uy[j])
        f0 = O.equilibrium(rr, rb, u_x, u_y, p)
        R, B = (rr / (rr + rb)) * f0, (rb / (rr + rb)) * f0
        Rpp, Bpp = O.collide_and_recolour(R, B, p)
        np.testing.assert_allclose(Rpp + Bpp, f0, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(Rpp, R, rtol=1e-13, atol=1e-16)


def test_recolour_conserves_colour_mass():
    """Sec. 2, Eq. eq_re_color: R++ + B++ = f+ and sum_i C_i++ = rho_C."""
    rng = np.random.default_rng(3)
    p = _params(alpha_r=0.95, alpha_b=0.5, beta=0.67)
    n = 40
    rho_r = rng.uniform(0.0, 1.0, n)
    rho_b = rng.uniform(0.0, 0.1, n)
    fplus = O.equilibrium(rho_r, rho_b, rng.uniform(-.05, .05, n), rng.uniform(-.05, .05, n), p)
    ang = rng.uniform(0, 2 * np.pi, n)
    R, B = O.recolour(fplus, rho_r, rho_b, np.cos(ang), np.sin(ang), p)
    np.testing.assert_allclose(R + B, fplus, rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(R.sum(0), rho_r, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(B.sum(0), rho_b, rtol=1e-13, atol=1e-16)
    # segregation moves red along e = grad rho^N / |grad rho^N|: net red flux along e
    flux = (O.CX[:, None] * R).sum(0) * np.cos(ang) + (O.CY[:, None] * R).sum(0) * np.sin(ang)
    base = (O.CX[:, None] * fplus * rho_r / (rho_r + rho_b)).sum(0) * np.cos(ang) \
        + (O.CY[:, None] * fplus * rho_r / (rho_r + rho_b)).sum(0) * np.sin(ang)
    assert np.all(flux - base >= -1e-15)


# ---------------------------------------------------------------- stencils
def _poly_field(nx, ny, fn):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    return x, y, fn(x, y)


def test_compact_stencil_exact_on_quadratics():
    """Sec. 2 / App. B (N = 1): 3 sum_i w_i f(r + c_i) c_i is exact for polynomials of degree <= 2."""
    p = O.Params(nx=16, ny=16)
    rng = np.random.default_rng(2)
    a = rng.normal(size=6)
    x, y, f = _poly_field(16, 16, lambda x, y: a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y)
    gx, gy = O.gradient(f, p)
    s = (slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(gx[s], (a[1] + 2 * a[3] * x + a[4] * y)[s], rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(gy[s], (a[2] + a[4] * x + 2 * a[5] * y)[s], rtol=1e-12, atol=1e-11)
    # and not exact at degree 3 (so the test can tell the orders apart)
    _, _, f3 = _poly_field(16, 16, lambda x, y: x ** 3)
    gx3, _ = O.gradient(f3, p)
    assert np.abs(gx3[s] - (3 * x ** 2)[s]).max() > 0.1


def test_app_b_stencil_golden_and_exactness():
    """App. B: the printed coefficients (9/2, -9/10, 1/10) cancel the N^3 and
    N^5 error terms of Eq. equ_HOstencil (sum a_N N = 3, sum a_N N^3 =
    sum a_N N^5 = 0), and the order-6 gradient is exact for degree <= 6."""
    coeffs = {}
    with open(os.path.join(GOLDEN, "app_b_stencil.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            n, num, den = line.split()
            coeffs[int(n)] = Fraction(int(num), int(den))
    assert sum(a * n for n, a in coeffs.items()) == 3
    assert sum(a * n ** 3 for n, a in coeffs.items()) == 0
    assert sum(a * n ** 5 for n, a in coeffs.items()) == 0
    p = O.Params(nx=24, ny=24)
    rng = np.random.default_rng(4)
    a = rng.normal(size=4)
    fn = lambda x, y: a[0] * x ** 5 + a[1] * x ** 3 * y ** 2 + a[2] * y ** 6 + a[3] * x * y ** 4
    dfx = lambda x, y: 5 * a[0] * x ** 4 + 3 * a[1] * x ** 2 * y ** 2 + a[3] * y ** 4
    dfy = lambda x, y: 2 * a[1] * x ** 3 * y + 6 * a[2] * y ** 5 + 4 * a[3] * x * y ** 3
    y, x = np.mgrid[0:24, 0:24].astype(float)
    x = x / 8.0 + 0.3
    y = y / 8.0 - 0.2
    # evaluate the stencil in lattice units on the scaled polynomial
    f = fn(x, y)
    gx, gy = O.gradient(f, p, order=6)
    s = (slice(3, -3), slice(3, -3))
    np.testing.assert_allclose(gx[s] * 8.0, dfx(x, y)[s], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(gy[s] * 8.0, dfy(x, y)[s], rtol=1e-9, atol=1e-9)


def test_wall_ghost_mirror():
    """With walls the value beyond y = -1/2 (ny - 1/2) is the mirror image, times the parity."""
    p = O.Params(nx=3, ny=5, wall_y=True)
    f = np.arange(15, dtype=float).reshape(5, 3)
    below = O.value_at_offset(f, 0, -1, p, parity=-1)
    np.testing.assert_array_equal(below[0], -f[0])
    np.testing.assert_array_equal(below[1:], f[:-1])
    above = O.value_at_offset(f, 1, 2, p)
    np.testing.assert_array_equal(above[3], np.roll(f[4], -1))
    np.testing.assert_array_equal(above[4], np.roll(f[3], -1))


# ---------------------------------------------------------------- streaming
@pytest.mark.parametrize("wall", [False, True])
def test_streaming_moves_along_links(wall):
    """Eq. equ_evolution: C_i(r + c_i, t+1) = C_i++(r, t); with walls a
    population leaving through y = -1/2 or ny - 1/2 returns reversed."""
    p = O.Params(nx=6, ny=5, wall_y=wall)
    for i in range(9):
        for (x0, y0) in [(2, 2), (0, 0), (5, 4)]:
            C = np.zeros((9, 5, 6))
            C[i, y0, x0] = 1.0
            out = O.stream(C, p)
            assert out.sum() == 1.0
            x1 = (x0 + O.CX[i]) % 6
            y1 = y0 + O.CY[i]
            if not wall:
                assert out[i, y1 % 5, x1] == 1.0
            elif 0 <= y1 < 5:
                assert out[i, y1, x1] == 1.0
            else:
                assert out[O.OPPOSITE[i], y0, x0] == 1.0


# ---------------------------------------------------------------- golden: Lambda / alpha table
def test_alpha_table_gives_mechanical_stability():
    """Sec. 2, Eq. equ_fred: Lambda = rho0_R/rho0_B = (1-alpha_B)/(1-alpha_R), so that
    rho0_R c_R^2 = rho0_B c_B^2: the oracle's pressure is the same in both bulk phases
    for every row of the paper's table."""
    from paper_2005_04642_gb300.inputs import alpha_split
    rows = np.loadtxt(os.path.join(GOLDEN, "alpha_lambda_table.txt"))
    for Lam, a_b, a_r in rows:
        p = O.Params(nx=2, ny=2, rho0_r=1.0, rho0_b=1.0 / Lam, alpha_r=a_r, alpha_b=a_b)
        np.testing.assert_allclose((1 - a_b) / (1 - a_r), Lam, rtol=1e-12)
        pr = O.pressure(np.array(p.rho0_r), np.array(0.0), p)
        pb = O.pressure(np.array(0.0), np.array(p.rho0_b), p)
        np.testing.assert_allclose(pr, pb, rtol=1e-12)
        got = alpha_split(Lam, 0.5)
        np.testing.assert_allclose(got, (a_r, a_b), rtol=0, atol=5e-5)
