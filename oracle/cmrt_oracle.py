"""Whole-field FP64 NumPy oracle of one chromodynamic MRT time step.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
CUDA library or its Python binding.

Notation follows the paper (arXiv 2005.04642).  A state is a pair of
population arrays ``R`` and ``B`` of shape ``(9, ny, nx)``: the red and blue
distributions R_i(r, t), B_i(r, t) *before* collision at time t (Sec. 2,
Eq. 1).  Position r = (x, y) is stored at ``[..., y, x]``.  One call of
:func:`step` applies, as separate whole-field sweeps and in the paper's
order,

    moments -> colour index and Phi' -> grad rho^N -> n-hat -> K -> G, u
    -> grad Phi', div u -> C -> modes, equilibria, sources -> relax
    -> reconstruct f+ -> recolour -> stream.

Readings taken where the paper is silent, garbled or at odds with itself are
stated in the docstring of the function that takes them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# Lattice (Sec. 3, Fig. 1 caption; App. A, Eq. equ_moments and the weights
# that follow it).  The figure itself is missing from the source: only "odd i
# are the longer links" survives.  Reading: links 1..8 run counter-clockwise
# from (1, 1), so odd i are the diagonals, and the opposite of link i is
# i + 4 (mod 8).  Results do not depend on this storage convention.
# ---------------------------------------------------------------------------
CX = np.array([0, 1, 0, -1, -1, -1, 0, 1, 1])
CY = np.array([0, 1, 1, 1, 0, -1, -1, -1, 0])
W_FRAC = [Fraction(4, 9)] + [Fraction(1, 36) if i % 2 else Fraction(1, 9) for i in range(1, 9)]
W = np.array([float(w) for w in W_FRAC])
# Dellar's ghost basis (App. A): g_0 = 1, g_odd = 4, g_even = -2.
GHOST = np.array([1, 4, -2, 4, -2, 4, -2, 4, -2])
OPPOSITE = np.array([0, 5, 6, 7, 8, 1, 2, 3, 4])
CS2 = 1.0 / 3.0  # colour-blind c_s^2 (Sec. 2; App. A, Eq. equ_moments)
K_PHI = 9.0 / 5.0  # k in Eq. eq_phi (D2Q9)


def projector_rows_exact():
    """Rows h^(p)_i of M as exact fractions (Table 1, App. A).

    Table 1 prints the rows weighted by w_i, but every projection in App. A
    (S^(p), h.f^(0)) and the duality h^(p).k^(p') = delta use the unweighted
    polynomials 1, c_x, c_y, c_x^2, c_y^2, c_x c_y, g, g c_x, g c_y.  Reading:
    the rows are unweighted.
    """
    rows = []
    for i in range(9):
        cx, cy, g = int(CX[i]), int(CY[i]), int(GHOST[i])
        rows.append([1, cx, cy, cx * cx, cy * cy, cx * cy, g, g * cx, g * cy])
    # transpose to [p][i]
    return [[Fraction(rows[i][p]) for i in range(9)] for p in range(9)]


def inverse_columns_exact():
    """Columns k^(p)_i of M^{-1} as exact fractions (App. A, the k vectors)."""
    cols = []
    for p in range(9):
        col = []
        for i in range(9):
            w = W_FRAC[i]
            cx, cy, g = Fraction(int(CX[i])), Fraction(int(CY[i])), Fraction(int(GHOST[i]))
            if p == 0:
                v = 2 * w - Fraction(3, 2) * w * (cx * cx + cy * cy)
            elif p == 1:
                v = 3 * w * cx
            elif p == 2:
                v = 3 * w * cy
            elif p == 3:
                v = Fraction(9, 2) * w * cx * cx - Fraction(3, 2) * w
            elif p == 4:
                v = Fraction(9, 2) * w * cy * cy - Fraction(3, 2) * w
            elif p == 5:
                v = 9 * w * cx * cy
            elif p == 6:
                v = Fraction(1, 4) * g * w
            elif p == 7:
                v = Fraction(3, 8) * g * w * cx
            else:
                v = Fraction(3, 8) * g * w * cy
            col.append(v)
        cols.append(col)
    return cols  # [p][i]


M = np.array([[float(v) for v in row] for row in projector_rows_exact()])          # [p][i]
MINV = np.array([[float(v) for v in col] for col in inverse_columns_exact()]).T    # [i][p]


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
@dataclass
class Params:
    """Physical and numerical parameters of the scheme (Sec. 2, App. A).

    ``rho0_r``, ``rho0_b``: bulk densities; Lambda = rho0_r / rho0_b must equal
    (1 - alpha_b) / (1 - alpha_r) (Eq. equ_fred).
    ``lambda3_r``, ``lambda3_b``: shear eigenvalues of the pure fluids,
    nu = (2 / lambda3 - 1) / 6 (Sec. 2 and Eq. Correction).
    ``lambda6``, ``lambda7``: ghost eigenvalues; the paper uses lambda7 = 1
    (Sec. 4) and never states lambda6: reading, default 1.
    ``g_acc``: body acceleration (force density rho * g_acc); ``g_vol``:
    uniform force per unit volume (App. D's pressure gradient).
    ``visc_mode``: 0 -> nu interpolated linearly in the colour index between
    the two fluids' values (the form of nu(rho^N) is not given, Sec. 2);
    1 -> constant shear viscosity eta, nu = eta / rho (Sec. 4.1, App. C).
    ``stencil_order``: 2 -> compact gradient for every derivative (Sec. 2);
    6 -> App. B's non-compact stencil for grad rho^N and grad Phi'.
    ``curvature_mode``: 0 -> K = div n-hat (Sec. 2); 1 -> K = fixed_K (Sec. 4.2).
    ``ghost_N_mode``: 0 -> N relaxes to h^(6).f^(0) (App. A projection of the
    equilibrium); 1 -> N relaxes to 0 (Table 1, Eq. moev for i = 6).
    ``wall_y``: False -> periodic in y; True -> half-way bounce-back walls at
    y = -1/2 and y = ny - 1/2.  x is always periodic.
    """
    nx: int
    ny: int
    rho0_r: float = 1.0
    rho0_b: float = 0.1
    alpha_r: float = 0.95
    alpha_b: float = 0.5
    sigma: float = 0.005
    beta: float = 0.67
    lambda3_r: float = 1.0
    lambda3_b: float = 1.0
    lambda6: float = 1.0
    lambda7: float = 1.0
    g_acc: tuple = (0.0, 0.0)
    g_vol: tuple = (0.0, 0.0)
    wall_y: bool = False
    visc_mode: int = 0
    eta: float = 1.0 / 6.0
    stencil_order: int = 2
    curvature_mode: int = 0
    fixed_K: float = 0.0
    ghost_N_mode: int = 0
    dtype: type = field(default=np.float64)

    @property
    def Lambda(self):
        return self.rho0_r / self.rho0_b


# Guard of the unit normal.  The paper's n-hat = -grad rho^N / |grad rho^N|
# (Sec. 2) has no direction where the colour gradient vanishes: at the centre
# of a symmetric drop and at the symmetry points between drops.  Reading: below
# NORMAL_TAU the normal is zero (no recolour bias, no contribution to K);
# at and above it, it is the paper's unit vector.  The threshold is far below
# the colour gradient of any resolved interface (an interface of width W has
# |grad rho^N| ~ 2/W at its centre) and above the round-off of the gradient
# at a drop's centre, where the same noise would otherwise set the direction.
NORMAL_TAU = 1e-9


# ---------------------------------------------------------------------------
# Local (per-node) definitions
# ---------------------------------------------------------------------------
def phi_weights(rho_r, rho_b, p: Params):
    """phi_i of Eq. eq_phi, shape (9, ...)."""
    dt = p.dtype
    rho = rho_r + rho_b
    phi = np.empty((9,) + np.shape(rho), dtype=dt)
    phi[0] = (dt(p.alpha_r) * rho_r + dt(p.alpha_b) * rho_b) / rho
    s = ((dt(1.0 - p.alpha_r)) * rho_r + dt(1.0 - p.alpha_b) * rho_b) / rho
    for i in range(1, 9):
        phi[i] = dt(K_PHI) * dt(W[i]) * s
    return phi


def equilibrium(rho_r, rho_b, ux, uy, p: Params):
    """f^(0)_i(rho, u) of Eq. equ_equ (density-contrast equilibrium)."""
    dt = p.dtype
    rho = rho_r + rho_b
    phi = phi_weights(rho_r, rho_b, p)
    usq = ux * ux + uy * uy
    f0 = np.empty_like(phi)
    for i in range(9):
        cu = dt(CX[i]) * ux + dt(CY[i]) * uy
        f0[i] = rho * phi[i] + dt(W[i]) * rho * (dt(3.0) * cu + dt(4.5) * cu * cu - dt(1.5) * usq)
    return f0


def colour_index(rho_r, rho_b, p: Params):
    """rho^N of Eq. equ_rhoN_def."""
    dt = p.dtype
    a = rho_r / dt(p.rho0_r)
    b = rho_b / dt(p.rho0_b)
    return (a - b) / (a + b)


def phi_prime(rho_r, rho_b, p: Params):
    """Phi' = 3/5 (1 - alpha_R)(rho_R + Lambda rho_B) - rho / 3 (App. A, after Eq. Pi_1)."""
    dt = p.dtype
    return dt(0.6 * (1.0 - p.alpha_r)) * (rho_r + dt(p.Lambda) * rho_b) - (rho_r + rho_b) / dt(3.0)


def pressure(rho_r, rho_b, p: Params):
    """Isotropic part of the equilibrium second moment (App. A, after Eq. eq_appb1):
    p = 3/5 [(1 - alpha_R) rho_R + (1 - alpha_B) rho_B]."""
    dt = p.dtype
    return dt(0.6 * (1.0 - p.alpha_r)) * rho_r + dt(0.6 * (1.0 - p.alpha_b)) * rho_b


def lambda3_field(rho_n, rho, p: Params):
    """Local shear eigenvalue lambda_3(rho^N) (Sec. 2: nu(rho^N) = (2/lambda_3 - 1)/6).

    Reading for ``visc_mode`` 0 (the paper gives no form): the kinematic
    viscosity is linear in the colour index between the pure fluids' values.
    ``visc_mode`` 1: constant shear viscosity eta, nu = eta / rho (Sec. 4.1).
    """
    dt = p.dtype
    if p.visc_mode == 1:
        nu = dt(p.eta) / rho
    else:
        nu_r = (2.0 / p.lambda3_r - 1.0) / 6.0
        nu_b = (2.0 / p.lambda3_b - 1.0) / 6.0
        nu = dt(0.5 * nu_r) * (dt(1.0) + rho_n) + dt(0.5 * nu_b) * (dt(1.0) - rho_n)
    return dt(2.0) / (dt(6.0) * nu + dt(1.0))


# ---------------------------------------------------------------------------
# Finite differences (the compact second-order stencils of Sec. 2; App. B)
# ---------------------------------------------------------------------------
def value_at_offset(field_, dx, dy, p: Params, parity=1):
    """field(r + (dx, dy)) on the lattice.

    x is periodic.  y is periodic, or, with walls, the value beyond a wall is
    the mirror image across the wall plane (y = -1/2 or ny - 1/2) times
    ``parity``.  Reading (the paper does not state its wall treatment for
    stencils): colour index and Phi' are mirrored evenly (neutral wetting, zero
    normal gradient), the normal's y component and both velocity components
    oddly (no-slip, impermeable wall).
    """
    out = np.roll(field_, -dx, axis=-1)
    if not p.wall_y:
        return np.roll(out, -dy, axis=-2)
    ny = field_.shape[-2]
    ys = np.arange(ny) + dy
    src = np.where(ys < 0, -1 - ys, np.where(ys >= ny, 2 * ny - 1 - ys, ys))
    res = out[..., src, :]
    if parity != 1:
        outside = (ys < 0) | (ys >= ny)
        res = res.copy()
        res[..., outside, :] *= parity
    return res


def gradient(field_, p: Params, parity=1, order=2):
    """Gradient of a scalar field.

    order 2: compact isotropic stencil d_a f = 3 sum_i w_i f(r + c_i) c_ia
    (Sec. 2; App. B, Eq. equ_HOstencil with N = 1).
    order 6: App. B's non-compact stencil d_a f = sum_N a_N sum_i w_i
    f(r + N c_i) c_ia with (a_1, a_2, a_3) = (9/2, -9/10, 1/10).  App. B's
    printed coefficient matrix has 2^3/5! where 2^5/5! belongs; the printed
    result (9/2, -9/10, 1/10) is the inverse of the corrected matrix, and is
    used here.
    """
    dt = p.dtype
    coeffs = [(1, 3.0)] if order == 2 else [(1, 4.5), (2, -0.9), (3, 0.1)]
    gx = np.zeros_like(field_)
    gy = np.zeros_like(field_)
    for n, a in coeffs:
        for i in range(1, 9):
            v = value_at_offset(field_, n * int(CX[i]), n * int(CY[i]), p, parity)
            gx = gx + dt(a * W[i] * CX[i]) * v
            gy = gy + dt(a * W[i] * CY[i]) * v
    return gx, gy


def unit_normal(gx, gy, p: Params):
    """n-hat = -grad rho^N / |grad rho^N| (Sec. 2) where |grad rho^N| >= NORMAL_TAU,
    and 0 where the gradient is below that guard (no direction)."""
    dt = p.dtype
    mag = np.sqrt(gx * gx + gy * gy)
    big = mag >= dt(NORMAL_TAU)
    inv = np.where(big, dt(1.0) / np.where(big, mag, dt(1.0)), dt(0.0))
    return -gx * inv, -gy * inv


def curvature(nx_, ny_, p: Params):
    """Mean curvature K = div n-hat (Sec. 2, after Eq. equ_stforce), compact stencil."""
    dxn, _ = gradient(nx_, p, parity=1)
    _, dyn = gradient(ny_, p, parity=-1)
    return dxn + dyn


# ---------------------------------------------------------------------------
# Collision (Sec. 3; App. A)
# ---------------------------------------------------------------------------
def correction_tensor(ux, uy, Gx, Gy, dPx, dPy, divu, rho, lam3, p: Params):
    """C_ab of Eq. Correction:
    (1 - l3/2)[u_a (G_b - d_b Phi') + u_b (G_a - d_a Phi')]
      - (1 - l3/2)[u.grad Phi' - rho div u / 3] delta_ab."""
    dt = p.dtype
    a = dt(1.0) - lam3 / dt(2.0)
    iso = ux * dPx + uy * dPy - rho * divu / dt(3.0)
    cxx = a * (dt(2.0) * ux * (Gx - dPx)) - a * iso
    cyy = a * (dt(2.0) * uy * (Gy - dPy)) - a * iso
    cxy = a * (ux * (Gy - dPy) + uy * (Gx - dPx))
    return cxx, cyy, cxy


def source_F1(ux, uy, dPx, dPy, divu, rho, lam3, p: Params):
    """F_1i = w_i T_ab (c_ia c_ib - c_s^2 delta_ab) (Eq. equ_source1) with T of
    Eq. equ_T_identity.  Used to cross-check the modal sources."""
    dt = p.dtype
    pre = dt(1.0 / (2.0 * CS2 * CS2)) * (dt(1.0) - lam3 / dt(2.0))
    udP = ux * dPx + uy * dPy
    txx = pre * (rho * divu / dt(3.0) - (dt(2.0) * ux * dPx + udP))
    tyy = pre * (rho * divu / dt(3.0) - (dt(2.0) * uy * dPy + udP))
    txy = pre * (-(ux * dPy + uy * dPx))
    out = np.empty((9,) + np.shape(rho), dtype=dt)
    for i in range(9):
        cx, cy = float(CX[i]), float(CY[i])
        out[i] = dt(W[i]) * (txx * dt(cx * cx - CS2) + tyy * dt(cy * cy - CS2) + dt(2.0 * cx * cy) * txy)
    return out


def source_F2(ux, uy, Gx, Gy, lam3, p: Params):
    """F_2i of Eq. equ_source2 (Luo's forcing with the MRT factor 1 - lambda_3/2)."""
    dt = p.dtype
    pre = dt(1.0 / (2.0 * CS2 * CS2)) * (dt(1.0) - lam3 / dt(2.0))
    sxx = dt(2.0) * Gx * ux
    syy = dt(2.0) * Gy * uy
    sxy = Gx * uy + Gy * ux
    out = np.empty((9,) + np.shape(ux), dtype=dt)
    for i in range(9):
        cx, cy = float(CX[i]), float(CY[i])
        lin = (dt(cx) * Gx + dt(cy) * Gy) / dt(CS2)
        quad = pre * (sxx * dt(cx * cx - CS2) + syy * dt(cy * cy - CS2) + dt(2.0 * cx * cy) * sxy)
        out[i] = dt(W[i]) * (lin + quad)
    return out


def modes(f, p: Params):
    """m = M f (Sec. 3; App. A, Eq. equ_key), shape (9, ...)."""
    dt = p.dtype
    return np.tensordot(M.astype(dt), f, axes=(1, 0))


def modal_equilibrium(rho_r, rho_b, ux, uy, p: Params):
    """Projections h^(p).f^(0) listed in App. A.

    Reading for the ghost N (Table 1 prints equilibrium 0, App. A computes
    h^(6).f^(0) = 9/5 alpha_R rho_R + 9/5 alpha_B rho_B - 4/5 rho): with
    ``ghost_N_mode`` 0 the projection is used, which is what the modal
    projection of Eq. 1 (App. A, Eq. evo-pro) requires; mode 1 uses 0.
    """
    dt = p.dtype
    rho = rho_r + rho_b
    pr = pressure(rho_r, rho_b, p)
    meq = np.zeros((9,) + np.shape(rho), dtype=dt)
    meq[0] = rho
    meq[1] = rho * ux
    meq[2] = rho * uy
    meq[3] = pr + rho * ux * ux
    meq[4] = pr + rho * uy * uy
    meq[5] = rho * ux * uy
    if p.ghost_N_mode == 0:
        meq[6] = dt(1.8 * p.alpha_r) * rho_r + dt(1.8 * p.alpha_b) * rho_b - dt(0.8) * rho
    return meq


def modal_sources(Gx, Gy, cxx, cyy, cxy, p: Params):
    """S^(p) = h^(p).(F_1 + F_2) (App. A), with n = 1.

    Reading: the projections of the explicit sources of Eqs. equ_source1 and
    equ_source2 are S = (0, G_x, G_y, C_xx, C_yy, C_xy, 0, 0, 0).  App. A
    prints S^(6) = -(C_xx + C_yy)/2 but also states that F has no projection
    onto N, J_x, J_y; projecting Eqs. equ_source1-2 gives exactly 0, which is
    taken.  Likewise Eq. equ_Fis writes sum_i c c F = C + C^T while the
    explicit sources give C (symmetric), as App. A's S^(3..5) list has it.
    """
    dt = p.dtype
    S = np.zeros((9,) + np.shape(Gx), dtype=dt)
    S[1] = Gx
    S[2] = Gy
    S[3] = cxx
    S[4] = cyy
    S[5] = cxy
    return S


def relax(m, meq, S, lam3, p: Params):
    """Forced scalar relaxation m+ = m + lambda_p (m^(0) - m) + S (App. A, Eq. 38),
    lambda_0..2 = 0, lambda_3..5 = lambda_3 (local), lambda_6, lambda_7 = lambda_8."""
    dt = p.dtype
    lam = [dt(0.0), dt(0.0), dt(0.0), lam3, lam3, lam3, dt(p.lambda6), dt(p.lambda7), dt(p.lambda7)]
    out = np.empty_like(m)
    for q in range(9):
        out[q] = m[q] + lam[q] * (meq[q] - m[q]) + S[q]
    return out


def reconstruct(mplus, p: Params):
    """f+ = M^{-1} m+ with the explicit k vectors of App. A (Eq. eq84)."""
    dt = p.dtype
    return np.tensordot(MINV.astype(dt), mplus, axes=(1, 0))


def recolour(fplus, rho_r, rho_b, ex, ey, p: Params):
    """d'Ortona segregation, Eq. eq_re_color.

    C_i++ = (rho_C / rho) f_i+ +/- beta phi_i rho_R rho_B / rho  (e . c-hat_i).
    Reading of the sign: with n-hat = -grad rho^N/|grad rho^N| (outward for a
    red drop), adding beta(...) n-hat.c-hat to red would push red out of the
    drop.  Red therefore takes +beta(...) e.c-hat_i with e = grad rho^N /
    |grad rho^N| = -n-hat, blue the negative.  c-hat_i = c_i / |c_i|
    (c-hat_0 = 0) and the weights are phi_i, as printed.
    """
    dt = p.dtype
    rho = rho_r + rho_b
    phi = phi_weights(rho_r, rho_b, p)
    seg = dt(p.beta) * rho_r * rho_b / rho
    R = np.empty_like(fplus)
    B = np.empty_like(fplus)
    for i in range(9):
        if i == 0:
            ec = np.zeros_like(rho)
        else:
            norm = np.sqrt(float(CX[i] ** 2 + CY[i] ** 2))
            ec = (dt(CX[i] / norm) * ex + dt(CY[i] / norm) * ey)
        d = seg * phi[i] * ec
        R[i] = rho_r / rho * fplus[i] + d
        B[i] = rho_b / rho * fplus[i] - d
    return R, B


def stream(Cpp, p: Params):
    """Streaming C_i(r + c_i, t + 1) = C_i++(r, t) (Eq. equ_evolution, left side).

    x periodic.  y periodic or, with walls, half-way bounce-back (the paper's
    benchmarks have no-slip walls but do not state the scheme; reading): a
    population that would cross a wall returns to its node reversed,
    C_opp(i)(r, t + 1) = C_i++(r, t).
    """
    out = np.empty_like(Cpp)
    ny = Cpp.shape[1]
    for i in range(9):
        moved = np.roll(Cpp[i], int(CX[i]), axis=1)
        if not p.wall_y:
            out[i] = np.roll(moved, int(CY[i]), axis=0)
        else:
            res = np.empty_like(moved)
            cy = int(CY[i])
            if cy == 0:
                res[:] = moved
            elif cy == 1:
                res[1:] = moved[:-1]
            else:
                res[:-1] = moved[1:]
            out[i] = res
    if p.wall_y:
        for i in range(9):
            cy = int(CY[i])
            if cy == 1:      # leaves through the top wall y = ny - 1/2
                out[OPPOSITE[i], ny - 1, :] = Cpp[i, ny - 1, :]
            elif cy == -1:   # leaves through the bottom wall y = -1/2
                out[OPPOSITE[i], 0, :] = Cpp[i, 0, :]
    return out


# ---------------------------------------------------------------------------
# Whole step
# ---------------------------------------------------------------------------
@dataclass
class Derived:
    """Intermediate fields of one step (exposed for the tests)."""
    rho_r: np.ndarray
    rho_b: np.ndarray
    rho: np.ndarray
    jx: np.ndarray
    jy: np.ndarray
    rho_n: np.ndarray
    phip: np.ndarray
    gnx: np.ndarray
    gny: np.ndarray
    nhx: np.ndarray
    nhy: np.ndarray
    K: np.ndarray
    Gx: np.ndarray
    Gy: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    dPx: np.ndarray = None
    dPy: np.ndarray = None
    divu: np.ndarray = None
    lam3: np.ndarray = None


def macroscopic(R, B, p: Params) -> Derived:
    """Observables at time t from the pre-collision state.

    Densities and colour-blind momentum (Eq. equ_u_def), rho^N (Eq.
    equ_rhoN_def), Phi', grad rho^N and n-hat, K, the total force
    G = sigma K grad rho^N / 2 + rho g_acc + g_vol (Eq. equ_stforce plus the
    body force) and the force-adjusted velocity u = (sum f c + G/2) / rho
    (Eq. equ_u_def; App. A, Eq. equ_constants m = 1/2).
    """
    dt = p.dtype
    rho_r = R.sum(axis=0)
    rho_b = B.sum(axis=0)
    f = R + B
    rho = rho_r + rho_b
    jx = np.tensordot(CX.astype(dt), f, axes=(0, 0))
    jy = np.tensordot(CY.astype(dt), f, axes=(0, 0))
    rho_n = colour_index(rho_r, rho_b, p)
    phip = phi_prime(rho_r, rho_b, p)
    gnx, gny = gradient(rho_n, p, parity=1, order=p.stencil_order)
    nhx, nhy = unit_normal(gnx, gny, p)
    if p.curvature_mode == 1:
        K = np.full_like(rho, dt(p.fixed_K))
    else:
        K = curvature(nhx, nhy, p)
    half_sigma = dt(0.5 * p.sigma)
    Gx = half_sigma * K * gnx + rho * dt(p.g_acc[0]) + dt(p.g_vol[0])
    Gy = half_sigma * K * gny + rho * dt(p.g_acc[1]) + dt(p.g_vol[1])
    ux = (jx + Gx / dt(2.0)) / rho
    uy = (jy + Gy / dt(2.0)) / rho
    return Derived(rho_r, rho_b, rho, jx, jy, rho_n, phip, gnx, gny, nhx, nhy, K, Gx, Gy, ux, uy)


def collide_and_recolour(R, B, p: Params, d: Derived = None):
    """Post-recolour populations R++, B++ (App. A Eqs. 38, eq84; Eq. eq_re_color)."""
    dt = p.dtype
    if d is None:
        d = macroscopic(R, B, p)
    d.dPx, d.dPy = gradient(d.phip, p, parity=1, order=p.stencil_order)
    dux, _ = gradient(d.ux, p, parity=-1)
    _, duy = gradient(d.uy, p, parity=-1)
    d.divu = dux + duy
    d.lam3 = lambda3_field(d.rho_n, d.rho, p)
    cxx, cyy, cxy = correction_tensor(d.ux, d.uy, d.Gx, d.Gy, d.dPx, d.dPy, d.divu, d.rho, d.lam3, p)
    f = R + B
    m = modes(f, p)
    meq = modal_equilibrium(d.rho_r, d.rho_b, d.ux, d.uy, p)
    S = modal_sources(d.Gx, d.Gy, cxx, cyy, cxy, p)
    mplus = relax(m, meq, S, d.lam3, p)
    fplus = reconstruct(mplus, p)
    ex, ey = -d.nhx, -d.nhy
    return recolour(fplus, d.rho_r, d.rho_b, ex, ey, p)


def step(R, B, p: Params):
    """One time step t -> t + 1: collide, recolour, stream (Eq. equ_evolution;
    Sec. 3 puts the recolouring last, after the collision)."""
    Rpp, Bpp = collide_and_recolour(R, B, p)
    return stream(Rpp, p), stream(Bpp, p)


def run(R, B, p: Params, nsteps: int):
    for _ in range(nsteps):
        R, B = step(R, B, p)
    return R, B


def init_state(rho_n0, u0x, u0y, p: Params):
    """Initial populations from a colour field and a velocity field.

    The paper does not state its initialisation.  Reading: rho_R =
    rho0_R (1 + rho^N_0)/2, rho_B = rho0_B (1 - rho^N_0)/2 (this inverts
    Eq. equ_rhoN_def exactly) and C_i = (rho_C / rho) f^(0)_i(rho, u_0)
    (Eq. equ_equ), with no segregation bias.
    """
    dt = p.dtype
    rho_n0 = np.asarray(rho_n0, dtype=dt)
    rho_r = dt(p.rho0_r) * (dt(1.0) + rho_n0) / dt(2.0)
    rho_b = dt(p.rho0_b) * (dt(1.0) - rho_n0) / dt(2.0)
    rho = rho_r + rho_b
    f0 = equilibrium(rho_r, rho_b, np.asarray(u0x, dtype=dt), np.asarray(u0y, dtype=dt), p)
    return (rho_r / rho) * f0, (rho_b / rho) * f0


def fields(R, B, p: Params):
    """rho_R, rho_B, force-adjusted u_x, u_y and pressure p at time t."""
    d = macroscopic(R, B, p)
    return {"rho_r": d.rho_r, "rho_b": d.rho_b, "ux": d.ux, "uy": d.uy,
            "p": pressure(d.rho_r, d.rho_b, p)}


def diagnostics(R, B, p: Params):
    """Colour masses, colour-blind lattice momentum sum_r sum_i f_i c_i and max |u|."""
    d = macroscopic(R, B, p)
    return {"mass_r": float(np.sum(d.rho_r, dtype=np.float64)),
            "mass_b": float(np.sum(d.rho_b, dtype=np.float64)),
            "mom_x": float(np.sum(d.jx, dtype=np.float64)),
            "mom_y": float(np.sum(d.jy, dtype=np.float64)),
            "umax": float(np.sqrt(np.max(d.ux * d.ux + d.uy * d.uy)))}
