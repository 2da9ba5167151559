"""Discrete adjoint (reverse mode) of the oracle's time step, FP64 NumPy.

TEST INFRASTRUCTURE ONLY: like :mod:`oracle.cmrt_oracle`, never imported by
the CUDA library or its binding.

The forward map is the oracle's step f(t+1) = stream(CR(f(t))), CR being
collide-and-recolour of Sec. 2 / App. A (:func:`oracle.cmrt_oracle.step`).
For an objective J of the final state, the adjoint lam(t) = dJ/df(t) obeys

    lam(t) = CR'(f(t))^T stream^T lam(t+1),

and a parameter theta of CR collects dJ/dtheta = sum_t (dCR/dtheta)^T
stream^T lam(t+1).  Every function below is the transpose (vector-Jacobian
product) of the forward function of the same name in the oracle, taken
operation by operation in reverse order: streaming, recolour (Eq.
eq_re_color), reconstruction and relaxation (App. A, Eqs. 38, eq84), modal
equilibrium and sources, the correction tensor (Eq. Correction), the local
shear eigenvalue, the compact (or App. B) gradient stencils with their wall
mirrors, the force-adjusted velocity (Eq. equ_u_def), the force (Eq.
equ_stforce plus the body force), the curvature and the unit normal, the
colour index (Eq. equ_rhoN_def) and Phi', and the moments.

The objective used by the tests and the library is the L2 mismatch of the
final colour index, J = 1/2 sum_r (rho^N(r, T) - target(r))^2; the
controls are sigma, beta, lambda3_r, lambda3_b, g_acc and rho^N_0.
"""
from __future__ import annotations

import numpy as np

from . import cmrt_oracle as O

PARAM_NAMES = ("sigma", "beta", "lambda3_r", "lambda3_b", "g_acc_x", "g_acc_y")


# ---------------------------------------------------------------------------
# Transposes of the linear pieces
# ---------------------------------------------------------------------------
def _offset_rows(ny, dy, p: O.Params):
    """Source row and sign of value_at_offset for each output row."""
    ys = np.arange(ny) + dy
    if not p.wall_y:
        return np.mod(ys, ny), np.ones(ny)
    src = np.where(ys < 0, -1 - ys, np.where(ys >= ny, 2 * ny - 1 - ys, ys))
    sign = np.where((ys < 0) | (ys >= ny), -1.0, 1.0)
    return src, sign


def value_at_offset_T(adj, dx, dy, p: O.Params, parity=1):
    """Transpose of :func:`oracle.cmrt_oracle.value_at_offset` on a (ny, nx) field."""
    ny = adj.shape[-2]
    src, sign = _offset_rows(ny, dy, p)
    if parity == 1:
        sign = np.ones(ny)
    tmp = np.roll(adj, dx, axis=-1) * sign[:, None]
    out = np.zeros_like(adj)
    np.add.at(out, src, tmp)
    return out


def gradient_T(ax, ay, p: O.Params, parity=1, order=2):
    """Transpose of :func:`oracle.cmrt_oracle.gradient`: the field adjoint
    given the adjoints of its two gradient components (either may be None)."""
    coeffs = [(1, 3.0)] if order == 2 else [(1, 4.5), (2, -0.9), (3, 0.1)]
    ref = ax if ax is not None else ay
    out = np.zeros_like(ref)
    for n, a in coeffs:
        for i in range(1, 9):
            cx, cy = int(O.CX[i]), int(O.CY[i])
            acc = np.zeros_like(ref)
            if ax is not None and cx != 0:
                acc = acc + (a * O.W[i] * cx) * ax
            if ay is not None and cy != 0:
                acc = acc + (a * O.W[i] * cy) * ay
            out = out + value_at_offset_T(acc, n * cx, n * cy, p, parity)
    return out


def stream_T(adj, p: O.Params):
    """Transpose of :func:`oracle.cmrt_oracle.stream` (adjoint of C++ from the
    adjoint of the streamed populations), bounce-back included."""
    out = np.zeros_like(adj)
    ny = adj.shape[1]
    for i in range(9):
        cx, cy = int(O.CX[i]), int(O.CY[i])
        if not p.wall_y:
            moved = np.roll(adj[i], -cy, axis=0)
        else:
            moved = np.zeros_like(adj[i])
            if cy == 0:
                moved[:] = adj[i]
            elif cy == 1:
                moved[:-1] = adj[i][1:]
            else:
                moved[1:] = adj[i][:-1]
        out[i] = np.roll(moved, -cx, axis=1)
    if p.wall_y:
        for i in range(9):
            cy = int(O.CY[i])
            if cy == 1:
                out[i, ny - 1, :] += adj[O.OPPOSITE[i], ny - 1, :]
            elif cy == -1:
                out[i, 0, :] += adj[O.OPPOSITE[i], 0, :]
    return out


def _normalise_T(gx, gy, bx, by):
    """Adjoint of g -> g / |g| with the guard of the unit normal (the recolour
    direction e, and minus the unit normal): (I - e e^T) b / |g| where
    |g| >= NORMAL_TAU, and 0 below it, where the map is the constant 0."""
    mag = np.sqrt(gx * gx + gy * gy)
    big = mag >= O.NORMAL_TAU
    safe = np.where(big, mag, 1.0)
    ex, ey = gx / safe, gy / safe
    dot = ex * bx + ey * by
    outx = np.where(big, (bx - ex * dot) / safe, 0.0)
    outy = np.where(big, (by - ey * dot) / safe, 0.0)
    return outx, outy


# ---------------------------------------------------------------------------
# One step
# ---------------------------------------------------------------------------
def step_vjp(R, B, lamR, lamB, p: O.Params):
    """Adjoint of one step.

    R, B: pre-collision state f(t); lamR, lamB: dJ/df(t+1).  Returns
    (dJ/dR(t), dJ/dB(t), {parameter: dJ/dtheta contribution of this step})."""
    d = O.macroscopic(R, B, p)
    Rpp, Bpp = O.collide_and_recolour(R, B, p, d)  # fills dPx, dPy, divu, lam3
    f = R + B
    rho_r, rho_b, rho = d.rho_r, d.rho_b, d.rho
    ux, uy, Gx, Gy = d.ux, d.uy, d.Gx, d.Gy
    lam3 = d.lam3
    m = O.modes(f, p)
    meq = O.modal_equilibrium(rho_r, rho_b, ux, uy, p)
    cxx, cyy, cxy = O.correction_tensor(ux, uy, Gx, Gy, d.dPx, d.dPy, d.divu, rho, lam3, p)
    S = O.modal_sources(Gx, Gy, cxx, cyy, cxy, p)
    mplus = O.relax(m, meq, S, lam3, p)
    fplus = O.reconstruct(mplus, p)
    ex, ey = -d.nhx, -d.nhy

    grads = {k: 0.0 for k in PARAM_NAMES}
    z = np.zeros_like(rho)
    rr_bar, rb_bar, rho_bar = z.copy(), z.copy(), z.copy()
    ux_bar, uy_bar, Gx_bar, Gy_bar = z.copy(), z.copy(), z.copy(), z.copy()

    # -- streaming
    aR = stream_T(lamR, p)
    aB = stream_T(lamB, p)

    # -- recolour: C++_i = (rho_C / rho) f+_i +/- seg phi_i (e . c-hat_i)
    xR, xB = rho_r / rho, rho_b / rho
    fplus_bar = xR * aR + xB * aB
    xR_bar = np.sum(aR * fplus, axis=0)
    xB_bar = np.sum(aB * fplus, axis=0)
    rr_bar += (xR_bar - xB_bar) * rho_b / rho ** 2
    rb_bar += (xB_bar - xR_bar) * rho_r / rho ** 2
    dbar = aR - aB
    phi = O.phi_weights(rho_r, rho_b, p)
    seg = p.beta * rho_r * rho_b / rho
    seg_bar = z.copy()
    s_bar = z.copy()
    ex_bar, ey_bar = z.copy(), z.copy()
    for i in range(1, 9):
        norm = np.sqrt(float(O.CX[i] ** 2 + O.CY[i] ** 2))
        chx, chy = O.CX[i] / norm, O.CY[i] / norm
        ec = chx * ex + chy * ey
        seg_bar += dbar[i] * phi[i] * ec
        s_bar += dbar[i] * seg * ec * (O.K_PHI * O.W[i])
        ex_bar += dbar[i] * seg * phi[i] * chx
        ey_bar += dbar[i] * seg * phi[i] * chy
    grads["beta"] += float(np.sum(seg_bar * rho_r * rho_b / rho))
    rr_bar += seg_bar * p.beta * rho_b ** 2 / rho ** 2
    rb_bar += seg_bar * p.beta * rho_r ** 2 / rho ** 2
    cr, cb = 1.0 - p.alpha_r, 1.0 - p.alpha_b
    rr_bar += s_bar * (cr - cb) * rho_b / rho ** 2
    rb_bar += s_bar * (cb - cr) * rho_r / rho ** 2
    gx_bar, gy_bar = _normalise_T(d.gnx, d.gny, ex_bar, ey_bar)

    # -- reconstruction and relaxation
    mplus_bar = np.tensordot(O.MINV.T, fplus_bar, axes=(1, 0))
    lam = [0.0, 0.0, 0.0, lam3, lam3, lam3, p.lambda6, p.lambda7, p.lambda7]
    m_bar = np.empty_like(mplus_bar)
    meq_bar = np.empty_like(mplus_bar)
    for q in range(9):
        m_bar[q] = (1.0 - lam[q]) * mplus_bar[q]
        meq_bar[q] = lam[q] * mplus_bar[q]
    lam3_bar = sum(mplus_bar[q] * (meq[q] - m[q]) for q in (3, 4, 5))
    f_bar = np.tensordot(O.M.T, m_bar, axes=(1, 0))  # common to both colours
    # modal equilibrium
    rho_bar += meq_bar[0] + meq_bar[1] * ux + meq_bar[2] * uy + meq_bar[3] * ux * ux \
        + meq_bar[4] * uy * uy + meq_bar[5] * ux * uy
    ux_bar += meq_bar[1] * rho + 2.0 * rho * ux * meq_bar[3] + meq_bar[5] * rho * uy
    uy_bar += meq_bar[2] * rho + 2.0 * rho * uy * meq_bar[4] + meq_bar[5] * rho * ux
    pr_bar = meq_bar[3] + meq_bar[4]
    rr_bar += 0.6 * (1.0 - p.alpha_r) * pr_bar
    rb_bar += 0.6 * (1.0 - p.alpha_b) * pr_bar
    if p.ghost_N_mode == 0:
        rr_bar += (1.8 * p.alpha_r - 0.8) * meq_bar[6]
        rb_bar += (1.8 * p.alpha_b - 0.8) * meq_bar[6]
    # sources S = (0, Gx, Gy, Cxx, Cyy, Cxy, 0, 0, 0)
    Gx_bar += mplus_bar[1]
    Gy_bar += mplus_bar[2]
    cxx_bar, cyy_bar, cxy_bar = mplus_bar[3], mplus_bar[4], mplus_bar[5]
    # correction tensor
    a = 1.0 - lam3 / 2.0
    iso = ux * d.dPx + uy * d.dPy - rho * d.divu / 3.0
    hx, hy = Gx - d.dPx, Gy - d.dPy
    a_bar = cxx_bar * (2.0 * ux * hx - iso) + cyy_bar * (2.0 * uy * hy - iso) + cxy_bar * (ux * hy + uy * hx)
    lam3_bar = lam3_bar - 0.5 * a_bar
    iso_bar = -a * (cxx_bar + cyy_bar)
    hx_bar = a * (2.0 * ux * cxx_bar + uy * cxy_bar)
    hy_bar = a * (2.0 * uy * cyy_bar + ux * cxy_bar)
    ux_bar += a * (2.0 * hx * cxx_bar + hy * cxy_bar) + iso_bar * d.dPx
    uy_bar += a * (2.0 * hy * cyy_bar + hx * cxy_bar) + iso_bar * d.dPy
    Gx_bar += hx_bar
    Gy_bar += hy_bar
    dPx_bar = -hx_bar + iso_bar * ux
    dPy_bar = -hy_bar + iso_bar * uy
    rho_bar += -iso_bar * d.divu / 3.0
    divu_bar = -iso_bar * rho / 3.0
    # local shear eigenvalue lambda_3 = 2 / (6 nu + 1)
    nu = 2.0 / lam3 / 6.0 - 1.0 / 6.0
    nu_bar = lam3_bar * (-12.0 / (6.0 * nu + 1.0) ** 2)
    rn_bar = z.copy()
    if p.visc_mode == 1:
        rho_bar += nu_bar * (-p.eta / rho ** 2)
    else:
        nu_r = (2.0 / p.lambda3_r - 1.0) / 6.0
        nu_b = (2.0 / p.lambda3_b - 1.0) / 6.0
        rn_bar += nu_bar * 0.5 * (nu_r - nu_b)
        grads["lambda3_r"] += float(np.sum(nu_bar * 0.5 * (1.0 + d.rho_n))) * (-1.0 / (3.0 * p.lambda3_r ** 2))
        grads["lambda3_b"] += float(np.sum(nu_bar * 0.5 * (1.0 - d.rho_n))) * (-1.0 / (3.0 * p.lambda3_b ** 2))

    # -- grad Phi' and div u
    phip_bar = gradient_T(dPx_bar, dPy_bar, p, parity=1, order=p.stencil_order)
    ux_bar += gradient_T(divu_bar, None, p, parity=-1)
    uy_bar += gradient_T(None, divu_bar, p, parity=-1)

    # -- force-adjusted velocity u = (j + G/2) / rho
    jx_bar = ux_bar / rho
    jy_bar = uy_bar / rho
    Gx_bar += ux_bar / (2.0 * rho)
    Gy_bar += uy_bar / (2.0 * rho)
    rho_bar += -(ux * ux_bar + uy * uy_bar) / rho

    # -- force G = sigma K grad rho^N / 2 + rho g_acc + g_vol
    hs = 0.5 * p.sigma
    K_bar = hs * (Gx_bar * d.gnx + Gy_bar * d.gny)
    gx_bar += hs * d.K * Gx_bar
    gy_bar += hs * d.K * Gy_bar
    rho_bar += Gx_bar * p.g_acc[0] + Gy_bar * p.g_acc[1]
    grads["sigma"] += float(np.sum(0.5 * d.K * (Gx_bar * d.gnx + Gy_bar * d.gny)))
    grads["g_acc_x"] += float(np.sum(rho * Gx_bar))
    grads["g_acc_y"] += float(np.sum(rho * Gy_bar))

    # -- curvature K = div n-hat, unit normal n-hat = -g / |g| (0 below the guard)
    if p.curvature_mode == 0:
        nx_bar = gradient_T(K_bar, None, p, parity=1)
        ny_bar = gradient_T(None, K_bar, p, parity=-1)
        tx, ty = _normalise_T(d.gnx, d.gny, nx_bar, ny_bar)
        gx_bar -= tx
        gy_bar -= ty

    # -- grad rho^N
    rn_bar += gradient_T(gx_bar, gy_bar, p, parity=1, order=p.stencil_order)

    # -- colour index, Phi', densities
    A = rho_r / p.rho0_r
    Bn = rho_b / p.rho0_b
    den = (A + Bn) ** 2
    rr_bar += rn_bar * 2.0 * Bn / den / p.rho0_r
    rb_bar += rn_bar * (-2.0 * A / den) / p.rho0_b
    rr_bar += phip_bar * (0.6 * (1.0 - p.alpha_r) - 1.0 / 3.0)
    rb_bar += phip_bar * (0.6 * (1.0 - p.alpha_r) * p.Lambda - 1.0 / 3.0)
    rr_bar += rho_bar
    rb_bar += rho_bar

    # -- moments of the gathered populations
    lR = np.empty_like(R)
    lB = np.empty_like(B)
    for i in range(9):
        mom = O.CX[i] * jx_bar + O.CY[i] * jy_bar + f_bar[i]
        lR[i] = rr_bar + mom
        lB[i] = rb_bar + mom
    return lR, lB, grads


# ---------------------------------------------------------------------------
# Objective, initial state, whole runs
# ---------------------------------------------------------------------------
def objective(R, B, target, p: O.Params):
    """J = 1/2 sum_r (rho^N(r) - target(r))^2 of a pre-collision state."""
    rn = O.colour_index(R.sum(axis=0), B.sum(axis=0), p)
    return 0.5 * float(np.sum((rn - target) ** 2))


def objective_vjp(R, B, target, p: O.Params):
    """dJ/dR, dJ/dB of :func:`objective`."""
    rr, rb = R.sum(axis=0), B.sum(axis=0)
    A, Bn = rr / p.rho0_r, rb / p.rho0_b
    res = (A - Bn) / (A + Bn) - target
    den = (A + Bn) ** 2
    gR = res * 2.0 * Bn / den / p.rho0_r
    gB = res * (-2.0 * A / den) / p.rho0_b
    return np.broadcast_to(gR, R.shape).copy(), np.broadcast_to(gB, B.shape).copy()


def init_vjp(rho_n0, u0x, u0y, lamR, lamB, p: O.Params):
    """dJ/drho^N_0 through :func:`oracle.cmrt_oracle.init_state`."""
    rho_n0 = np.asarray(rho_n0, dtype=np.float64)
    rr = p.rho0_r * (1.0 + rho_n0) / 2.0
    rb = p.rho0_b * (1.0 - rho_n0) / 2.0
    rho = rr + rb
    f0 = O.equilibrium(rr, rb, u0x, u0y, p)
    xR, xB = rr / rho, rb / rho
    f0_bar = xR * lamR + xB * lamB
    xR_bar = np.sum(lamR * f0, axis=0)
    xB_bar = np.sum(lamB * f0, axis=0)
    rr_bar = (xR_bar - xB_bar) * rb / rho ** 2
    rb_bar = (xB_bar - xR_bar) * rr / rho ** 2
    # f0_i = rho phi_i(rho_R, rho_B) + w_i rho Q_i(u): rho phi_0 = alpha_r rho_R + alpha_b rho_B,
    # rho phi_i = k w_i ((1 - alpha_r) rho_R + (1 - alpha_b) rho_B)
    usq = u0x * u0x + u0y * u0y
    for i in range(9):
        cu = O.CX[i] * u0x + O.CY[i] * u0y
        Q = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq
        if i == 0:
            kr, kb = p.alpha_r, p.alpha_b
        else:
            kr, kb = O.K_PHI * O.W[i] * (1.0 - p.alpha_r), O.K_PHI * O.W[i] * (1.0 - p.alpha_b)
        rr_bar = rr_bar + f0_bar[i] * (kr + O.W[i] * Q)
        rb_bar = rb_bar + f0_bar[i] * (kb + O.W[i] * Q)
    return rr_bar * p.rho0_r / 2.0 - rb_bar * p.rho0_b / 2.0


def gradient_of_objective(rho_n0, u0x, u0y, target, p: O.Params, nsteps: int, ckpt_every: int = 200):
    """J and its gradient after ``nsteps`` steps from init_state(rho^N_0, u_0).

    Checkpoints every ``ckpt_every`` steps; each segment is recomputed
    forward from its checkpoint and then reversed.  Returns
    (J, {parameter: dJ/dtheta}, dJ/drho^N_0)."""
    R, B = O.init_state(rho_n0, u0x, u0y, p)
    ckpts = {0: (R, B)}
    for t in range(nsteps):
        R, B = O.step(R, B, p)
        if (t + 1) % ckpt_every == 0 and t + 1 < nsteps:
            ckpts[t + 1] = (R, B)
    J = objective(R, B, target, p)
    lR, lB = objective_vjp(R, B, target, p)
    grads = {k: 0.0 for k in PARAM_NAMES}
    starts = sorted(ckpts)
    for s0 in reversed(starts):
        s1 = min(s0 + ckpt_every, nsteps)
        states = [ckpts[s0]]
        for _ in range(s0, s1 - 1):
            states.append(O.step(*states[-1], p))
        for t in range(s1 - 1, s0 - 1, -1):
            lR, lB, g = step_vjp(*states[t - s0], lR, lB, p)
            for k in grads:
                grads[k] += g[k]
    return J, grads, init_vjp(rho_n0, u0x, u0y, lR, lB, p)
