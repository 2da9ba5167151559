"""Reference solutions used to pin the oracle (TEST INFRASTRUCTURE ONLY).

* single-phase shear-wave decay and body-force Poiseuille flow (textbook
  Navier-Stokes solutions that the scheme must reduce to when Lambda = 1 and
  sigma = 0; viscosity nu = (2/lambda_3 - 1)/6 from App. A, Eq. Correction);
* steady unidirectional flow through a continuous transverse density and
  viscosity profile, the generalisation of App. D to an arbitrary rho(y),
  nu(y) and a body force that may be per unit mass;
* transient unidirectional two-layer flow by Sturm-Liouville expansion
  (App. C, flat interface), written for unequal shear viscosities so that it
  reduces to App. C when eta_1 = eta_2.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import cumulative_trapezoid
from scipy.optimize import brentq


def nu_of_lambda3(lam3):
    """Kinematic viscosity of the MRT scheme, nu = (2/lambda_3 - 1)/6 (App. A)."""
    return (2.0 / lam3 - 1.0) / 6.0


def shear_wave_amplitude(nu, k, t):
    """Amplitude ratio of a decaying shear wave u_x = U sin(k y): exp(-nu k^2 t)."""
    return np.exp(-nu * k * k * t)


def poiseuille(ny, force_density, eta):
    """Steady channel flow between no-slip planes at y = -1/2 and y = ny - 1/2,
    eta u'' = -f:  u(y) = f/(2 eta) s (H - s), s = y + 1/2, H = ny."""
    s = np.arange(ny) + 0.5
    return force_density / (2.0 * eta) * s * (ny - s)


def layered_steady(rho_nodes, nu_nodes, g_acc=0.0, g_vol=0.0, samples_per_lu=400):
    """Steady u(y) of d/dy(eta du/dy) = -(rho g_acc + g_vol), u = 0 on the walls.

    Generalises App. D (Eqs. equ_ODE, equ_integral) from a symmetric profile
    and a pressure gradient to any continuous rho(y), nu(y) and a body force
    per unit mass and/or per unit volume.  Nodes sit at y = 0..H-1, walls at
    y = -1/2 and H - 1/2.  rho and nu are interpolated linearly between nodes
    and held constant over the half cell next to each wall.  Integrals are
    evaluated on a fine grid (trapezoid rule; App. D used Simpson's rule).
    Returns u at the nodes.
    """
    rho_nodes = np.asarray(rho_nodes, dtype=np.float64)
    nu_nodes = np.asarray(nu_nodes, dtype=np.float64)
    H = rho_nodes.size
    s = np.linspace(0.0, H, H * samples_per_lu + 1)
    y = s - 0.5
    yn = np.arange(H, dtype=np.float64)
    rho = np.interp(y, yn, rho_nodes)
    nu = np.interp(y, yn, nu_nodes)
    eta = rho * nu
    f = rho * g_acc + g_vol
    F = cumulative_trapezoid(f, s, initial=0.0)            # int_0^s f
    inv_eta = 1.0 / eta
    I1 = cumulative_trapezoid(inv_eta, s, initial=0.0)     # int_0^s 1/eta
    I2 = cumulative_trapezoid(F * inv_eta, s, initial=0.0)  # int_0^s F/eta
    tau0 = I2[-1] / I1[-1]
    u = tau0 * I1 - I2                                      # u(s), u(0) = u(H) = 0
    return np.interp(yn + 0.5, s, u)


def two_layer_transient(H, h, rho1, rho2, eta1, eta2, u1, u2, y, t, nmodes=200):
    """u(y, t) of rho(y) du/dt = d/dy(eta du/dy), u(0) = u(H) = 0, with a flat
    interface at y = h, fluid 1 (rho1, eta1) below, fluid 2 above, and the
    initial velocity u1 below, u2 above (App. C, flat interface).

    Eigenfunctions (App. C, Eqs. PHI1, PHI2): sin(c k_1 y) below and
    sin(c k_2 (y - H)) above, k_j = sqrt(rho_j / eta_j); continuity of u and
    of the traction eta du/dy at y = h gives the characteristic equation
    eta_1 k_1 cos(c k_1 h) sin(c k_2 (h - H)) = eta_2 k_2 sin(c k_1 h) cos(c k_2 (h - H)),
    written without tangents so that it has no poles.  With eta_1 = eta_2
    and h = H/2 it is App. C's tan-form equation.  Modes are normalised with
    weight rho (Eq. eq:Guess) and sigma_n = int rho u(y, 0) phi_n dy.
    """
    k1 = np.sqrt(rho1 / eta1)
    k2 = np.sqrt(rho2 / eta2)

    def char(c):
        return (eta1 * k1 * np.cos(c * k1 * h) * np.sin(c * k2 * (h - H))
                - eta2 * k2 * np.sin(c * k1 * h) * np.cos(c * k2 * (h - H)))

    # bracket sign changes on a fine scan
    cmax = (nmodes + 2) * np.pi / min(k1 * h, k2 * (H - h)) * 1.2
    grid = np.linspace(1e-9, cmax, 400 * (nmodes + 2))
    vals = char(grid)
    roots = []
    for a, b, fa, fb in zip(grid[:-1], grid[1:], vals[:-1], vals[1:]):
        if fa == 0.0:
            roots.append(a)
        elif fa * fb < 0.0:
            roots.append(brentq(char, a, b, xtol=1e-14, rtol=1e-14))
        if len(roots) >= nmodes:
            break
    y = np.asarray(y, dtype=np.float64)
    u = np.zeros_like(y)
    for c in roots:
        s1 = np.sin(c * k1 * h)
        s2 = np.sin(c * k2 * (h - H))
        if abs(s2) > 1e-12:
            A1, A2 = 1.0, s1 / s2
        else:  # interface at a node of the upper piece: use traction matching
            A1 = 1.0
            A2 = eta1 * k1 * np.cos(c * k1 * h) / (eta2 * k2 * np.cos(c * k2 * (h - H)))
        # rho-weighted norm, exact integrals of sin^2
        n1 = rho1 * A1 * A1 * (h / 2.0 - np.sin(2.0 * c * k1 * h) / (4.0 * c * k1))
        L2 = H - h
        n2 = rho2 * A2 * A2 * (L2 / 2.0 - np.sin(2.0 * c * k2 * L2) / (4.0 * c * k2))
        norm = np.sqrt(n1 + n2)
        A1 /= norm
        A2 /= norm
        # sigma_n = int rho u0 phi
        i1 = A1 * (1.0 - np.cos(c * k1 * h)) / (c * k1)
        i2 = A2 * (np.cos(c * k2 * (h - H)) - 1.0) / (c * k2)
        sig = rho1 * u1 * i1 + rho2 * u2 * i2
        phi = np.where(y < h, A1 * np.sin(c * k1 * y), A2 * np.sin(c * k2 * (y - H)))
        u += sig * np.exp(-c * c * t) * phi
    return u


def layered_transient(rho_nodes, eta_nodes, u_init_nodes, t, refine=2):
    """u(y, t) of rho(y) du/dt = d/dy(eta(y) du/dy), u = 0 on walls at
    y = -1/2 and H - 1/2 (App. C, Eq. eq:Main), for a continuous density and
    viscosity profile given at the nodes y = 0..H-1.

    The paper's App. C treats the interface as sharp; this solves the same
    equation with the diffuse profile the lattice actually carries, by
    expansion on the eigenvectors of a fine second-order finite-volume
    discretisation (``refine`` cells per lattice unit; the generalised
    symmetric eigenproblem K v = c^2 M v mirrors App. C's Sturm-Liouville
    problem with weight rho).  The initial velocity is piecewise constant on
    each lattice cell.  Returns u at the nodes.
    """
    from scipy.linalg import eigh
    rho_nodes = np.asarray(rho_nodes, dtype=np.float64)
    eta_nodes = np.asarray(eta_nodes, dtype=np.float64)
    H = rho_nodes.size
    n = H * refine
    h = 1.0 / refine
    yc = (np.arange(n) + 0.5) * h - 0.5          # fine cell centres in lattice y
    node_of = np.clip(np.floor(yc + 0.5).astype(int), 0, H - 1)
    rho = np.interp(yc, np.arange(H), rho_nodes)
    eta_c = np.interp(yc, np.arange(H), eta_nodes)
    # face viscosities (harmonic mean inside, wall faces use the cell value)
    eta_f = np.empty(n + 1)
    eta_f[1:-1] = 2.0 * eta_c[:-1] * eta_c[1:] / (eta_c[:-1] + eta_c[1:])
    eta_f[0] = eta_c[0]
    eta_f[-1] = eta_c[-1]
    # stiffness (walls: u = 0 at the faces, half-cell distance)
    diag = np.empty(n)
    diag[:] = (eta_f[:-1] + eta_f[1:]) / (h * h)
    diag[0] = (eta_f[1] + 2.0 * eta_f[0]) / (h * h)
    diag[-1] = (eta_f[-2] + 2.0 * eta_f[-1]) / (h * h)
    off = -eta_f[1:-1] / (h * h)
    K = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    Mdiag = rho
    # symmetric form: M^{-1/2} K M^{-1/2}
    s = 1.0 / np.sqrt(Mdiag)
    A = K * s[:, None] * s[None, :]
    lam, V = eigh(A)
    u0 = np.asarray(u_init_nodes, dtype=np.float64)[node_of]
    w0 = V.T @ (u0 * np.sqrt(Mdiag))
    w = w0 * np.exp(-lam * t)
    uf = (V @ w) * s
    # average the fine cells back onto the nodes
    return uf.reshape(H, refine).mean(axis=1)


def app_d_steady(rho_nodes, nu, G, samples_per_half_lu=200):
    """App. D, Eq. equ_integral: steady pressure-driven flow through the
    symmetric stratified channel (walls at y = -1/2 and H - 1/2, profile
    symmetric about the channel centre):

        u(x) = G / (2 nu) * int_0^x (H - 2a) / rho(a) da,   x <= H/2,

    mirrored about H/2, with x = y + 1/2 the distance from the wall.  The sign
    is taken so that the flow follows the force (the printed form has
    d/dx(eta du/dx) = +G with the pressure gradient -G).  rho is interpolated
    linearly between nodes and held constant over the half cell next to each
    wall; the integral is evaluated by the composite Simpson rule, as App. D
    does, on a grid of 2 * samples_per_half_lu intervals per lattice unit.
    Returns u at the nodes."""
    rho_nodes = np.asarray(rho_nodes, dtype=np.float64)
    H = rho_nodes.size
    m = 2 * int(samples_per_half_lu)            # intervals per lattice unit (even)
    x = np.linspace(0.0, H / 2.0, H * m // 2 + 1)
    rho = np.interp(x - 0.5, np.arange(H, dtype=np.float64), rho_nodes)
    f = (H - 2.0 * x) / rho
    h = x[1] - x[0]
    # cumulative composite Simpson rule at every even grid point
    pair = h / 3.0 * (f[:-2:2] + 4.0 * f[1:-1:2] + f[2::2])
    I = np.concatenate([[0.0], np.cumsum(pair)])
    xe = x[::2]
    half = G / (2.0 * nu) * I
    s = np.arange(H, dtype=np.float64) + 0.5
    d = np.minimum(s, H - s)                   # distance to the nearer wall
    return np.interp(d, xe, half)
