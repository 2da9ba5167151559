"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the lattice Boltzmann method itself: it
only builds initial colour fields rho^N_0(x, y), initial velocities u_0 and
plain dictionaries of parameter values for the workloads the library is
measured on.  Both the CUDA path and the CPU oracle consume its arrays.

Colour fields are tanh profiles of width ``width`` lattice units: a drop of
radius R centred at c is rho^N_0 = tanh((R - |r - c|) / width) with the
minimum-image distance on periodic axes; several drops are combined by taking
the pointwise maximum (union).  A flat layer is tanh((y_i - y) / width) with
the heavy (red, rho^N = +1) fluid below y_i.
"""
from __future__ import annotations

import math

import numpy as np


def alpha_split(Lambda: float, alpha_light: float = 0.5):
    """(alpha_r, alpha_b) for density ratio Lambda = rho0_r / rho0_b.

    The lighter fluid keeps the rest fraction ``alpha_light`` (0.5 in the
    paper's micro-current tables) and the heavier one gets
    1 - (1 - alpha_light) / Lambda, so that (1 - alpha_b)/(1 - alpha_r) = Lambda.
    For Lambda < 1 the roles swap.
    """
    if Lambda >= 1.0:
        return 1.0 - (1.0 - alpha_light) / Lambda, alpha_light
    return alpha_light, 1.0 - (1.0 - alpha_light) * Lambda


def base_params(nx, ny, rho0_r=1.0, rho0_b=0.1, alpha_light=0.5, **kw):
    """Plain parameter dictionary (keys match both the oracle and the binding)."""
    a_r, a_b = alpha_split(rho0_r / rho0_b, alpha_light)
    d = dict(nx=int(nx), ny=int(ny), rho0_r=float(rho0_r), rho0_b=float(rho0_b),
             alpha_r=a_r, alpha_b=a_b, sigma=0.005, beta=0.67,
             lambda3_r=1.0, lambda3_b=1.0, lambda6=1.0, lambda7=1.0,
             g_acc=(0.0, 0.0), g_vol=(0.0, 0.0), wall_y=False, visc_mode=0,
             eta=1.0 / 6.0, stencil_order=2, curvature_mode=0, fixed_K=0.0,
             ghost_N_mode=0)
    d.update(kw)
    return d


def lambda3_for_nu(nu: float) -> float:
    """Shear eigenvalue giving kinematic viscosity nu (nu = (2/lambda3 - 1)/6)."""
    return 2.0 / (6.0 * nu + 1.0)


def drops_field(nx, ny, centres, radii, width=2.0, periodic_y=True, dtype=np.float64):
    """Union of tanh drops; only a bounding box around each drop is touched."""
    out = np.full((ny, nx), -1.0, dtype=np.float64)
    pad = 12.0 * width
    for (cx, cy), r in zip(centres, radii):
        half = int(math.ceil(r + pad))
        xs = np.arange(int(math.floor(cx)) - half, int(math.floor(cx)) + half + 2)
        ys = np.arange(int(math.floor(cy)) - half, int(math.floor(cy)) + half + 2)
        xs = np.unique(np.mod(xs, nx))
        if periodic_y:
            ys = np.unique(np.mod(ys, ny))
        else:
            ys = ys[(ys >= 0) & (ys < ny)]
        dx = xs[None, :] - cx
        dx = dx - nx * np.round(dx / nx)
        dy = ys[:, None] - cy
        if periodic_y:
            dy = dy - ny * np.round(dy / ny)
        d = np.sqrt(dx * dx + dy * dy)
        val = np.tanh((r - d) / width)
        sub = out[np.ix_(ys, xs)]
        out[np.ix_(ys, xs)] = np.maximum(sub, val)
    return out.astype(dtype)


def layer_field(nx, ny, y_interface, width=2.0, heavy_below=True, dtype=np.float64):
    """Flat interface at y = y_interface, heavy (rho^N = +1) fluid below."""
    y = np.arange(ny, dtype=np.float64)[:, None]
    prof = np.tanh((y_interface - y) / width)
    if not heavy_below:
        prof = -prof
    return np.broadcast_to(prof, (ny, nx)).astype(dtype).copy()


def velocity_noise(nx, ny, amplitude, seed, dtype=np.float64):
    """u_0 with both components uniform in [-amplitude, amplitude]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-amplitude, amplitude, size=(2, ny, nx))
    return u.astype(dtype)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def static_drop(n=64, radius=16.0, Lambda=10.0, noise=1e-6, seed=1):
    """Centred drop, fully periodic, heavy fluid (1.0) inside, light (1/Lambda) outside."""
    p = base_params(n, n, rho0_r=1.0, rho0_b=1.0 / Lambda, sigma=0.005, beta=0.67)
    rho_n = drops_field(n, n, [(n / 2.0, n / 2.0)], [radius])
    u = velocity_noise(n, n, noise, seed)
    return p, rho_n, u


def layered_channel(nx=1024, ny=128, Lambda=100.0, visc_ratio=1.0, g=1e-6, seed=2):
    """Heavy fluid below y = ny/2, light above, walls in y, body force along x."""
    nu_r = 1.0 / 6.0
    p = base_params(nx, ny, rho0_r=1.0, rho0_b=1.0 / Lambda, sigma=0.005, beta=0.67,
                    lambda3_r=lambda3_for_nu(nu_r), lambda3_b=lambda3_for_nu(nu_r * visc_ratio),
                    g_acc=(g, 0.0), wall_y=True)
    rho_n = layer_field(nx, ny, ny / 2.0)
    u = np.zeros((2, ny, nx))
    return p, rho_n, u


def random_drops(nx, ny, ndrops, rmin, rmax, seed, Lambda=10.0, periodic_y=True, **kw):
    """``ndrops`` drops with centres uniform in the box and radii uniform in [rmin, rmax]."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(0.0, nx, ndrops)
    cy = rng.uniform(0.0, ny, ndrops)
    r = rng.uniform(rmin, rmax, ndrops)
    p = base_params(nx, ny, rho0_r=1.0, rho0_b=1.0 / Lambda, **kw)
    rho_n = drops_field(nx, ny, list(zip(cx, cy)), list(r), periodic_y=periodic_y)
    return p, rho_n, np.zeros((2, ny, nx))


def drops_8192(seed=3, n=8192, ndrops=64):
    """Throughput workload: n x n periodic, 64 drops, radii uniform in [8, 64], Lambda = 10."""
    return random_drops(n, n, ndrops, 8.0, 64.0, seed, Lambda=10.0)


def random_state_fields(nx, ny, seed, amplitude=0.05):
    """A rough, non-equilibrium colour field and velocity for brute-force parity:
    rho^N_0 uniform in (-1, 1) smoothed over one neighbour, u_0 uniform."""
    rng = np.random.default_rng(seed)
    rn = rng.uniform(-0.95, 0.95, size=(ny, nx))
    rn = 0.5 * rn + 0.125 * (np.roll(rn, 1, 0) + np.roll(rn, -1, 0) + np.roll(rn, 1, 1) + np.roll(rn, -1, 1))
    u = rng.uniform(-amplitude, amplitude, size=(2, ny, nx))
    return rn, u


def buoyant_drops(nx=16384, ny=8192, ndrops=256, seed=4, rmin=10.0, rmax=40.0, g=1e-6, Lambda=10.0):
    """Light drops rising in a heavy ambient between walls at y = -1/2 and ny - 1/2.

    Heavy (red, rho0 = 1) ambient, light (blue, rho0 = 1/Lambda) drops with
    centres uniform in the box (kept clear of the walls by their radius) and
    radii uniform in [rmin, rmax], gravity g along -y.  Smaller boxes keep the
    drop count per unit area (replicas of the same seeded field)."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, ndrops)
    cx = rng.uniform(0.0, nx, ndrops)
    cy = rng.uniform(0.0, 1.0, ndrops) * (ny - 2 * r - 4) + r + 2
    p = base_params(nx, ny, rho0_r=1.0, rho0_b=1.0 / Lambda, wall_y=True, g_acc=(0.0, -g))
    blue = drops_field(nx, ny, list(zip(cx, cy)), list(r), periodic_y=False)
    return p, -blue, np.zeros((2, ny, nx))


def buoyant_replica(side=512, seed=4, **kw):
    """Same generator on a side x side box with the drop count scaled by area."""
    ndrops = max(1, int(round(256 * side * side / (16384 * 8192))))
    return buoyant_drops(nx=side, ny=side, ndrops=ndrops, seed=seed, **kw)


BATCH_SIDES = (64, 128, 256, 512)


def batch_ensemble(n=512, seed=5, sides=BATCH_SIDES):
    """``n`` independent periodic lattices: side drawn uniformly from ``sides``,
    one centred drop of radius side/4, sigma uniform in [0.001, 0.02], Lambda
    log-uniform in [1, 100] (heavy fluid inside).  Returns a list of
    (params, rho^N_0 as float32, None) triples; u_0 = 0."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=n)
    sigma = rng.uniform(0.001, 0.02, size=n)
    Lam = np.exp(rng.uniform(0.0, math.log(100.0), size=n))
    members = []
    for k in range(n):
        s = int(side[k])
        p = base_params(s, s, rho0_r=1.0, rho0_b=1.0 / float(Lam[k]), sigma=float(sigma[k]))
        rho_n = drops_field(s, s, [(s / 2.0, s / 2.0)], [s / 4.0], dtype=np.float32)
        members.append((p, rho_n, None))
    return members


def ba_channel(H=200, nx=4, nu=0.333, G=1e-8, width=2.0, beta=0.67, stencil_order=6):
    """Steady stratified channel flow of Sec. 4 (the Ba test, App. D).

    Walls at y = -1/2 and H - 1/2 (H = L_x = 200 in the paper), the heavy (red)
    fluid in the middle half and the light (blue) fluid next to both walls,
    interfaces at H/4 and 3H/4 from the wall; alpha_B = 0.2, alpha_R = 0.9,
    so Lambda = (1 - alpha_B) / (1 - alpha_R) = 8; both fluids nu = 0.333; a
    uniform force per unit volume G along x stands for the pressure gradient.
    The flow is invariant along x, so a few columns carry it.  The paper
    computes the colour gradient with App. B's stencil here.  beta (the
    recolour parameter) is not printed for this test: 0.67 as elsewhere."""
    p = base_params(nx, H, rho0_r=1.0, rho0_b=0.125, sigma=0.005, beta=beta, wall_y=True,
                    lambda3_r=lambda3_for_nu(nu), lambda3_b=lambda3_for_nu(nu), g_vol=(G, 0.0),
                    stencil_order=stencil_order)
    p["alpha_r"], p["alpha_b"] = 0.9, 0.2
    y = np.arange(H, dtype=np.float64)
    lo, hi = H / 4.0 - 0.5, 3.0 * H / 4.0 - 0.5  # node coordinates of the two interfaces
    prof = np.where(y < (H - 1) / 2.0, np.tanh((y - lo) / width), np.tanh((hi - y) / width))
    rho_n = np.broadcast_to(prof[:, None], (H, nx)).copy()
    return p, rho_n, np.zeros((2, H, nx))


MICRO_CURRENT_LAMBDAS = (0.001, 0.01, 0.1, 10.0, 100.0, 1000.0)


def micro_current_drop(Lambda, n=200, radius=60.0, fixed_K=False, sigma=0.005, beta=0.67, nu=1.0 / 6.0,
                       centre=None):
    """Static red drop of Sec. 4.2 (the micro-current study): radius 60,
    centred in a 200 x 200 periodic box, at rest.  Lambda = rho0_R / rho0_B
    with the larger density 1; alpha as in the paper's tables (the lighter
    fluid 0.5).  fixed_K replaces the computed curvature by K = 1/R.  The
    paper prints neither sigma, beta nor nu for this study: 0.005, 0.67 and
    1/6 as in the static-drop workload.  centre (x, y) moves the drop off
    the box centre (default (n/2, n/2), a lattice node)."""
    rho0_r, rho0_b = (1.0, 1.0 / Lambda) if Lambda >= 1.0 else (Lambda, 1.0)
    p = base_params(n, n, rho0_r=rho0_r, rho0_b=rho0_b, sigma=sigma, beta=beta,
                    lambda3_r=lambda3_for_nu(nu), lambda3_b=lambda3_for_nu(nu))
    if fixed_K:
        p["curvature_mode"], p["fixed_K"] = 1, 1.0 / radius
    rho_n = drops_field(n, n, [(n / 2.0, n / 2.0) if centre is None else tuple(centre)], [radius])
    return p, rho_n, np.zeros((2, n, n))
