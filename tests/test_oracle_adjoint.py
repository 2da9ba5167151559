"""Pins of the oracle's discrete adjoint (oracle/cmrt_adjoint.py).

The adjoint is checked against the forward oracle, never against itself:
- each transposed linear piece (offsets with wall mirrors, gradient stencils,
  streaming with bounce-back) satisfies <A x, y> = <x, A^T y> with the
  oracle's own forward A;
- the vector-Jacobian product of a whole step, the parameter gradients and
  the gradient of the colour-field objective through several checkpointed
  steps agree with fourth-order central finite differences of the FP64
  forward oracle (step h = 1e-6: truncation ~h^4 and round-off ~1e-16/h
  both far below the 1e-6 tolerance, also on rough states where 1/|grad
  rho^N| makes the higher derivatives large).
"""
import dataclasses

import numpy as np
import pytest

from oracle import cmrt_adjoint as A
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I


H = 1e-6


def fd4(fun):
    """d/ds fun(s) at 0, fourth-order central difference with step H."""
    return (8.0 * (fun(H) - fun(-H)) - (fun(2 * H) - fun(-2 * H))) / (12.0 * H)


def _params(nx, ny, **kw):
    d = I.base_params(nx, ny, **kw)
    return O.Params(**d)


@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("dx,dy", [(1, 0), (-1, 1), (2, -2), (-3, 3), (0, -1)])
def test_offset_transpose(wall, parity, dx, dy):
    p = _params(7, 6, wall_y=wall)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((2, 6, 7))
    lhs = np.sum(O.value_at_offset(a, dx, dy, p, parity) * b)
    rhs = np.sum(a * A.value_at_offset_T(b, dx, dy, p, parity))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-13


@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("order", [2, 6])
def test_gradient_transpose(wall, parity, order):
    p = _params(9, 8, wall_y=wall)
    rng = np.random.default_rng(2)
    a, bx, by = rng.standard_normal((3, 8, 9))
    gx, gy = O.gradient(a, p, parity=parity, order=order)
    lhs = np.sum(gx * bx + gy * by)
    rhs = np.sum(a * A.gradient_T(bx, by, p, parity=parity, order=order))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("wall", [False, True])
def test_stream_transpose(wall):
    p = _params(6, 5, wall_y=wall)
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2, 9, 5, 6))
    lhs = np.sum(O.stream(a, p) * b)
    rhs = np.sum(a * A.stream_T(b, p))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _shifted(p, name, s):
    """p with parameter ``name`` (one of PARAM_NAMES) moved by s."""
    if name.startswith("g_acc"):
        g = list(p.g_acc)
        g[0 if name.endswith("x") else 1] += s
        return dataclasses.replace(p, g_acc=tuple(g))
    return dataclasses.replace(p, **{name: getattr(p, name) + s})


def _state(p, seed, drop=True):
    """A drop with a rough velocity: interfaces, forces and recolour all active."""
    rng = np.random.default_rng(seed)
    if drop:
        rn = I.drops_field(p.nx, p.ny, [(p.nx / 2 + 0.3, p.ny / 2 - 0.2)], [min(p.nx, p.ny) / 3.0],
                           periodic_y=not p.wall_y)
        rn = np.clip(rn + 0.05 * rng.standard_normal(rn.shape), -0.97, 0.97)
    else:
        rn, _ = I.random_state_fields(p.nx, p.ny, seed)
    u = rng.uniform(-0.03, 0.03, size=(2, p.ny, p.nx))
    R, B = O.init_state(rn, u[0], u[1], p)
    # one step of the scheme off equilibrium, plus noise in every population
    R, B = O.step(R, B, p)
    R = R * (1.0 + 0.01 * rng.standard_normal(R.shape))
    B = B * (1.0 + 0.01 * rng.standard_normal(B.shape))
    return R, B


STEP_CASES = [
    ("periodic", dict()),
    ("walls_gravity", dict(wall_y=True, g_acc=(2e-4, -3e-4))),
    ("rates_ghostN", dict(lambda3_r=1.5, lambda3_b=0.7, lambda6=1.2, lambda7=0.8, ghost_N_mode=1)),
    ("visc_eta_fixedK", dict(visc_mode=1, eta=0.2, curvature_mode=1, fixed_K=0.05, g_vol=(1e-4, 0.0))),
    ("order6_lambda100", dict(stencil_order=6, rho0_b=0.01, alpha_r=0.995, sigma=0.02)),
]


@pytest.mark.parametrize("name,kw", STEP_CASES)
def test_step_vjp_matches_finite_differences(name, kw):
    p = _params(10, 9, sigma=kw.pop("sigma", 0.01), **kw)
    R, B = _state(p, seed=4, drop=(name != "rates_ghostN"))
    rng = np.random.default_rng(5)
    lR, lB = rng.standard_normal((2,) + R.shape)
    vR, vB = rng.standard_normal((2,) + R.shape)
    gR, gB, _ = A.step_vjp(R, B, lR, lB, p)

    def lin(s):
        Rn, Bn = O.step(R + s * vR, B + s * vB, p)
        return np.sum(lR * Rn) + np.sum(lB * Bn)

    fd = fd4(lin)
    ad = np.sum(gR * vR) + np.sum(gB * vB)
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("wall", [False, True])
def test_step_parameter_gradients_match_finite_differences(wall):
    p = _params(10, 8, sigma=0.01, wall_y=wall, g_acc=(1e-4, -2e-4), lambda3_r=1.3, lambda3_b=0.8)
    R, B = _state(p, seed=6)
    rng = np.random.default_rng(7)
    lR, lB = rng.standard_normal((2,) + R.shape)
    _, _, g = A.step_vjp(R, B, lR, lB, p)

    def lin(q):
        Rn, Bn = O.step(R, B, q)
        return np.sum(lR * Rn) + np.sum(lB * Bn)

    for name in A.PARAM_NAMES:
        fd = fd4(lambda s: lin(_shifted(p, name, s)))
        assert abs(fd - g[name]) <= 1e-6 * max(abs(g[name]), 1e-3), (name, fd, g[name])


def test_objective_gradient_through_checkpointed_steps():
    """J after 7 steps, checkpoints every 3 (segments of 3, 3 and 1 steps)."""
    p = _params(12, 10, sigma=0.01, g_acc=(0.0, -1e-4), lambda3_r=1.2, lambda3_b=0.9)
    rng = np.random.default_rng(8)
    rn0 = I.drops_field(12, 10, [(6.2, 4.9)], [3.5])
    u0 = rng.uniform(-0.01, 0.01, size=(2, 10, 12))
    target = np.clip(rn0 + 0.2 * rng.standard_normal(rn0.shape), -1.0, 1.0)
    nsteps = 7
    J, g, grn = A.gradient_of_objective(rn0, u0[0], u0[1], target, p, nsteps, ckpt_every=3)

    def J_of(q, rn):
        R, B = O.init_state(rn, u0[0], u0[1], q)
        R, B = O.run(R, B, q, nsteps)
        return A.objective(R, B, target, q)

    assert abs(J - J_of(p, rn0)) <= 1e-12 * J
    v = rng.standard_normal(rn0.shape)
    fd = fd4(lambda s: J_of(p, rn0 + s * v))
    ad = float(np.sum(grn * v))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    for name in A.PARAM_NAMES:
        fd = fd4(lambda s: J_of(_shifted(p, name, s), rn0))
        assert abs(fd - g[name]) <= 1e-6 * max(abs(g[name]), 1e-4 * J), (name, fd, g[name])


def test_checkpoint_interval_does_not_change_gradient():
    p = _params(8, 8, sigma=0.01)
    rn0 = I.drops_field(8, 8, [(4.0, 4.0)], [2.5])
    z = np.zeros((8, 8))
    target = np.zeros((8, 8))
    a = A.gradient_of_objective(rn0, z, z, target, p, 5, ckpt_every=1)
    b = A.gradient_of_objective(rn0, z, z, target, p, 5, ckpt_every=200)
    assert a[0] == b[0]
    np.testing.assert_allclose(a[2], b[2], rtol=0, atol=1e-15 * np.abs(a[2]).max())
    for k in A.PARAM_NAMES:
        assert abs(a[1][k] - b[1][k]) <= 1e-13 * max(abs(a[1][k]), 1e-300)
