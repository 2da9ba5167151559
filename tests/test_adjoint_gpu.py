"""Discrete adjoint of the CUDA step (cmrt_step_vjp, cmrt_adjoint) against the
FP64 oracle adjoint (oracle/cmrt_adjoint.py, itself pinned by finite
differences of the forward oracle) and against central finite differences of
the FP64 forward oracle.

Tolerances: the CUDA adjoint runs in FP32 on an FP32 forward trajectory.  One
reverse step, given the same FP32 state, is compared element by element at
2e-5 of the largest adjoint entry and parameter gradients at 1e-4 relative
(FP32 rounding of O(1) populations, amplified by the 1/rho and 1/|grad rho^N|
factors of the recolour and normal adjoints).  Over tens to hundreds of steps
the FP32 forward trajectory itself moves the final colour field by ~1e-6, so
J is compared at 1e-4 relative, and the objective's target is chosen so that
the residual rho^N - target (O(0.1) at the interface) is far above that
drift; gradients are then held to 1e-4 relative, the bar the target
statement sets against finite differences.
"""
import numpy as np
import pytest

from oracle import cmrt_adjoint as A
from oracle import cmrt_oracle as O
from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()

PN = cm.ADJOINT_PARAMS


def _state32(d, seed):
    """An FP32 off-equilibrium state with a drop: (R, B) as float32."""
    p = O.Params(**d)
    rng = np.random.default_rng(seed)
    rn = I.drops_field(d["nx"], d["ny"], [(d["nx"] / 2 + 0.3, d["ny"] / 2 - 0.2)], [min(d["nx"], d["ny"]) / 3.5],
                       periodic_y=not d["wall_y"])
    u = rng.uniform(-0.02, 0.02, size=(2, d["ny"], d["nx"]))
    R, B = O.init_state(rn, u[0], u[1], p)
    R, B = O.step(R, B, p)
    R = R * (1.0 + 0.005 * rng.standard_normal(R.shape))
    B = B * (1.0 + 0.005 * rng.standard_normal(B.shape))
    return R.astype(np.float32), B.astype(np.float32)


VJP_CASES = [
    ("periodic", dict()),
    ("walls_gravity", dict(wall_y=True, g_acc=(2e-4, -3e-4))),
    ("rates_ghostN", dict(lambda3_r=1.5, lambda3_b=0.7, lambda6=1.2, lambda7=0.8, ghost_N_mode=1)),
    ("visc_eta_fixedK", dict(visc_mode=1, eta=0.2, curvature_mode=1, fixed_K=0.05, g_vol=(1e-4, 0.0))),
    ("ragged_walls", dict(wall_y=True, sigma=0.02, size=(131, 37))),
    # the fused reverse kernels' tiling: a lattice narrower than their 128-column
    # window and shorter than a row segment; three strips of many 4-row
    # segments, so that every strip and segment seam is crossed
    ("tiny_periodic", dict(size=(5, 4))),
    ("multi_segment", dict(size=(250, 70), g_acc=(1e-4, 2e-4))),
]


@pytest.mark.parametrize("fused", [1, 2], ids=["fused_kernels", "plane_passes"])
@pytest.mark.parametrize("name,kw", VJP_CASES)
def test_step_vjp_matches_oracle_adjoint(name, kw, fused):
    kw = dict(kw)
    nx, ny = kw.pop("size", (40, 24))
    d = I.base_params(nx, ny, sigma=kw.pop("sigma", 0.01), **kw)
    p = O.Params(**d)
    R, B = _state32(d, seed=3)
    lat = cm.Lattice(dict(d, adjoint_fused=fused), None, None)
    lat.set_populations(np.stack([R, B]))
    rng = np.random.default_rng(4)
    lam_next = rng.standard_normal((2, 9, ny, nx)).astype(np.float32)
    got, g = lat.step_vjp(lam_next)
    lR, lB, gref = A.step_vjp(R.astype(np.float64), B.astype(np.float64), lam_next[0].astype(np.float64),
                              lam_next[1].astype(np.float64), p)
    ref = np.stack([lR, lB])
    err = np.abs(got.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err <= 2e-5, err
    scale = max(abs(v) for v in gref.values())
    for k, name_ in enumerate(PN):
        assert abs(g[k] - gref[name_]) <= 1e-4 * max(abs(gref[name_]), 1e-3 * scale), (name_, g[k], gref[name_])
    assert lat.time == 0  # the VJP does not advance the state
    lat.close()


# Drop centres sit off the lattice nodes.  At a node-centred drop the colour
# gradient at the centre node is zero by symmetry and, once gravity breaks the
# symmetry, grows through the unit normal's guard (1e-9): there the normal's
# direction, and through K the force on the neighbours, depends on the
# gradient with a gain 1/|grad rho^N| of up to 1e9, so a derivative of the
# step is fixed only as well as that tiny gradient is -- in FP32 to ~1e-10,
# i.e. to tens of percent.  Off-node centres keep every gradient near a drop's
# centre at ~1e-3, where FP32 resolves the map's derivative like any other.
DROP_OFFSET = (0.3, -0.2)


def _drop_setup(n, radius, nsteps, g=1e-5, sigma=0.005, Lam=10.0, seed=9, wall=False, shift=(1.0, 0.5)):
    d = I.base_params(n, n, rho0_r=1.0, rho0_b=1.0 / Lam, sigma=sigma, g_acc=(0.0, -g), wall_y=wall,
                      lambda3_r=1.1, lambda3_b=0.9)
    cx, cy = n / 2.0 + DROP_OFFSET[0], n / 2.0 + DROP_OFFSET[1]
    rn0 = I.drops_field(n, n, [(cx, cy)], [radius], periodic_y=not wall)
    u0 = np.zeros((2, n, n))
    # target: the final colour field of a run with sigma 5 % larger (Sec. 2
    # force) from a drop displaced by `shift`, so that the residual at the
    # interface is O(0.1), far above the FP32 drift of the forward run
    pt = O.Params(**dict(d, sigma=1.05 * sigma))
    rt0 = I.drops_field(n, n, [(cx + shift[0], cy + shift[1])], [radius], periodic_y=not wall)
    Rt, Bt = O.run(*O.init_state(rt0, u0[0], u0[1], pt), pt, nsteps)
    target = O.colour_index(Rt.sum(0), Bt.sum(0), pt)
    return d, rn0, u0, target


def _gpu_trajectory(d, rn32, u32, nsteps):
    """Pre-collision FP32 states f(0..nsteps) of the CUDA forward run, as float64."""
    lat = cm.Lattice(d, rn32, u32)
    states = []
    for t in range(nsteps + 1):
        if t:
            lat.step(1)
        s = lat.populations().double().cpu().numpy()
        states.append((s[0], s[1]))
    lat.close()
    return states


@pytest.mark.parametrize("wall", [False, True])
def test_adjoint_gradient_matches_oracle(wall):
    """Through 30 steps with checkpoints every 7.  (a) The oracle adjoint
    evaluated on the CUDA forward trajectory (the same FP32 states) isolates
    the reverse arithmetic: FP32 rounding accumulated over 30 reverse steps,
    held to 1e-4 of each gradient plus 1e-5 of the largest one (a component
    that is a small sum of large, cancelling node contributions, here
    dJ/dlambda3_b, is only known to that absolute level).  (b) The oracle's
    own FP64 trajectory differs from the FP32 one by the drift of the forward
    run, which moves the gradients by up to ~1e-3 here (gravity 1e-4 on a
    radius-6 drop): that comparison is held to 3e-3 plus 1e-4 of the largest."""
    nsteps, K = 30, 7
    d, rn0, u0, target = _drop_setup(24, 6.0, nsteps, g=1e-4, wall=wall)
    p = O.Params(**d)
    rn32 = rn0.astype(np.float32)
    u32 = u0.astype(np.float32)
    lat = cm.Lattice(d, rn32, u32)
    J, g, grn = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=K, want_rho_n0=True)
    assert lat.time == nsteps
    lat.close()
    grn = grn.double().cpu().numpy()
    # (a) same trajectory
    states = _gpu_trajectory(d, rn32, u32, nsteps)
    Ja = A.objective(*states[-1], target, p)
    lR, lB = A.objective_vjp(*states[-1], target, p)
    ga = {k: 0.0 for k in A.PARAM_NAMES}
    for t in range(nsteps - 1, -1, -1):
        lR, lB, gs = A.step_vjp(*states[t], lR, lB, p)
        for k in ga:
            ga[k] += gs[k]
    grn_a = A.init_vjp(rn32.astype(np.float64), u0[0], u0[1], lR, lB, p)
    assert abs(J - Ja) <= 1e-6 * Ja
    gmax = max(abs(v) for v in ga.values())
    for name_ in PN:
        assert abs(g[name_] - ga[name_]) <= 1e-4 * abs(ga[name_]) + 1e-5 * gmax, (name_, g[name_], ga[name_])
    assert np.abs(grn - grn_a).max() <= 1e-4 * np.abs(grn_a).max()
    # (b) the FP64 trajectory
    J_ref, g_ref, grn_ref = A.gradient_of_objective(rn32.astype(np.float64), u0[0], u0[1], target, p, nsteps, K)
    assert abs(J - J_ref) <= 1e-4 * J_ref
    for name_ in PN:
        assert abs(g[name_] - g_ref[name_]) <= 3e-3 * abs(g_ref[name_]) + 1e-4 * gmax, (name_, g[name_], g_ref[name_])
    assert np.abs(grn - grn_ref).max() <= 3e-3 * np.abs(grn_ref).max()


@pytest.mark.parametrize("wall", [False, True])
def test_fused_kernels_equal_plane_passes(wall):
    """The whole checkpointed adjoint through the two fused reverse kernels
    and through the eight plane passes they replace: the same objective and,
    up to the summation order of the partial sums, the same gradients."""
    nsteps = 12
    d, rn0, u0, target = _drop_setup(96, 20.0, nsteps, g=1e-4, wall=wall)
    outs = []
    for fused in (1, 2):
        lat = cm.Lattice(dict(d, adjoint_fused=fused), rn0.astype(np.float32), None)
        J, g, grn = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=5, want_rho_n0=True)
        outs.append((J, g, grn.double().cpu().numpy()))
        lat.close()
    (J1, g1, r1), (J2, g2, r2) = outs
    assert J1 == J2
    gmax = max(abs(v) for v in g2.values())
    for k in g2:
        assert abs(g1[k] - g2[k]) <= 1e-5 * abs(g2[k]) + 1e-7 * gmax, (k, g1[k], g2[k])
    assert np.abs(r1 - r2).max() <= 1e-5 * np.abs(r2).max()


@pytest.mark.parametrize("fused,wall", [(2, False), (1, False), (1, True), (0, False)],
                         ids=["planes", "fused", "fused_walls", "automatic"])
def test_checkpoint_interval_gives_identical_gradients(fused, wall):
    """Every checkpoint interval gives the same objective and gradients, bit
    for bit.  With the fused reverse step the forward fields of a state come
    from the forward step that read it (every state with K = 1, all but a
    segment's last with K > 1) or are recomputed by the reverse step (a
    segment's last state): the two sources must agree exactly."""
    nsteps = 12
    d, rn0, u0, target = _drop_setup(32, 8.0, nsteps, g=1e-4, wall=wall)
    d["adjoint_fused"] = fused
    outs = []
    launches = {}
    for K in (1, 5, 12, 200):
        lat = cm.Lattice(d, rn0.astype(np.float32), None)
        J, g, grn = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=K, want_rho_n0=True)
        outs.append((J, g, grn.cpu().numpy()))
        launches[K] = lat.launches
        lat.close()
    for J, g, grn in outs[1:]:
        assert J == outs[0][0]
        assert g == outs[0][1]
        assert np.array_equal(grn, outs[0][2])
    # one segment of 12 replays 11 steps.  Fused, every forward step writes the
    # forward fields its reverse step reads -- with every state kept all 12,
    # in the segment the 11 replayed ones -- so K = 12 runs one forward-field
    # recomputation more; the plane passes recompute them in every reverse step
    # (automatic: the fused kernels, since the forward steps write the fields)
    assert launches[12] - launches[1] == (11 if fused == 2 else 12)


def test_recorded_segment_graphs_are_replayed_exactly():
    """A second adjoint sweep on the same context replays the CUDA graphs
    recorded by the first (same segment lengths and start buffers) and must
    give the same objective and gradients bit for bit."""
    nsteps = 12
    d, rn0, u0, target = _drop_setup(32, 8.0, nsteps, g=1e-4)
    lat = cm.Lattice(d, rn0.astype(np.float32), None)
    start = lat.populations().clone()
    J1, g1, _ = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=5)
    lat.set_populations(start)
    J2, g2, _ = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=5)
    lat.close()
    assert J2 == J1
    assert g2 == g1


def test_checkpoint_interval_invariance_walls_order6():
    """Walls and App. B's order-6 stencil inside the recorded segments (the
    order-6 replay step is four launches): every checkpoint interval gives
    the same gradients."""
    nsteps = 7
    d, rn0, u0, target = _drop_setup(24, 6.0, nsteps, g=1e-4, wall=True)
    d["stencil_order"] = 6
    outs = []
    for K in (1, 3, 7):
        lat = cm.Lattice(d, rn0.astype(np.float32), None)
        J, g, grn = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=K, want_rho_n0=True)
        outs.append((J, g, grn.cpu().numpy()))
        lat.close()
    for J, g, grn in outs[1:]:
        assert J == outs[0][0]
        assert g == outs[0][1]
        assert np.array_equal(grn, outs[0][2])


def test_adjoint_matches_finite_differences_64():
    """64^2 drop (radius 8), Lambda = 10, gravity 1e-5, 200 steps, checkpoints
    every 50: gradients with respect to sigma, beta, both shear rates, the
    body force and (one direction of) the initial colour field against
    fourth-order central differences of the FP64 forward oracle (steps
    chosen so that truncation and round-off stay below 1e-6 relative)."""
    nsteps, K = 200, 50
    d, rn0, u0, target = _drop_setup(64, 8.0, nsteps, g=1e-5)
    p = O.Params(**d)
    rn32 = rn0.astype(np.float32)
    lat = cm.Lattice(d, rn32, None)
    J, g, grn = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=K, want_rho_n0=True)
    lat.close()

    def J_of(q, rn):
        R, B = O.run(*O.init_state(rn, u0[0], u0[1], q), q, nsteps)
        return A.objective(R, B, target, q)

    import dataclasses
    h = {"sigma": 1e-5, "beta": 1e-4, "lambda3_r": 1e-4, "lambda3_b": 1e-4, "g_acc_x": 1e-6, "g_acc_y": 1e-6}

    def shifted(name, s):
        if name.startswith("g_acc"):
            gg = list(p.g_acc)
            gg[0 if name.endswith("x") else 1] += s
            return dataclasses.replace(p, g_acc=tuple(gg))
        return dataclasses.replace(p, **{name: getattr(p, name) + s})

    rn64 = rn32.astype(np.float64)
    for name_ in PN:
        H = h[name_]
        fd = (8 * (J_of(shifted(name_, H), rn64) - J_of(shifted(name_, -H), rn64))
              - (J_of(shifted(name_, 2 * H), rn64) - J_of(shifted(name_, -2 * H), rn64))) / (12 * H)
        assert abs(g[name_] - fd) <= 1e-4 * abs(fd), (name_, g[name_], fd)
    v = np.random.default_rng(2).standard_normal(rn0.shape) * (np.abs(rn64) < 0.99)
    H = 1e-5
    fd = (8 * (J_of(p, rn64 + H * v) - J_of(p, rn64 - H * v))
          - (J_of(p, rn64 + 2 * H * v) - J_of(p, rn64 - 2 * H * v))) / (12 * H)
    ad = float(np.sum(grn.double().cpu().numpy() * v))
    assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)


def test_autograd_function():
    nsteps = 20
    d, rn0, u0, target = _drop_setup(32, 8.0, nsteps, g=1e-4)
    theta = torch.tensor([d["sigma"], d["beta"], d["lambda3_r"], d["lambda3_b"], 0.0, -1e-4],
                         dtype=torch.float64, requires_grad=True)
    rn = torch.from_numpy(rn0.astype(np.float32)).cuda().requires_grad_(True)
    J = cm.colour_mismatch(theta, rn, d, torch.from_numpy(target.astype(np.float32)).cuda(), nsteps, 8)
    J.backward()
    lat = cm.Lattice(d, rn0.astype(np.float32), None)
    J2, g2, grn2 = lat.adjoint(nsteps, target.astype(np.float32), ckpt_every=8, want_rho_n0=True)
    lat.close()
    assert float(J) == J2
    assert theta.grad.tolist() == [g2[k] for k in PN]
    assert torch.equal(rn.grad, grn2)


def test_adjoint_rejects_bad_use():
    d, _, _ = I.static_drop(n=16, radius=4.0)
    lat = cm.Lattice(dict(d, precision=2), None, None)
    with pytest.raises(cm.CmrtError) as ei:
        lat.adjoint(2, np.zeros((16, 16), np.float32))
    assert ei.value.status == cm.CMRT_EINVAL
    lat.close()
    lat = cm.Lattice(d, None, None)
    lat.step(1)
    with pytest.raises(cm.CmrtError) as ei:
        lat.adjoint(2, np.zeros((16, 16), np.float32), want_rho_n0=True)
    assert ei.value.status == cm.CMRT_EINVAL
    J, g, _ = lat.adjoint(2, np.zeros((16, 16), np.float32))  # without rho^N_0 any time is fine
    assert lat.time == 3 and J > 0
    lat.close()
