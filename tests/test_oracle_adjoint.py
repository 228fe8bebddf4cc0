"""Pins of the oracle's reverse step (``orc_step_vjp``): the vector-Jacobian product of
one step against central finite differences of the oracle's own forward step, which the
other pin suites fix independently.  For random cotangents gbar and directions v,
<gbar, (F(x + h v) - F(x - h v)) / 2h> must equal <VJP(gbar), v>.

Scenes are small tanks whose fluid AND wall / dummy particles are jittered: on an exact
lattice some wall pairs sit exactly at r = re, where the step is not differentiable (a
neighbour enters with w = 0 but w' != 0), and a central difference there averages the two
one-sided derivatives.  With jitter every pair is away from the cut-offs by far more than
h, so neighbour sets, flags, the clamp set and the p_hat minimiser are the same at x +- h v
and the step is smooth between them.  Central differences then agree to ~1e-9 relative
(truncation O(h^2) plus rounding ~1e-16/h); the bound 1e-6 leaves room for the CG
tolerance of both solves (1e-14).

A viscosity of 0.5 m^2/s in the viscous case makes the Laplacian's share of the Jacobian
~1e-2 (at the water value 1e-6 it would be ~1e-8, below any finite-difference check)."""
import numpy as np
import pytest

import oracle
import scenes

TOL = 1e-6


def _scene(dim=2, seed=3):
    if dim == 2:
        sc = scenes.tank_scene(2, 0.01, (20, 14), (8, 10), jitter=0.05, wall_jitter=0.02,
                               seed=seed)
    else:
        sc = scenes.tank_scene(3, 0.01, (9, 6, 8), (4, 6, 5), jitter=0.05, wall_jitter=0.02,
                               seed=seed)
    f = sc.types == scenes.FLUID
    u = scenes.splitmix_uniform(seed + 17, np.arange(sc.pos.size, dtype=np.uint64))
    sc.vel[f] = 0.2 * (u.reshape(sc.pos.shape)[f] - 0.5)
    return sc


def _forward(prm, sc, pos, vel, g=None):
    if g is not None:
        prm = oracle.StepParams(**{**prm.__dict__, "g": tuple(g)})
    st = oracle.State(pos.copy(), vel.copy(), sc.types.copy(), np.zeros(sc.n), np.zeros(sc.n),
                      np.zeros(sc.n, np.uint8))
    oracle.step(prm, st)
    return st.pos, st.vel


def _check(sc, prm, which, h, seed=0, mask=None):
    rng = np.random.default_rng(seed)
    gpos = rng.standard_normal(sc.pos.shape)
    gvel = rng.standard_normal(sc.vel.shape)
    gr, gu, gg = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel)
    g0 = np.array(prm.g, dtype=np.float64)
    if which == "g":
        v = rng.standard_normal(3)
        if sc.dim == 2:
            v[2] = 0.0
        fp = _forward(prm, sc, sc.pos, sc.vel, g0 + h * v)
        fm = _forward(prm, sc, sc.pos, sc.vel, g0 - h * v)
        adj = float(gg @ v)
    else:
        v = rng.standard_normal(sc.pos.shape)
        if mask is not None:
            v = v * mask[:, None]
        if which == "pos":
            fp = _forward(prm, sc, sc.pos + h * v, sc.vel)
            fm = _forward(prm, sc, sc.pos - h * v, sc.vel)
            adj = float((gr * v).sum())
        else:
            fp = _forward(prm, sc, sc.pos, sc.vel + h * v)
            fm = _forward(prm, sc, sc.pos, sc.vel - h * v)
            adj = float((gu * v).sum())
    fd = float(((fp[0] - fm[0]) * gpos + (fp[1] - fm[1]) * gvel).sum()) / (2.0 * h)
    assert abs(fd - adj) <= TOL * abs(adj), (which, fd, adj, abs(fd - adj) / abs(adj))
    return adj


STEPS = {"pos": 1e-8, "vel": 1e-6, "g": 1e-3}
CASES = [
    ("ppe", dict(pressure_mode=0)),
    ("ppe-no-clamp", dict(pressure_mode=0, clamp_negative_p=0)),
    ("eos", dict(pressure_mode=1, c0=20.0)),
    ("viscous", dict(pressure_mode=1, c0=1e-6, nu=0.5)),
]


@pytest.mark.parametrize("which", ["pos", "vel", "g"])
@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_vjp_matches_central_differences_2d(name, kw, which):
    sc = _scene(2)
    prm = oracle.params_for(sc, cg_tol=1e-14, **kw)
    _check(sc, prm, which, STEPS[which])


@pytest.mark.parametrize("kind", [scenes.FLUID, scenes.WALL, scenes.DUMMY])
def test_vjp_position_blocks_per_kind(kind):
    """Directions confined to one particle kind: the wall and dummy positions enter only
    through pair terms (number density, PPE coefficients, gradient, viscosity)."""
    sc = _scene(2, seed=5)
    prm = oracle.params_for(sc, cg_tol=1e-14)
    _check(sc, prm, "pos", 1e-8, seed=2, mask=(sc.types == kind).astype(float))


@pytest.mark.parametrize("which", ["pos", "vel"])
@pytest.mark.parametrize("mode", [0, 1])
def test_vjp_matches_central_differences_3d(mode, which):
    sc = _scene(3, seed=4)
    prm = oracle.params_for(sc, cg_tol=1e-14, pressure_mode=mode, c0=20.0, nu=0.05)
    _check(sc, prm, which, STEPS[which], seed=1)


@pytest.mark.parametrize("which", ["pos", "vel"])
def test_vjp_two_phase(which):
    sc = _scene(2, seed=6)
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 600.0), nu=(0.05, 0.3))
    prm = oracle.params_for(sc, cg_tol=1e-14, rho_i=rho, nu_i=nu)
    _check(sc, prm, which, STEPS[which], seed=3)


def test_vjp_ghost_particles():
    """A particle that leaves the grid in this step is a GHOST from then on: its velocity is
    reset (gradient 0) and its position is carried over (gradient = the cotangent)."""
    sc = _scene(2, seed=7)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    sc.pos[f[0]] = [sc.box_max[0] + 0.05, 0.05]   # outside the grid: becomes a GHOST
    sc.types[f[1]] = scenes.GHOST                 # already a GHOST: carried unchanged
    prm = oracle.params_for(sc, cg_tol=1e-14)
    rng = np.random.default_rng(9)
    gpos = rng.standard_normal(sc.pos.shape)
    gvel = rng.standard_normal(sc.vel.shape)
    gr, gu, _ = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel)
    assert np.all(gu[f[0]] == 0.0)
    assert np.array_equal(gr[f[0]], gpos[f[0]])
    assert np.array_equal(gu[f[1]], gvel[f[1]]) and np.array_equal(gr[f[1]], gpos[f[1]])
    for which in ("pos", "vel"):
        _check(sc, prm, which, STEPS[which], seed=4)


def test_vjp_is_linear_in_the_cotangent():
    sc = _scene(2, seed=8)
    prm = oracle.params_for(sc, cg_tol=1e-14)
    rng = np.random.default_rng(1)
    a = [rng.standard_normal(sc.pos.shape) for _ in range(4)]
    st = oracle.State.from_scene(sc)
    r1 = oracle.step_vjp(prm, st, a[0], a[1])
    r2 = oracle.step_vjp(prm, st, a[2], a[3])
    r3 = oracle.step_vjp(prm, st, a[0] + 2.0 * a[2], a[1] + 2.0 * a[3])
    for x, y, z in zip(r1, r2, r3):
        assert np.allclose(z, x + 2.0 * y, rtol=1e-9, atol=1e-9 * np.abs(z).max())


def test_vjp_rejects_options_without_a_reverse():
    sc = _scene(2)
    st = oracle.State.from_scene(sc)
    z = np.zeros_like(sc.pos)
    for kw in (dict(kernel=1, pressure_mode=1), dict(grad_form=1), dict(source=1)):
        with pytest.raises(oracle.OracleError):
            oracle.step_vjp(oracle.params_for(sc, **kw), st, z, z)


# ------------------------------------------------------------------ the viscosity
def _forward_nu(prm, sc, nu=None, nu_i=None):
    kw = dict(prm.__dict__)
    if nu is not None:
        kw["nu"] = float(nu)
    if nu_i is not None:
        kw["nu_i"] = np.ascontiguousarray(nu_i, dtype=np.float64)
    return _forward(oracle.StepParams(**kw), sc, sc.pos, sc.vel)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_vjp_viscosity_matches_central_differences(dim, mode):
    """dL/dnu (Eq. 7's viscosity in the prediction, one value for all): the sum of the
    per-particle cotangents against (F(nu + h) - F(nu - h)) / 2h, PPE and EOS paths."""
    sc = _scene(dim, seed=10 + dim)
    nu = 0.05
    prm = oracle.params_for(sc, cg_tol=1e-14, pressure_mode=mode, c0=20.0, nu=nu)
    rng = np.random.default_rng(11)
    gpos = rng.standard_normal(sc.pos.shape)
    gvel = rng.standard_normal(sc.vel.shape)
    _, _, _, gnu = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel, with_nu=True)
    assert np.all(gnu[sc.types != scenes.FLUID] == 0.0)
    h = 1e-6 * nu
    fp = _forward_nu(prm, sc, nu=nu + h)
    fm = _forward_nu(prm, sc, nu=nu - h)
    fd = float(((fp[0] - fm[0]) * gpos + (fp[1] - fm[1]) * gvel).sum()) / (2.0 * h)
    adj = float(gnu.sum())
    assert abs(fd - adj) <= TOL * abs(adj), (fd, adj, abs(fd - adj) / abs(adj))


def test_vjp_per_particle_viscosity_matches_central_differences():
    """Two phases: dL/dnu_i along a random direction of the per-particle viscosities."""
    sc = _scene(2, seed=12)
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 600.0), nu=(0.05, 0.3))
    prm = oracle.params_for(sc, cg_tol=1e-14, rho_i=rho, nu_i=nu)
    rng = np.random.default_rng(13)
    gpos = rng.standard_normal(sc.pos.shape)
    gvel = rng.standard_normal(sc.vel.shape)
    _, _, _, gnu = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel, with_nu=True)
    v = rng.uniform(0.5, 1.5, size=sc.n) * 0.05   # one sign: no cancellation in the sum
    h = 1e-6
    fp = _forward_nu(prm, sc, nu_i=nu + h * v)
    fm = _forward_nu(prm, sc, nu_i=nu - h * v)
    fd = float(((fp[0] - fm[0]) * gpos + (fp[1] - fm[1]) * gvel).sum()) / (2.0 * h)
    adj = float(gnu @ v)
    assert abs(fd - adj) <= TOL * abs(adj), (fd, adj, abs(fd - adj) / abs(adj))


def test_vjp_viscosity_of_a_fluid_at_rest_is_zero():
    """With u = 0 the Laplacian of the velocity vanishes: dL/dnu = 0 exactly."""
    sc = _scene(2, seed=14)
    sc.vel[:] = 0.0
    prm = oracle.params_for(sc, cg_tol=1e-14, nu=0.05)
    rng = np.random.default_rng(15)
    g = rng.standard_normal(sc.pos.shape)
    _, _, _, gnu = oracle.step_vjp(prm, oracle.State.from_scene(sc), g, g, with_nu=True)
    assert np.all(gnu == 0.0)
