"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

None of these retypes the oracle's formulas: each compares it with a closed form
(lattice shell sums, exactness of the Laplacian on quadratics and of the gradient on linear
fields), an independent computation (numpy brute force, a dense Cholesky solve), an
invariant (symmetry, definiteness, hydrostatic balance) or a hand-derived special case.
"""
import math
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _shells():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lattice_shells.txt"))
            if l.strip() and not l.startswith("#")]
    out = {2: {}, 3: {}}
    for d, k, c in rows:
        out[int(d)][int(k)] = int(c)
    return out


def _closed_form(dim, re_l0, l0=1.0):
    sh = _shells()[dim]
    n0 = 0.0
    m2 = 0.0
    for k, c in sh.items():
        if k < re_l0 ** 2:
            w = re_l0 / math.sqrt(k) - 1.0
            n0 += c * w
            m2 += c * w * k * l0 * l0
    return n0, m2 / n0


# ---------------------------------------------------------------- Eq. 5 / Eq. 7 constants
def test_shell_table_totals():
    sh = _shells()
    assert sum(sh[2].values()) == 44 and sum(sh[3].values()) == 250


@pytest.mark.parametrize("dim,re", [(2, 2.1), (2, 4.0), (3, 2.1), (3, 4.0)])
def test_lattice_constants_match_shell_closed_form(dim, re):
    n0, lam = oracle.lattice(dim, 1.0, re)
    n0_c, lam_c = _closed_form(dim, re)
    assert n0 == pytest.approx(n0_c, rel=1e-14)
    assert lam == pytest.approx(lam_c, rel=1e-14)


def test_lattice_constants_match_golden_digits():
    for line in open(os.path.join(GOLDEN, "lattice_constants.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        d, re, n0, lam = line.split()
        got_n0, got_lam = oracle.lattice(int(d), 1.0, float(re))
        assert got_n0 == pytest.approx(float(n0), abs=2e-12)
        if lam != "nan":
            assert got_lam == pytest.approx(float(lam), abs=2e-12)


def test_lattice_constants_scale_with_l0():
    # n0 is dimensionless, lambda scales with l0^2 (re given in metres)
    n0a, la = oracle.lattice(3, 1.0, 4.0)
    n0b, lb = oracle.lattice(3, 0.0075, 0.03)
    assert n0b == pytest.approx(n0a, rel=1e-13)
    assert lb == pytest.approx(la * 0.0075 ** 2, rel=1e-13)


# ---------------------------------------------------------------- lattice helpers
def lattice_block(dim, m, l0=1.0, spacing=None):
    s = l0 if spacing is None else spacing
    g = np.meshgrid(*[np.arange(m)] * dim, indexing="ij")
    pos = np.stack([a.reshape(-1) for a in g], axis=1).astype(np.float64) * s
    return pos, np.zeros(len(pos), np.int8)


def interior_mask(pos, margin):
    lo, hi = pos.min(0), pos.max(0)
    return np.all((pos >= lo + margin) & (pos <= hi - margin), axis=1)


# ---------------------------------------------------------------- Eq. 5 on a lattice
@pytest.mark.parametrize("dim,re", [(2, 2.1), (2, 4.0), (3, 2.1), (3, 4.0)])
def test_pnd_of_interior_lattice_particle_is_n0(dim, re):
    pos, t = lattice_block(dim, 13 if dim == 3 else 21)
    nd = oracle.pnd(dim, pos, t, re)
    n0_c, _ = _closed_form(dim, re)
    inner = interior_mask(pos, re + 0.5)
    assert inner.sum() > 0
    np.testing.assert_allclose(nd[inner], n0_c, rtol=1e-13)
    assert np.all(nd[~inner] <= n0_c * (1 + 1e-13))


# ---------------------------------------------------------------- neighbour sets
def numpy_brute_sets(dim, pos, types, re):
    """Independent O(N^2) sets: same predicate ((dx*dx)+(dy*dy))+(dz*dz) < re*re."""
    n = len(pos)
    P = np.zeros((n, 3))
    P[:, :dim] = pos
    dx = P[None, :, 0] - P[:, None, 0]
    dy = P[None, :, 1] - P[:, None, 1]
    dz = P[None, :, 2] - P[:, None, 2]
    r2 = (dx * dx + dy * dy) + dz * dz
    ok = r2 < re * re
    np.fill_diagonal(ok, False)
    g = types == oracle.GHOST
    ok[g, :] = False
    ok[:, g] = False
    return [np.nonzero(ok[i])[0] for i in range(n)]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("clustered", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_neighbor_sets_brute_cells_numpy_agree(dim, clustered, seed):
    sc = scenes.random_cloud(600 if dim == 3 else 400, dim, seed, clustered=clustered)
    types = sc.types.copy()
    types[::37] = oracle.GHOST
    re = 0.11
    ref = numpy_brute_sets(dim, sc.pos, types, re)
    for mode in (0, 1):
        off, ids = oracle.neighbors(dim, sc.pos, types, re, mode=mode)
        for i in range(len(ref)):
            np.testing.assert_array_equal(ids[off[i]:off[i + 1]], ref[i])


def test_neighbor_sets_on_boundary_distance_are_excluded():
    # two particles exactly re apart are not neighbours (w = 0 at r >= re, Eq. 4)
    pos = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 0.49999999]])
    off, ids = oracle.neighbors(2, pos, np.zeros(3, np.int8), 0.5, mode=0)
    assert list(ids[off[0]:off[1]]) == [2]


# ---------------------------------------------------------------- cell keys (Morton)
def test_cell_keys_closed_form():
    prm = oracle.StepParams(dim=3, l0=1.0, re_n_l0=1.0, re_lap_l0=1.0, cell_skin=0.0,
                            box_min=(0.0, 0.0, 0.0), box_max=(7.5, 7.5, 7.5))
    # cell side h = 1; hand-interleaved Morton keys (x in bit 0, y bit 1, z bit 2)
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0],
                    [3.5, 5.0, 6.99], [7.5, 0.0, 0.0], [-1e-12, 0.0, 0.0], [8.0, 0.0, 0.0],
                    [0.9999999999, 0.0, 0.0]])
    key, cell = oracle.cell_keys(prm, pos, np.zeros(len(pos), np.int8))
    assert list(key[:5]) == [0, 1, 2, 4, 427]
    assert key[5] == 0b001001001          # cx = 7 -> x bits at positions 0, 3, 6
    assert key[6] == 0xFFFFFFFF and key[7] == 0xFFFFFFFF      # outside the grid
    assert key[8] == 0
    assert list(cell[4]) == [3, 5, 6]


def test_cell_keys_2d_interleave():
    prm = oracle.StepParams(dim=2, l0=1.0, re_n_l0=1.0, re_lap_l0=1.0, cell_skin=0.0,
                            box_min=(0.0, 0.0, 0.0), box_max=(15.0, 15.0, 0.0))
    pos = np.array([[5.5, 9.5], [15.0, 15.0]])
    key, _ = oracle.cell_keys(prm, pos, np.zeros(2, np.int8))
    # x=0101, y=1001 -> interleave y3x3 y2x2 y1x1 y0x0 = 10 01 00 11 = 0b10010011
    assert key[0] == 0b10010011
    assert key[1] == 0xFF


# ---------------------------------------------------------------- Eq. 7 on quadratics
def test_laplacian_exact_on_quadratic_2d():
    pos, t = lattice_block(2, 25, l0=0.01)
    re = 0.04
    n0, lam = oracle.lattice(2, 0.01, re)
    x, y = pos[:, 0], pos[:, 1]
    phi = x * x + 3 * x * y - 2 * y * y            # Laplacian = 2 - 4 = -2
    lap = oracle.laplacian(2, pos, t, re, n0, lam, phi)
    inner = interior_mask(pos, re + 0.005)
    np.testing.assert_allclose(lap[inner], -2.0, rtol=0, atol=1e-9)


def test_laplacian_exact_on_quadratic_3d():
    pos, t = lattice_block(3, 13, l0=0.01)
    re = 0.04
    n0, lam = oracle.lattice(3, 0.01, re)
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    phi = np.stack([x * x + 2 * y * y - 3 * z * z + x * y + y * z,   # Laplacian 0
                    x * x,                                          # Laplacian 2
                    5 * z * z - x * z], axis=1)                     # Laplacian 10
    lap = oracle.laplacian(3, pos, t, re, n0, lam, phi)
    inner = interior_mask(pos, re + 0.005)
    np.testing.assert_allclose(lap[inner, 0], 0.0, atol=1e-9)
    np.testing.assert_allclose(lap[inner, 1], 2.0, atol=1e-9)
    np.testing.assert_allclose(lap[inner, 2], 10.0, atol=1e-9)


# ---------------------------------------------------------------- gradient on linear p
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("use_min", [False, True])
def test_gradient_exact_on_linear(dim, use_min):
    pos, t = lattice_block(dim, 21 if dim == 2 else 11, l0=0.01)
    re = 0.021
    n0, _ = oracle.lattice(dim, 0.01, re)
    a = np.array([3.0, -2.0, 0.5])[:dim]
    p = 100.0 + pos @ a
    if use_min:
        # a stabilising shift p_hat_i != p_i leaves the gradient of a lattice particle exact
        phat = p - 7.0
    else:
        phat = p.copy()
    gr = oracle.gradient(dim, pos, t, re, n0, p, phat)
    inner = interior_mask(pos, re + 0.005)
    np.testing.assert_allclose(gr[inner], np.broadcast_to(a, gr[inner].shape), rtol=1e-9)


def test_gradient_excludes_dummy_neighbours():
    pos, t = lattice_block(2, 11, l0=0.01)
    t = t.copy()
    t[pos[:, 0] > 0.055] = oracle.DUMMY
    p = np.full(len(pos), 5.0)
    p[t == oracle.DUMMY] = 1e6                        # dummies carry no pressure force
    gr = oracle.gradient(2, pos, t, 0.021, 1.0, p, np.full(len(pos), 5.0))
    assert np.all(gr[t != oracle.DUMMY] == 0.0)


# ---------------------------------------------------------------- PPE system
@pytest.fixture(scope="module")
def dam2d_system():
    sc = scenes.dam_break_2d(seed=1)
    prm = oracle.params_for(sc)
    return sc, prm, oracle.ppe_system(prm, sc)


def _dense(off, col, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[off[i]:off[i + 1]]] += val[off[i]:off[i + 1]]
    return A


def test_ppe_matrix_bitwise_symmetric(dam2d_system):
    sc, prm, (off, col, val, b, ps, ns, fl) = dam2d_system
    A = _dense(off, col, val, sc.n)
    assert np.array_equal(A, A.T)


def test_ppe_matrix_definite_and_dominant(dam2d_system):
    sc, prm, (off, col, val, b, ps, ns, fl) = dam2d_system
    A = _dense(off, col, val, sc.n)
    np.linalg.cholesky(A)                      # SPD
    diag = np.diag(A)
    off_sum = np.abs(A).sum(1) - np.abs(diag)
    rows = (sc.types <= oracle.WALL) & (fl == 0)
    assert np.all(diag[rows] - off_sum[rows] >= prm.alpha_c / prm.dt ** 2 * (1 - 1e-12))
    assert np.all(A[~rows][:, ~rows] == np.eye((~rows).sum()))
    assert np.all(b[~rows] == 0.0)


def test_ppe_rows_are_fluid_or_wall_off_surface(dam2d_system):
    sc, prm, (off, col, val, b, ps, ns, fl) = dam2d_system
    n0, _ = oracle.lattice(2, prm.l0, prm.re_n)
    assert np.all(fl[sc.types >= oracle.DUMMY] == 0)
    surf = (sc.types <= oracle.WALL) & (ns < prm.beta * n0)
    assert np.array_equal(fl == 1, surf)
    # the column's top row and its right face are on the free surface; the bottom-left
    # corner is not
    f = sc.types == oracle.FLUID
    top = f & (sc.pos[:, 1] > 0.395)
    assert np.all(fl[top] == 1)
    corner = f & (sc.pos[:, 0] < 0.05) & (sc.pos[:, 1] < 0.05)
    assert np.all(fl[corner] == 0)


def test_cg_matches_dense_solve(dam2d_system):
    sc, prm, (off, col, val, b, ps, ns, fl) = dam2d_system
    A = _dense(off, col, val, sc.n)
    x_dense = oracle.dense_spd_solve(A, b)
    x_cg, it, res = oracle.cg(off, col, val, b, tol=1e-13)
    assert res <= 1e-13
    scale = np.abs(x_dense).max()
    assert np.abs(x_cg - x_dense).max() <= 1e-10 * scale
    x8, it8, res8 = oracle.cg(off, col, val, b, tol=1e-8)
    true = np.linalg.norm(b - A @ x8) / np.linalg.norm(b)
    assert true <= 1e-8 and it8 < it


def test_dense_solver_against_numpy():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((40, 40))
    A = M @ M.T + 40 * np.eye(40)
    b = rng.standard_normal(40)
    np.testing.assert_allclose(oracle.dense_spd_solve(A, b), np.linalg.solve(A, b), rtol=1e-10)
    with pytest.raises(oracle.OracleError):
        oracle.dense_spd_solve(-A, b)


# ---------------------------------------------------------------- Eq. 16 (equation of state)
def test_wc_pressure_on_uniformly_scaled_lattice():
    """A lattice compressed to spacing s*l0 has n* = n0(re/(s l0)) everywhere inside:
    Eq. 16 then gives a closed-form pressure from the shell sums."""
    l0, s = 0.01, 0.995
    pos, t = lattice_block(3, 13, spacing=s * l0)
    sc = scenes.Scene(3, l0, pos + 0.05, np.zeros_like(pos), t, np.full(3, 0.0), np.full(3, 0.3))
    prm = oracle.params_for(sc, pressure_mode=1, c0=20.0, g=(0.0, 0.0, 0.0), nu=0.0)
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st, solve_only=True)
    n0_ref, _ = _closed_form(3, 2.1)
    n_scaled, _ = _closed_form(3, 2.1 / s)          # re/(s l0) in units of s*l0
    p_ref = 1000 * 20.0 ** 2 / 7.0 * ((n_scaled / n0_ref) ** 7 - 1.0)
    inner = interior_mask(pos, 2.1 * l0 + 0.5 * l0)
    np.testing.assert_allclose(st.nstar[inner], n_scaled, rtol=1e-13)
    np.testing.assert_allclose(st.p[inner], p_ref, rtol=1e-11)
    assert p_ref > 0


def test_wc_pressure_zero_at_reference_density():
    pos, t = lattice_block(2, 21, spacing=0.01)
    sc = scenes.Scene(2, 0.01, pos + 0.05, np.zeros_like(pos), t, np.zeros(3), np.array([0.4, 0.4, 0]))
    prm = oracle.params_for(sc, pressure_mode=1, g=(0.0, 0.0, 0.0))
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    inner = interior_mask(pos, 0.03)
    # p = rho c0^2/gamma ((n*/n0)^gamma - 1) with n* = n0 (1 + e), |e| ~ 1e-14 from
    # rounding: |p| <= rho c0^2 |e|
    assert np.abs(st.p[inner]).max() < 1e-12 * prm.rho * prm.c0 ** 2
    surf = st.flags == 1
    assert np.all(st.p[surf] == 0.0) and surf.sum() > 0


# ---------------------------------------------------------------- predict (Eq. 2, 7)
def test_lone_particle_free_fall():
    sc = scenes.Scene(2, 0.01, np.array([[0.3, 0.3]]), np.array([[0.2, -0.1]]),
                      np.zeros(1, np.int8), np.zeros(3), np.array([1.0, 1.0, 0.0]))
    prm = oracle.params_for(sc, dt=1e-3)
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    u1 = np.array([0.2, -0.1 - 9.81e-3])
    np.testing.assert_allclose(st.vel[0], u1, rtol=1e-15)
    np.testing.assert_allclose(st.pos[0], [0.3 + 1e-3 * 0.2, 0.3 + 1e-3 * u1[1]], rtol=1e-15)
    assert st.flags[0] == 1 and st.p[0] == 0.0 and st.nstar[0] == 0.0


def test_viscosity_term_on_quadratic_velocity():
    """u_x = y^2 on a lattice: nu lap(u_x) = 2 nu, so u*_x = y^2 + 2 nu dt (Eq. 2, 7).
    With the equation of state at c0 = 0 the pressure vanishes and u^{k+1} = u*."""
    l0 = 0.01
    pos, t = lattice_block(2, 25, spacing=l0)
    pos = pos + 0.1
    vel = np.zeros_like(pos)
    vel[:, 0] = pos[:, 1] ** 2
    sc = scenes.Scene(2, l0, pos, vel, t, np.zeros(3), np.array([0.5, 0.5, 0.0]))
    nu, dt = 1e-2, 1e-4
    prm = oracle.params_for(sc, pressure_mode=1, c0=0.0, nu=nu, dt=dt, g=(0.0, 0.0, 0.0))
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    inner = interior_mask(pos, 0.045)
    np.testing.assert_allclose(st.vel[inner, 0], pos[inner, 1] ** 2 + 2 * nu * dt, rtol=1e-12)
    np.testing.assert_allclose(st.vel[inner, 1], 0.0, atol=1e-15)
    np.testing.assert_allclose(st.pos[inner, 0], pos[inner, 0] + dt * st.vel[inner, 0], rtol=1e-14)


def test_walls_and_dummies_do_not_move():
    sc = scenes.dam_break_2d(seed=2)
    prm = oracle.params_for(sc)
    st = oracle.State.from_scene(sc)
    for _ in range(3):
        oracle.step(prm, st)
    b = sc.types != oracle.FLUID
    assert np.array_equal(st.pos[b], sc.pos[b]) and np.all(st.vel[b] == 0.0)


def test_step_p_hat_is_minimum_over_non_dummy_neighbours():
    """The stabilising p_hat_i of the gradient (Eq. 14 with p_hat) is the minimum of p over i
    and its neighbours within re, dummies left out.  A block compressed to 0.98 l0 on a
    wall row with two dummy rows below, no gravity, viscosity or initial velocity: u* = 0,
    r* = r, and after the step u = -(dt/rho) grad p with p_hat taken here by brute force.
    The bottom fluid row has dummies (p = 0) at 1.96 l0 < re, so p_hat with the dummies in
    would differ (checked below)."""
    l0 = 0.01
    s = 0.98 * l0
    rows = []
    for k, kind in [(-2, oracle.DUMMY), (-1, oracle.DUMMY), (0, oracle.WALL)]:
        rows += [(x, k * s, kind) for x in np.arange(-4, 20) * s]
    for j in range(1, 9):
        rows += [(x, j * s, oracle.FLUID) for x in np.arange(16) * s]
    a = np.array(rows)
    pos, t = a[:, :2] + 0.1, a[:, 2].astype(np.int8)
    sc = scenes.Scene(2, l0, pos, np.zeros_like(pos), t, np.zeros(3), np.array([0.5, 0.5, 0.0]))
    prm = oracle.params_for(sc, g=(0.0, 0.0, 0.0), nu=0.0)
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    re = prm.re_n
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    nbr = (d2 < re * re) & ~np.eye(len(pos), dtype=bool)

    def p_hat(mask):
        return np.array([min(st.p[i], st.p[nbr[i] & mask].min(initial=np.inf))
                         for i in range(len(pos))])

    ph = p_hat(t != oracle.DUMMY)
    ph_with_dummies = p_hat(np.ones(len(pos), bool))
    f = t == oracle.FLUID
    assert np.count_nonzero(f & (ph != ph_with_dummies)) >= 8
    n0, _ = oracle.lattice(2, l0, re)
    u = -(prm.dt / prm.rho) * oracle.gradient(2, pos, t, re, n0, st.p, ph)
    u_with_dummies = -(prm.dt / prm.rho) * oracle.gradient(2, pos, t, re, n0, st.p,
                                                             ph_with_dummies)
    np.testing.assert_allclose(st.vel[f], u[f], rtol=1e-12, atol=1e-12 * np.abs(u[f]).max())
    assert np.abs(u_with_dummies[f] - u[f]).max() > 1e-3 * np.abs(u[f]).max()


# ---------------------------------------------------------------- error statuses
def test_error_statuses():
    sc = scenes.dam_break_2d(seed=1)
    prm = oracle.params_for(sc)
    st = oracle.State.from_scene(sc)
    st.pos[3, 0] = np.nan
    rc, _ = oracle.step(prm, st, check=False)
    assert rc == -4
    st = oracle.State.from_scene(sc)
    st.pos[5] = st.pos[6]
    rc, _ = oracle.step(prm, st, check=False)
    assert rc == -6
    st = oracle.State.from_scene(sc)
    rc, _ = oracle.step(oracle.params_for(sc, cg_max_iter=1), st, check=False)
    assert rc == -3
    st = oracle.State.from_scene(sc)
    rc, _ = oracle.step(oracle.params_for(sc, cell_skin=0.0), st, check=False)
    assert rc == -5
    st = oracle.State.from_scene(sc)
    st.pos[7] = [5.0, 5.0]
    rc, rep = oracle.step(prm, st, check=False)
    assert rc == 0 and st.types[7] == oracle.GHOST and rep["n_ghost"] == 1


# ---------------------------------------------------------------- hydrostatics
@pytest.mark.slow
def test_hydrostatic_pressure_slope_still_tank():
    """Fluid at rest in a tank: the time-averaged pressure grows with depth at rho g."""
    sc = scenes.still_tank_2d(width=0.2, depth=0.2)
    prm = oracle.params_for(sc)
    st = oracle.State.from_scene(sc)
    acc = np.zeros(sc.n)
    cnt = 0
    for k in range(2000):
        oracle.step(prm, st)
        if k >= 500:
            acc += st.p
            cnt += 1
    f = sc.types == oracle.FLUID
    depth = 0.2 - sc.pos[f, 1]
    slope = np.polyfit(depth, acc[f] / cnt, 1)[0]
    assert abs(slope / (prm.rho * 9.81) - 1.0) < 0.10
    assert np.all(st.types != oracle.GHOST)


def test_dam_break_100_steps_sane():
    sc = scenes.dam_break_2d(seed=3)
    prm = oracle.params_for(sc)
    st = oracle.State.from_scene(sc)
    n0, _ = oracle.lattice(2, prm.l0, prm.re_n)
    for _ in range(100):
        rc, rep = oracle.step(prm, st)
        assert rep["cg_resid"] <= prm.cg_tol
    assert np.all(np.isfinite(st.pos)) and np.all(np.isfinite(st.p))
    assert st.nstar[st.types == oracle.FLUID].max() < 1.2 * n0
    assert np.count_nonzero(st.types == oracle.GHOST) == 0
    assert np.count_nonzero(st.types == oracle.FLUID) == 800


# ---------------------------------------------------------------- the assembled operator
@pytest.mark.parametrize("dim", [2, 3])
def test_ppe_operator_is_minus_laplacian_over_rho_on_quadratics(dim):
    """On a lattice at rest, rows of the PPE whose whole neighbourhood is in the PPE apply
    A = -(1/rho) L + alpha_c/dt^2 I: for p = |r|^2 (Laplacian 2d, exact by Eq. 7's
    construction) (A p)_i - alpha_c/dt^2 p_i = -2d/rho.  Pins the sign and scale of the
    off-diagonal coefficients and the diagonal sum of the assembly."""
    m = 21
    pos, t = lattice_block(dim, m, spacing=0.01)
    pos = pos + 0.05
    sc = scenes.Scene(dim, 0.01, pos, np.zeros_like(pos), t, np.zeros(3),
                      np.full(3, 0.05 + m * 0.01 + 0.1) if dim == 3 else
                      np.array([0.05 + m * 0.01 + 0.1] * 2 + [0.0]))
    g0 = (0.0, 0.0, 0.0)
    prm = oracle.params_for(sc, g=g0, nu=0.0)
    off, col, val, b, ps, ns, fl = oracle.ppe_system(prm, sc)
    p = ((pos - pos.mean(0)) ** 2).sum(1)
    y = np.array([val[off[i]:off[i + 1]] @ p[col[off[i]:off[i + 1]]] for i in range(len(p))])
    inner = interior_mask(pos, 0.04 + 0.045)   # re_lap plus the surface band
    assert inner.sum() > 0 and np.all(fl[inner] == 0)
    diag_add = prm.alpha_c / prm.dt ** 2
    np.testing.assert_allclose(y[inner] - diag_add * p[inner], -2.0 * dim / prm.rho, rtol=1e-8)


def test_particles_beyond_the_skin_keep_exact_sets_up_to_the_limit():
    """The neighbour sets at r* are searched at r*: a few particles moving farther than half
    the cell skin in one step change nothing (the step equals the one with a skin so large
    that nobody outruns it, bit for bit); more than max(64, n/256) such particles is
    MPS_ESKIN, the limit of the library's direct search."""
    sc = scenes.dam_break_2d(seed=4)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    kicked = sc.copy()
    kicked.vel[f[[5, 300, 700]]] = [[40.0, 0.0], [0.0, 35.0], [-30.0, 20.0]]   # 3-4 mm/step
    out = []
    for skin in (0.1, 2.0):
        st = oracle.State.from_scene(kicked)
        rc, rep = oracle.step(oracle.params_for(kicked, cell_skin=skin), st, check=False)
        assert rc == 0 and rep["max_disp"] > 0.5 * 0.1 * 4.0 * sc.l0
        out.append(st)
    for k in ("pos", "vel", "p", "nstar", "flags"):
        assert np.array_equal(getattr(out[0], k), getattr(out[1], k)), k
    many = sc.copy()
    many.vel[f[:65]] = [30.0, 0.0]
    rc, _ = oracle.step(oracle.params_for(many, cell_skin=0.1), oracle.State.from_scene(many),
                        check=False)
    assert rc == -5
    many.vel[f[64]] = [0.0, 0.0]
    rc, _ = oracle.step(oracle.params_for(many, cell_skin=0.1), oracle.State.from_scene(many),
                        check=False)
    assert rc == 0
