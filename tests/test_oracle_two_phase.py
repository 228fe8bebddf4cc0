"""Pins of the oracle's two-phase (multi-density, multi-viscosity) flow, Sec. 3.2.1.

Readings: per-particle density rho_i and viscosity nu_i are inputs; the equation of state
gives p_i = rho_i alpha_i; the correction is u' = -(dt/rho_i) grad p (the multi-density
pressure term, since (rho_j/rho_i) alpha_j - alpha_i = (p_j - p_i)/rho_i); the PPE's 1/rho
becomes the pair factor 2/(rho_i + rho_j); the viscosity term uses the particle's own nu_i.

Each pin is fixed by something other than the oracle's own formula: a closed form on a
scaled lattice, exact invariance of the motion under a common scaling of every density,
bitwise symmetry, the exactness of the Laplacian on a quadratic field, and hydrostatic
balance in a still two-layer tank."""
import numpy as np
import pytest

import oracle
import scenes
from test_oracle_pins import _closed_form, interior_mask, lattice_block


def test_uniform_properties_reduce_to_single_phase():
    sc = scenes.dam_break_2d(seed=1)
    for mode in (0, 1):
        a = oracle.State.from_scene(sc)
        b = oracle.State.from_scene(sc)
        oracle.step(oracle.params_for(sc, pressure_mode=mode), a)
        oracle.step(oracle.params_for(sc, pressure_mode=mode, rho_i=np.full(sc.n, 1000.0),
                                      nu_i=np.full(sc.n, 1e-6)), b)
        assert np.abs(b.p - a.p).max() <= 1e-13 * np.abs(a.p).max()
        assert np.abs(b.vel - a.vel).max() <= 1e-13 * np.abs(a.vel).max()
        assert np.array_equal(a.flags, b.flags)


@pytest.mark.parametrize("mode", [0, 1])
def test_motion_invariant_under_common_density_scaling(mode):
    """Multiplying every density by 2 doubles the pressure and leaves the motion unchanged:
    Eq. 16 scales p with rho_i; the PPE's pair factor halves the Laplacian, so with
    alpha_c = 0 its solution doubles; the correction divides by rho_i."""
    sc = scenes.dam_break_2d(seed=2)
    rho, nu = scenes.two_phase(sc)
    kw = dict(pressure_mode=mode, alpha_c=0.0, cg_tol=1e-13, nu_i=nu, clamp_negative_p=0)
    a = oracle.State.from_scene(sc)
    b = oracle.State.from_scene(sc)
    for _ in range(2):
        oracle.step(oracle.params_for(sc, rho_i=rho, **kw), a)
        oracle.step(oracle.params_for(sc, rho_i=2.0 * rho, **kw), b)
    assert np.abs(b.p - 2.0 * a.p).max() <= 1e-10 * np.abs(a.p).max()
    assert np.abs(b.vel - a.vel).max() <= 1e-10 * np.abs(a.vel).max()
    assert np.abs(b.pos - a.pos).max() <= 1e-15
    assert np.abs(a.p).max() > 0


def test_wc_pressure_per_phase_on_scaled_lattice():
    """Compressed lattice, two densities: p_i = rho_i c0^2/gamma ((n*/n0)^gamma - 1) with n*
    from the shell sums (closed form), on each phase."""
    l0, s = 0.01, 0.995
    pos, t = lattice_block(3, 13, spacing=s * l0)
    sc = scenes.Scene(3, l0, pos + 0.05, np.zeros_like(pos), t, np.full(3, 0.0), np.full(3, 0.3))
    rho = np.where(pos[:, 0] < pos[:, 0].mean(), 1000.0, 800.0)
    prm = oracle.params_for(sc, pressure_mode=1, c0=20.0, g=(0.0, 0.0, 0.0), nu=0.0, rho_i=rho)
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st, solve_only=True)
    n0_ref, _ = _closed_form(3, 2.1)
    n_scaled, _ = _closed_form(3, 2.1 / s)
    alpha = 20.0 ** 2 / 7.0 * ((n_scaled / n0_ref) ** 7 - 1.0)
    inner = interior_mask(pos, 2.1 * l0 + 0.5 * l0)
    for r in (1000.0, 800.0):
        sel = inner & (rho == r)
        assert sel.sum() > 0
        np.testing.assert_allclose(st.p[sel], r * alpha, rtol=1e-11)


def test_viscosity_per_particle_on_quadratic_velocity():
    """u_x = y^2: lap(u_x) = 2 exactly at interior lattice particles (Eq. 7), so
    u*_x = y^2 + 2 nu_i dt with each particle's own viscosity."""
    l0 = 0.01
    pos, t = lattice_block(2, 25, spacing=l0)
    pos = pos + 0.1
    vel = np.zeros_like(pos)
    vel[:, 0] = pos[:, 1] ** 2
    sc = scenes.Scene(2, l0, pos, vel, t, np.zeros(3), np.array([0.5, 0.5, 0.0]))
    nu = np.where(pos[:, 0] < pos[:, 0].mean(), 1e-2, 3e-2)
    dt = 1e-4
    prm = oracle.params_for(sc, pressure_mode=1, c0=0.0, nu_i=nu, dt=dt, g=(0.0, 0.0, 0.0))
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    inner = interior_mask(pos, 0.045)
    np.testing.assert_allclose(st.vel[inner, 0], pos[inner, 1] ** 2 + 2 * nu[inner] * dt,
                               rtol=1e-12)


def test_two_phase_ppe_matrix_symmetric_definite():
    sc = scenes.dam_break_2d(seed=1)
    rho, nu = scenes.two_phase(sc)
    prm = oracle.params_for(sc, rho_i=rho, nu_i=nu)
    off, col, val, b, ps, ns, fl = oracle.ppe_system(prm, sc)
    A = np.zeros((sc.n, sc.n))
    for i in range(sc.n):
        A[i, col[off[i]:off[i + 1]]] += val[off[i]:off[i + 1]]
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)
    # a pair across the interface weighs between the two single-phase pairs
    one = oracle.ppe_system(oracle.params_for(sc, rho_i=np.full(sc.n, 1000.0)), sc)
    A1 = np.zeros_like(A)
    for i in range(sc.n):
        A1[i, one[1][one[0][i]:one[0][i + 1]]] += one[2][one[0][i]:one[0][i + 1]]
    heavy = rho == 1000.0
    cross = np.outer(heavy, ~heavy) & (A1 != 0)
    ratio = A[cross] / A1[cross]
    assert cross.sum() > 0
    np.testing.assert_allclose(ratio, 2000.0 / 1800.0, rtol=1e-14)


@pytest.mark.slow
def test_two_layer_hydrostatic_balance():
    """Still tank, 10 lattice layers of light fluid (800) over 10 of heavy fluid (1000): the
    time-averaged pressure at the bottom row carries the weight of both layers above it, and
    inside each layer the pressure grows with depth at about that layer's rho g (the
    interface and the free surface smear the profile over a few layers, as in one phase)."""
    sc = scenes.still_tank_2d(width=0.2, depth=0.2)
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 800.0), nu=(1e-6, 1e-6))
    prm = oracle.params_for(sc, rho_i=rho, nu_i=nu)
    st = oracle.State.from_scene(sc)
    acc = np.zeros(sc.n)
    cnt = 0
    for k in range(2000):
        oracle.step(prm, st)
        if k >= 500:
            acc += st.p
            cnt += 1
    f = sc.types == oracle.FLUID
    y = sc.pos[:, 1]
    pm = acc / cnt
    g = 9.81
    bottom = f & (y < 0.01)
    weight = 800.0 * g * 0.1 + 1000.0 * g * (0.1 - 0.005)
    assert abs(pm[bottom].mean() / weight - 1.0) < 0.05
    slopes = {}
    for r, sel in ((800.0, f & (y > 0.115) & (y < 0.185)), (1000.0, f & (y > 0.015) & (y < 0.085))):
        slopes[r] = np.polyfit(0.2 - y[sel], pm[sel], 1)[0]
        assert abs(slopes[r] / (r * g) - 1.0) < 0.15, (r, slopes[r])
    assert slopes[800.0] < slopes[1000.0]
