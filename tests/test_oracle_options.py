"""Pins of the oracle's numerical options (Sec. 3.1 and 3.3 of the paper):

- kernel 1, the cubic weight (1 - r/re)^3 the paper recommends with the equation of state:
  n0 and lambda from the lattice shell table, Laplacian exact on quadratic fields and
  gradient exact on linear fields at interior lattice particles (both hold for any radial
  weight on a cubic lattice, with n0 and lambda of that weight);
- gradient form 1, CMPS (Eq. 18): its pair term is symmetric in i, j, so the gradients of
  a free cluster sum to zero (linear momentum is conserved), unlike the difference form;
- PPE source 1, HS (Eq. 21): the source is (Dn/Dt)*/(n0 dt); it vanishes for a fluid at
  rest, equals the shell-sum closed form for a uniform dilation, and matches a central
  finite difference of Eq. 5 along the predicted velocity field;
- PPE source 2, HS with the error-compensating source (Eq. 24-25): closed form on a
  compressed, dilating lattice, whose number density and its rate at r^k are shell sums."""
import math

import numpy as np
import pytest

import oracle
import scenes
from test_oracle_pins import _shells, interior_mask, lattice_block


def _cubic_closed_form(dim, re_l0):
    n0 = m2 = 0.0
    for k, c in _shells()[dim].items():
        if k < re_l0 ** 2:
            w = (1.0 - math.sqrt(k) / re_l0) ** 3
            n0 += c * w
            m2 += c * w * k
    return n0, m2 / n0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("re", [2.1, 4.0])
def test_cubic_lattice_constants_from_shells(dim, re):
    n0, lam = oracle.lattice(dim, 0.01, re * 0.01, kernel=1)
    n0_ref, lam_ref = _cubic_closed_form(dim, re)
    assert n0 == pytest.approx(n0_ref, rel=1e-13)
    assert lam == pytest.approx(lam_ref * 1e-4, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_cubic_pnd_of_interior_particle_is_n0(dim):
    m = 15 if dim == 2 else 11
    pos, t = lattice_block(dim, m, spacing=0.01)
    nd = oracle.pnd(dim, pos, t, 0.021, kernel=1)
    inner = interior_mask(pos, 0.03)
    n0, _ = _cubic_closed_form(dim, 2.1)
    np.testing.assert_allclose(nd[inner], n0, rtol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_cubic_laplacian_exact_on_quadratic(dim):
    m = 17 if dim == 2 else 13
    pos, t = lattice_block(dim, m, spacing=0.01)
    x = pos[:, 0]
    y = pos[:, 1]
    phi = x ** 2 + 3 * x * y - 2 * y ** 2 + (0.5 * pos[:, 2] ** 2 if dim == 3 else 0.0)
    expect = 2.0 - 4.0 + (1.0 if dim == 3 else 0.0)
    n0, lam = oracle.lattice(dim, 0.01, 0.04, kernel=1)
    lap = oracle.laplacian(dim, pos, t, 0.04, n0, lam, phi, kernel=1)
    inner = interior_mask(pos, 0.045)
    np.testing.assert_allclose(lap[inner], expect, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_cubic_gradient_exact_on_linear(dim):
    m = 15 if dim == 2 else 11
    pos, t = lattice_block(dim, m, spacing=0.01)
    gvec = np.array([3.0, -2.0, 0.5])[:dim]
    p = pos @ gvec
    n0, _ = oracle.lattice(dim, 0.01, 0.021, kernel=1)
    g = oracle.gradient(dim, pos, t, 0.021, n0, p, p, kernel=1)
    inner = interior_mask(pos, 0.03)
    np.testing.assert_allclose(g[inner], np.broadcast_to(gvec, g[inner].shape), rtol=1e-12)


def _free_cluster(seed=3):
    """A jittered all-fluid block with no walls: every pair of neighbours is inside it."""
    pos, t = lattice_block(2, 21, spacing=0.01)
    u = scenes.splitmix_uniform(seed, np.arange(pos.size, dtype=np.uint64)).reshape(pos.shape)
    return pos + (u - 0.5) * 2e-3, t


@pytest.mark.parametrize("kernel", [0, 1])
def test_cmps_gradient_conserves_momentum(kernel):
    pos, t = _free_cluster()
    rng = np.random.default_rng(1)
    p = 1000.0 + 50.0 * rng.standard_normal(len(t))
    off, ids = oracle.neighbors(2, pos, t, 0.021)
    phat = np.array([min(p[i], p[ids[off[i]:off[i + 1]]].min()) for i in range(len(t))])
    n0, _ = oracle.lattice(2, 0.01, 0.021, kernel=kernel)
    g1 = oracle.gradient(2, pos, t, 0.021, n0, p, phat, kernel=kernel, form=1)
    g0 = oracle.gradient(2, pos, t, 0.021, n0, p, phat, kernel=kernel, form=0)
    scale = np.abs(g1).sum(0)
    assert np.all(np.abs(g1.sum(0)) <= 1e-12 * scale)      # pair forces cancel
    assert np.all(np.abs(g0.sum(0)) > 1e-6 * np.abs(g0).sum(0))   # the difference form does not


def _hs_system(sc, vel, **kw):
    prm = oracle.params_for(sc, source=1, nu=0.0, g=(0.0, 0.0, 0.0), **kw)
    st = oracle.State.from_scene(sc)
    st.vel = vel
    off, col, val, b, ps, ns, fl = oracle.ppe_system(prm, st)
    return prm, b, ps, fl


def test_hs_source_zero_at_rest():
    sc = scenes.dam_break_2d(seed=1)
    prm, b, ps, fl = _hs_system(sc, np.zeros_like(sc.vel))
    assert np.all(b == 0.0)


def test_hs_source_uniform_dilation_closed_form():
    """u = a (r - c): r* is the lattice scaled by s = 1 + a dt about c, r_ij . u_ij =
    a |r*_ij|^2 / s, so (Dn/Dt)* = -(a/s) re sum 1/|r*_ij| over the shells inside re."""
    l0, a, dt = 0.01, -3.0, 1e-4
    pos, t = lattice_block(2, 21, spacing=l0)
    pos = pos + 0.05
    c = pos.mean(0)
    vel = a * (pos - c)
    sc = scenes.Scene(2, l0, pos, vel, t, np.zeros(3), np.array([0.4, 0.4, 0.0]))
    prm, b, ps, fl = _hs_system(sc, vel, dt=dt)
    s = 1.0 + a * dt
    re_l0 = 2.1
    inv = sum(cnt / (s * math.sqrt(k)) for k, cnt in _shells()[2].items() if s * s * k < re_l0 ** 2)
    n0, _ = oracle.lattice(2, l0, re_l0 * l0)
    expect = -(a / s) * re_l0 * inv / (n0 * dt)
    inner = interior_mask(pos, 0.03) & (fl == 0)
    assert inner.sum() > 50
    np.testing.assert_allclose(b[inner], expect, rtol=1e-12)
    assert expect > 0            # a compressing flow (a < 0) gives a positive source


def test_hs_source_matches_finite_difference_of_pnd():
    """(Dn/Dt)* against a central difference of Eq. 5 along u*, for a smooth random flow."""
    sc = scenes.dam_break_2d(seed=2)
    x, y = sc.pos[:, 0], sc.pos[:, 1]
    vel = np.stack([0.3 * np.sin(7 * y) + 0.1, 0.2 * np.cos(5 * x)], axis=1)
    vel[sc.types != scenes.FLUID] = 0.0
    dt = 1e-4
    prm, b, ps, fl = _hs_system(sc, vel, dt=dt)
    us = vel.copy()                               # nu = 0, g = 0: u* = u
    h = 1e-7
    n0, _ = oracle.lattice(2, sc.l0, prm.re_n)
    npl = oracle.pnd(2, ps + h * us, sc.types, prm.re_n)
    nmi = oracle.pnd(2, ps - h * us, sc.types, prm.re_n)
    fd = (npl - nmi) / (2 * h) / (n0 * dt)
    rows = (sc.types <= scenes.WALL) & (fl == 0)
    scale = np.abs(fd[rows]).max()
    assert scale > 0
    assert np.abs(b[rows] - fd[rows]).max() <= 1e-5 * scale


def test_hs_requires_the_standard_kernel():
    sc = scenes.dam_break_2d(seed=1)
    prm = oracle.params_for(sc, source=1, kernel=1)
    with pytest.raises(oracle.OracleError):
        oracle.step(prm, oracle.State.from_scene(sc))


def test_ecs_source_closed_form_on_compressed_dilating_lattice():
    """Lattice at spacing s0 l0 (compressed: n^k > n0) with u = a (r - c): eps, (Dn/Dt)^k at
    r^k and (Dn/Dt)* at r* are all shell sums, so the HS + ECS source (Eq. 21, 24, 25) has
    a closed form at interior particles."""
    # compressed (eps > 0) and compressing (a < 0): both ECS terms are positive; with the
    # opposite signs they cancel, which is how Eq. 24 compensates only same-sign errors
    l0, s0, a, dt = 0.01, 0.99, -2.0, 1e-4
    pos, t = lattice_block(2, 21, spacing=s0 * l0)
    pos = pos + 0.05
    c = pos.mean(0)
    vel = a * (pos - c)
    sc = scenes.Scene(2, l0, pos, vel, t, np.zeros(3), np.array([0.4, 0.4, 0.0]))
    re_l0 = 2.1
    sh = _shells()[2]
    n0, _ = oracle.lattice(2, l0, re_l0 * l0)

    def sums(spacing):   # (sum w, sum re/r) over the shells inside re at this lattice spacing
        sw = sinv = 0.0
        for k, cnt in sh.items():
            r = spacing * math.sqrt(k)
            if r < re_l0:
                sw += cnt * (re_l0 / r - 1.0)
                sinv += cnt * re_l0 / r
        return sw, sinv

    nk, inv_k = sums(s0)
    s1 = s0 * (1.0 + a * dt)
    _, inv_s = sums(s1)
    dk = -a * inv_k                          # (Dn/Dt)^k = -a sum re/r
    dstar = -(a / (1.0 + a * dt)) * inv_s
    eps = (nk - n0) / n0
    ecs = abs(eps) * dk / n0 + abs(dt * dk / n0) * eps / dt
    expect = dstar / (n0 * dt) + ecs / dt
    prm2, b2, ps, fl = _hs_system(sc, vel, dt=dt)
    prm = oracle.params_for(sc, source=2, nu=0.0, g=(0.0, 0.0, 0.0), dt=dt)
    st = oracle.State.from_scene(sc)
    off, col, val, b, ps, ns, fl = oracle.ppe_system(prm, st)
    inner = interior_mask(pos, 0.03) & (fl == 0)
    assert inner.sum() > 50 and eps > 0 and ecs > 0
    np.testing.assert_allclose(b[inner], expect, rtol=1e-11)
    np.testing.assert_allclose(b[inner] - b2[inner], ecs / dt, rtol=1e-9)


def test_ecs_terms_cancel_for_an_expanded_compressing_lattice():
    """Expanded (eps < 0) and compressing ((Dn/Dt)^k > 0): the two terms of Eq. 24 cancel
    exactly, so the source is the HS term alone."""
    l0, s0, a, dt = 0.01, 1.01, -2.0, 1e-4
    pos, t = lattice_block(2, 21, spacing=s0 * l0)
    pos = pos + 0.05
    vel = a * (pos - pos.mean(0))
    sc = scenes.Scene(2, l0, pos, vel, t, np.zeros(3), np.array([0.4, 0.4, 0.0]))
    prm1, b1, ps, fl = _hs_system(sc, vel, dt=dt)
    prm = oracle.params_for(sc, source=2, nu=0.0, g=(0.0, 0.0, 0.0), dt=dt)
    st = oracle.State.from_scene(sc)
    off, col, val, b2, ps, ns, fl = oracle.ppe_system(prm, st)
    inner = interior_mask(pos, 0.03) & (fl == 0)
    assert inner.sum() > 50
    np.testing.assert_allclose(b2[inner], b1[inner], rtol=1e-12)
    assert np.all(b1[inner] > 0)
