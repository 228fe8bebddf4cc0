"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on the same
seeded inputs.  Bit-exact: cell keys, neighbour sets, free-surface flags (outside a
documented rounding band, asserted empty).  FP64: relative error <= 1e-10 with both CG
solves run to 1e-13.  Mixed precision: the stated bound (p: relative L2 over fluid <= 1e-5,
positions: <= 1e-6 l0) against the FP64 oracle."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, oracle_params, rel_err,
                     run_gpu, run_oracle, small_3d)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    oracle.set_threads(0)


def _mps():
    from paper_2105_01677_gb300 import mps
    return mps


# ------------------------------------------------------------------ constants, keys, sets
@pytest.mark.parametrize("dim", [2, 3])
def test_constants_match_oracle(dim):
    sc = scenes.dam_break_2d() if dim == 2 else small_3d()
    mps = _mps()
    sim = mps.Simulation(sc, **{})
    c = sim.constants()
    sim.close()
    n0n, _ = oracle.lattice(dim, sc.l0, 2.1 * sc.l0)
    n0l, lam = oracle.lattice(dim, sc.l0, 4.0 * sc.l0)
    assert c["n0_pnd"] == pytest.approx(n0n, rel=1e-14)
    assert c["n0_lap"] == pytest.approx(n0l, rel=1e-14)
    assert c["lambda_"] == pytest.approx(lam, rel=1e-14)


def _key_scenes():
    out = [scenes.dam_break_2d(seed=2), small_3d(seed=2)]
    for n, dim in ((2049, 2), (4097, 3), (6143, 3)):
        out.append(scenes.random_cloud(n, dim, seed=n, clustered=(dim == 3)))
    # particles exactly on cell faces and just outside the grid
    sc = scenes.random_cloud(3000, 3, seed=5)
    h = 4.0 * sc.l0 * 1.1
    k = np.arange(30) % 7
    sc.pos[:30, 0] = sc.box_min[0] + k * h
    sc.pos[30:40, 1] = sc.box_max[1] + 0.01
    sc.pos[40:50, 2] = sc.box_min[2] - 1e-12
    out.append(sc)
    # coordinates a relative 1e-10 ... 1e-5 of a cell side either side of cell faces: the
    # binary32 first tier of the cell floor decides the far ones, binary64 the near ones
    sc = scenes.random_cloud(3000, 3, seed=6)
    h = 4.0 * sc.l0 * 1.1
    rng = np.random.default_rng(6)
    m = 2400
    face = rng.integers(0, 8, size=(m, 3))
    rel = 10.0 ** rng.uniform(-10, -5, size=(m, 3)) * rng.choice([-1.0, 1.0], size=(m, 3))
    sc.pos[:m] = sc.box_min + (face + rel) * h
    out.append(sc)
    return out


@pytest.mark.parametrize("idx", range(7))
def test_cell_keys_bit_exact(idx):
    sc = _key_scenes()[idx]
    mps = _mps()
    sim = mps.Simulation(sc)
    got = mps.mps_debug_cells(sim.h, sc.n)
    sim.close()
    prm = oracle_params(sc)
    ref, _ = oracle.cell_keys(prm, sc.pos, sc.types)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("idx", range(5))
@pytest.mark.parametrize("which", [0, 1])
def test_neighbor_sets_bit_exact(idx, which):
    sc = _key_scenes()[idx]
    types = sc.types.copy()
    types[::29] = scenes.GHOST
    sc = scenes.Scene(sc.dim, sc.l0, sc.pos, sc.vel, types, sc.box_min, sc.box_max)
    mps = _mps()
    sim = mps.Simulation(sc)
    off, ids = mps.mps_debug_neighbors(sim.h, sc.n, which)
    sim.close()
    re = (2.1 if which == 0 else 4.0) * sc.l0
    mode = 0 if sc.n <= 5000 else 1
    roff, rids = oracle.neighbors(sc.dim, sc.pos, types, re, mode=mode)
    assert np.array_equal(off, roff)
    assert np.array_equal(ids, rids)


# ------------------------------------------------------------------ one FP64 step
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_step_fp64_dam_break_2d(seed):
    sc = scenes.dam_break_2d(seed=seed)
    kw = dict(cg_tol=PARITY_CG_TOL)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    compare_step(sc, got, ost, prm)
    assert rep["n_surface"] == orep["n_surface"] and rep["n_ppe_rows"] == orep["n_ppe_rows"]
    assert rep["cg_resid"] <= PARITY_CG_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_step_in_a_large_sparse_grid(precision):
    """The 2D dam break in a 10 m x 10 m grid: the cell table (228 x 228 cells, 2^16 Morton
    entries) is far larger than the particle count, so it is built by counts and their scan
    (not by a binary search per cell, as for the dense grids of the other tests)."""
    sc = scenes.dam_break_2d(seed=4)
    sc.box_max = sc.box_min + np.array([10.0, 10.0, 0.0])[: len(sc.box_min)]
    tol = PARITY_CG_TOL if precision == 0 else 1e-8
    rc, rep, got, consts = run_gpu(sc, **gpu_params(sc, precision=precision, cg_tol=tol))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL)
    assert consts["ncell"][0] * consts["ncell"][1] > 16 * sc.n
    if precision == 0:
        compare_step(sc, got, ost, prm)
    else:
        f = sc.types == scenes.FLUID
        assert np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f]) <= 1e-5
    assert np.array_equal(got["flags"], ost.flags)


@pytest.mark.parametrize("seed", [1, 2])
def test_step_fp64_dam_break_3d_small(seed):
    sc = small_3d(seed=seed)
    kw = dict(cg_tol=PARITY_CG_TOL)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    compare_step(sc, got, ost, prm)
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"]


def test_solve_ppe_fp64_leaves_state():
    sc = scenes.dam_break_2d(seed=1)
    kw = dict(cg_tol=PARITY_CG_TOL)
    rc, rep, got, _ = run_gpu(sc, solve_only=True, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, solve_only=True, **kw)
    assert rel_err(got["p"], ost.p) <= FP64_TOL
    rows = ost.types <= oracle.WALL
    assert rel_err(got["n_star"][rows], ost.nstar[rows]) <= FP64_TOL
    assert np.array_equal(got["pos"], sc.pos) and np.array_equal(got["vel"], sc.vel)


@pytest.mark.parametrize("dim", [2, 3])
def test_step_eos_fp64(dim):
    sc = scenes.dam_break_2d(seed=3) if dim == 2 else small_3d(seed=3)
    kw = dict(pressure_mode=1, c0=20.0)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    compare_step(sc, got, ost, prm)


def test_step_without_clamp_and_with_viscosity():
    sc = scenes.dam_break_2d(seed=2)
    rng = np.random.default_rng(0)
    sc.vel[sc.types == 0] = rng.standard_normal((sc.n_fluid, 2)) * 0.1
    kw = dict(cg_tol=PARITY_CG_TOL, clamp_negative_p=0, nu=1e-3)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    compare_step(sc, got, ost, prm)


# ------------------------------------------------------------------ mixed precision
def _mixed_errors(sc, got, ost):
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    return ep, ex


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_step_mixed_precision_bound(dim, op):
    sc = scenes.dam_break_2d(seed=1) if dim == 2 else small_3d(seed=1)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=1, ppe_operator=op, cg_tol=1e-8))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL)
    ep, ex = _mixed_errors(sc, got, ost)
    assert rep["cg_resid"] <= 1e-8
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)
    rows = ost.types <= oracle.WALL
    assert rel_err(got["n_star"][rows], ost.nstar[rows]) <= 1e-12


# ------------------------------------------------------------------ along a trajectory
def test_single_steps_from_oracle_states_along_dam_break():
    """Oracle trajectory; at steps 0, 50 and 99 the GPU restarts from the oracle state
    (mps_write_state) and both take one step."""
    sc = scenes.dam_break_2d(seed=1)
    kw = dict(cg_tol=PARITY_CG_TOL)
    prm = oracle_params(sc, **kw)
    st = oracle.State.from_scene(sc)
    mps = _mps()
    sim = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, **kw))
    try:
        for k in range(100):
            if k in (0, 50, 99):
                sim.write(st.pos, st.vel, st.types)
                sim.step(1)
                got = sim.read()
                before = oracle.State(st.pos.copy(), st.vel.copy(), st.types.copy(), st.p, st.nstar, st.flags)
                nxt = st.copy()
                oracle.step(prm, nxt)
                ref_scene = scenes.Scene(2, sc.l0, before.pos, before.vel, before.types, sc.box_min, sc.box_max)
                compare_step(ref_scene, got, nxt, prm)
            oracle.step(prm, st)
    finally:
        sim.close()


def test_gpu_dam_break_100_steps():
    sc = scenes.dam_break_2d(seed=3)
    mps = _mps()
    sim = mps.Simulation(sc, torch_alloc=True)
    n0, _ = oracle.lattice(2, sc.l0, 2.1 * sc.l0)
    for _ in range(100):
        rc, rep = sim.step(1)
        assert rep["cg_resid"] <= 1e-8
    got = sim.read()
    sim.close()
    assert np.all(np.isfinite(got["pos"])) and np.all(np.isfinite(got["p"]))
    assert np.count_nonzero(got["types"] == scenes.FLUID) == 800
    assert got["n_star"][got["types"] == scenes.FLUID].max() < 1.2 * n0
    assert np.all(got["n_star"][got["types"] == scenes.DUMMY] == 0.0)
    assert rep["steps_done"] == 100


def test_deterministic_bits():
    sc = small_3d(seed=1)
    outs = []
    for _ in range(2):
        rc, rep, got, _ = run_gpu(sc, nsteps=3, **gpu_params(sc))
        outs.append(got)
    for k in ("pos", "vel", "p", "n_star", "flags"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


# ------------------------------------------------------------------ edge cases and errors
def test_lone_particle_free_fall():
    sc = scenes.Scene(2, 0.01, np.array([[0.3, 0.3]]), np.array([[0.2, -0.1]]),
                      np.zeros(1, np.int8), np.zeros(3), np.array([1.0, 1.0, 0.0]))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, dt=1e-3))
    u1 = np.array([0.2, -0.1 - 9.81e-3])
    np.testing.assert_allclose(got["vel"][0], u1, rtol=1e-15)
    np.testing.assert_allclose(got["pos"][0], [0.3 + 1e-3 * 0.2, 0.3 + 1e-3 * u1[1]], rtol=1e-15)
    assert got["flags"][0] == 1 and got["p"][0] == 0.0


def test_all_ghost_scene_is_a_no_op():
    sc = scenes.dam_break_2d(seed=1)
    sc.types[:] = scenes.GHOST
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc))
    assert rc == 0 and rep["n_ppe_rows"] == 0 and rep["n_ghost"] == sc.n
    assert np.array_equal(got["pos"], sc.pos)


def test_particle_leaving_grid_becomes_ghost():
    sc = scenes.dam_break_2d(seed=1)
    sc.pos[7] = [5.0, 5.0]
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc))
    orep, ost, prm = run_oracle(sc)
    assert got["types"][7] == scenes.GHOST and rep["n_ghost"] == 1 == orep["n_ghost"]
    assert np.all(got["vel"][7] == 0.0)


def _lattice_block(dim, m, spacing, origin):
    g = np.meshgrid(*[np.arange(k) for k in m], indexing="ij")
    return np.stack([a.reshape(-1) for a in g], axis=1).astype(np.float64) * spacing + origin


def _mixed_bound(sc, got, ost):
    f = sc.types == scenes.FLUID
    assert np.linalg.norm(got["p"][f] - ost.p[f]) <= 1e-5 * np.linalg.norm(ost.p[f])
    assert np.abs(got["pos"] - ost.pos).max() <= 1e-6 * sc.l0


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_fluid_block_without_walls(dim, precision):
    """Degenerate scene: FLUID only, no walls or dummies, a block compressed to 0.98 l0 in
    free fall.  Every row of the PPE is a FLUID row; its surface rows (1/4 of the particles in
    2D, more than half in 3D) are the only Dirichlet conditions."""
    l0 = 0.01
    pos = _lattice_block(dim, (20, 12) if dim == 2 else (8, 8, 8), 0.98 * l0, 0.2)
    box = np.array([1.0, 1.0, 1.0 if dim == 3 else 0.0])
    sc = scenes.Scene(dim, l0, pos, np.zeros_like(pos), np.zeros(len(pos), np.int8),
                      np.zeros(3), box)
    tol = PARITY_CG_TOL if precision == 0 else 1e-8
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=precision, cg_tol=tol))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL)
    assert orep["n_ppe_rows"] > 0 and ost.p.max() > 0.0
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"] and rep["n_surface"] == orep["n_surface"]
    if precision == 0:
        compare_step(sc, got, ost, prm)
    else:
        _mixed_bound(sc, got, ost)
        assert np.array_equal(got["flags"], ost.flags)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_walls_and_dummies_only(dim, precision):
    """Degenerate scene: the dam-break tank with its fluid taken out.  The PPE still has
    rows (wall particles backed by dummies on two sides, n* between beta n0 and n0), with a
    negative right-hand side: with the clamp off their pressure is negative and compared;
    nothing moves."""
    full = scenes.dam_break_2d(seed=1) if dim == 2 else small_3d(seed=1)
    keep = full.types != scenes.FLUID
    sc = scenes.Scene(dim, full.l0, full.pos[keep].copy(), full.vel[keep].copy(),
                      full.types[keep].copy(), full.box_min, full.box_max)
    tol = PARITY_CG_TOL if precision == 0 else 1e-8
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=precision, cg_tol=tol,
                                               clamp_negative_p=0))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, clamp_negative_p=0)
    assert orep["n_ppe_rows"] > 0 and ost.p.min() < 0.0
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"]
    assert np.array_equal(got["pos"], sc.pos) and np.all(got["vel"] == 0.0)
    assert np.array_equal(got["flags"], ost.flags)
    if precision == 0:
        compare_step(sc, got, ost, prm, fields=("p", "n_star"))
    else:
        w = ost.types == scenes.WALL
        assert np.linalg.norm(got["p"][w] - ost.p[w]) <= 1e-5 * np.linalg.norm(ost.p[w])


@pytest.mark.parametrize("case", ["coincident", "noconv", "skin", "cap"])
def test_error_statuses(case):
    mps = _mps()
    sc = scenes.dam_break_2d(seed=1)
    kw = {}
    if case == "coincident":
        sc.pos[5] = sc.pos[6]
        expect = mps.ECOINCIDENT
    elif case == "noconv":
        kw = dict(cg_max_iter=1)
        expect = mps.ECG_NOCONV
    elif case == "skin":
        kw = dict(cell_skin=0.0)
        expect = mps.ESKIN
    else:
        kw = dict(nbr_cap=8)
        expect = mps.ECAP
    rc, rep, got, _ = run_gpu(sc, check=False, **gpu_params(sc, **kw))
    assert rc == expect, mps.mps_strerror(rc)
    if case != "cap":
        orc, _ = oracle.step(oracle_params(sc, **kw), oracle.State.from_scene(sc), check=False)
        assert orc == expect


def test_default_allocator_and_own_stream():
    sc = scenes.dam_break_2d(seed=1)
    rc, rep, got, _ = run_gpu(sc, torch_alloc=False, **gpu_params(sc, cg_tol=PARITY_CG_TOL))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL)
    compare_step(sc, got, ost, prm)


def test_mixed_precision_drift_over_100_steps():
    """The mixed path's N-step drift against the FP64 path (reported, not bounded
    by the paper): 100 steps of the 2D dam break (10 ms of flow).  Printed for the record;
    the assertion is only a sanity bound far above the single-step error."""
    sc = scenes.dam_break_2d(seed=3)
    mps = _mps()
    out = {}
    for prec in (0, 1):
        sim = mps.Simulation(sc, torch_alloc=True, precision=prec, cg_tol=1e-8)
        for _ in range(100):
            sim.step(1)
        out[prec] = sim.read()
        sim.close()
    f = sc.types == scenes.FLUID
    dx = np.abs(out[1]["pos"][f] - out[0]["pos"][f]).max() / sc.l0
    dp = np.linalg.norm(out[1]["p"][f] - out[0]["p"][f]) / np.linalg.norm(out[0]["p"][f])
    print(f"mixed vs FP64 after 100 steps: max |dx| = {dx:.3e} l0, relative L2 of p = {dp:.3e}")
    assert dx < 1e-2 and dp < 1e-2


def test_work_counters_match_oracle_sets():
    """The report's work counters (the bench's roofline work) count the pairs the method
    defines: number-density terms = neighbours of every kind within re_n at r* of the
    FLUID / WALL particles; PPE coefficients = their non-dummy neighbours within re_lap."""
    sc = scenes.dam_break_2d(seed=5)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, cg_tol=1e-10))
    prm = oracle_params(sc, cg_tol=1e-10)
    _, _, _, _, pstar, _, _ = oracle.ppe_system(prm, sc)
    fw = (sc.types == scenes.FLUID) | (sc.types == scenes.WALL)
    off_n, ids_n = oracle.neighbors(2, pstar, sc.types, prm.re_n, mode=0)
    off_l, ids_l = oracle.neighbors(2, pstar, sc.types, prm.re_lap, mode=0)
    rows_n = np.repeat(np.arange(sc.n), np.diff(off_n))
    rows_l = np.repeat(np.arange(sc.n), np.diff(off_l))
    pnd = int(np.count_nonzero(fw[rows_n]))
    ppe = int(np.count_nonzero(fw[rows_l] & (sc.types[ids_l] != scenes.DUMMY)))
    assert rep["pairs_pnd"] == pnd
    assert rep["pairs_ppe"] == ppe
    # the build classifies every FLUID / WALL row's candidate list: a superset of each row's
    # neighbours within max(re) at r*, within what the gather's tests produced
    off_h, ids_h = oracle.neighbors(2, pstar, sc.types, prm.re_lap, mode=0)
    within = int(np.count_nonzero(fw[np.repeat(np.arange(sc.n), np.diff(off_h))]))
    assert within <= rep["list_tests"] <= rep["cand_tests"]
