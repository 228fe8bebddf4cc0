"""Parity at the bench's full size: the 3D dam break with 440,032 particles (169,600
fluid), in the launch configuration bench.py times (library defaults, dt = 5e-5).

The oracle runs one full FP64 step (cell-list neighbours, OpenMP over particles) on the
host; both CG solves run to 1e-13 for the FP64 comparison.  Keys and neighbour sets are
compared bit-exactly; the mixed-precision step against its stated bound."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, oracle_params, rel_err,
                     run_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    oracle.set_threads(0)
    return scenes.dam_break_3d(seed=1)


@pytest.fixture(scope="module")
def oracle_step(scene):
    kw = dict(dt=5e-5, cg_tol=PARITY_CG_TOL)
    prm = oracle_params(scene, **kw)
    st = oracle.State.from_scene(scene)
    _, rep = oracle.step(prm, st)
    return prm, st, rep


def test_fullsize_cell_keys_and_neighbor_sets(scene):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(scene, torch_alloc=True, **gpu_params(scene, dt=5e-5))
    try:
        keys = mps.mps_debug_cells(sim.h, scene.n)
        off_n, ids_n = mps.mps_debug_neighbors(sim.h, scene.n, 0)
        off_l, ids_l = mps.mps_debug_neighbors(sim.h, scene.n, 1)
    finally:
        sim.close()
    ref_keys, _ = oracle.cell_keys(oracle_params(scene, dt=5e-5), scene.pos, scene.types)
    assert np.array_equal(keys, ref_keys)
    for (off, ids), re in (((off_n, ids_n), 2.1), ((off_l, ids_l), 4.0)):
        roff, rids = oracle.neighbors(3, scene.pos, scene.types, re * scene.l0, mode=1)
        assert np.array_equal(off, roff)
        assert np.array_equal(ids, rids)


def test_fullsize_step_fp64(scene, oracle_step):
    prm, ost, orep = oracle_step
    rc, rep, got, _ = run_gpu(scene, **gpu_params(scene, dt=5e-5, cg_tol=PARITY_CG_TOL))
    errs = compare_step(scene, got, ost, prm)
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"] and rep["n_surface"] == orep["n_surface"]
    assert max(errs.values()) <= FP64_TOL


def test_fullsize_step_mixed_bound(scene, oracle_step):
    prm, ost, orep = oracle_step
    rc, rep, got, _ = run_gpu(scene, **gpu_params(scene, dt=5e-5, precision=1, cg_tol=1e-8))
    f = scene.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / scene.l0
    assert rep["cg_resid"] <= 1e-8
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)
    rows = ost.types <= oracle.WALL
    assert rel_err(got["n_star"][rows], ost.nstar[rows]) <= 1e-12


# ------------------------------------------------------------------ the bench's trajectory
TRAJ_STEPS = 5


@pytest.fixture(scope="module")
def oracle_trajectory(scene):
    """The oracle's first five steps (PPE from zero to 1e-13), a copy after each."""
    prm = oracle_params(scene, dt=5e-5, cg_tol=PARITY_CG_TOL)
    st = oracle.State.from_scene(scene)
    out = []
    for _ in range(TRAJ_STEPS):
        oracle.step(prm, st)
        out.append(st.copy())
    return prm, out


def _gpu_trajectory(scene, tune_after=None, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(scene, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(scene, dt=5e-5, **kw))
    states, reps = [], []
    try:
        for k in range(TRAJ_STEPS):
            if tune_after is not None and k == tune_after:
                sim.tuning = sim.autotune(1)
            _, rep = sim.step(1)
            reps.append(rep)
            states.append(sim.read())
    finally:
        sim.close()
    return states, reps


def test_fullsize_mixed_trajectory_with_quadratic_guess(scene, oracle_trajectory):
    """The headline configuration over five steps: mixed precision, PPE started from the
    extrapolation of the previous solutions (cg_x0 = 3), true FP64 residual <= 1e-8 each
    step; every step's state within the mixed bound of the oracle's trajectory."""
    prm, ref = oracle_trajectory
    got, reps = _gpu_trajectory(scene, precision=1, cg_tol=1e-8, cg_x0=3)
    f = scene.types == scenes.FLUID
    n0, _ = oracle.lattice(3, scene.l0, 2.1 * scene.l0)
    for k in range(TRAJ_STEPS):
        assert reps[k]["cg_resid"] <= 1e-8
        ep = np.linalg.norm(got[k]["p"][f] - ref[k].p[f]) / np.linalg.norm(ref[k].p[f])
        ex = np.abs(got[k]["pos"] - ref[k].pos).max() / scene.l0
        assert ep <= 1e-5, (k, ep)
        assert ex <= 1e-6, (k, ex)
        # after the first step the positions differ at the mixed bound, so n* may too:
        # flags agree outside a band of 1e-7 n0 around the threshold
        band = np.abs(ref[k].nstar - prm.beta * n0) <= 1e-7 * n0
        assert np.array_equal(got[k]["flags"][~band], ref[k].flags[~band]), k
    # the guess is used from the second step on: fewer inner iterations than the cold start
    assert min(r["cg_iters"] for r in reps[2:]) < reps[0]["cg_iters"]


def test_fullsize_mixed_trajectory_tuned(scene, oracle_trajectory):
    """The benchmarked configuration: two steps, the autotuner (cell side, gather and build
    blocks, threads per prediction row, SpMV block, inner-CG form and unrolling), three more
    steps; every step within the mixed bound of the oracle's trajectory (the tuned choices
    change the order of sums, not the method), the FP64 residual <= 1e-8 each step."""
    prm, ref = oracle_trajectory
    got, reps = _gpu_trajectory(scene, tune_after=2, precision=1, cg_tol=1e-8, cg_x0=3)
    f = scene.types == scenes.FLUID
    n0, _ = oracle.lattice(3, scene.l0, 2.1 * scene.l0)
    for k in range(TRAJ_STEPS):
        assert reps[k]["cg_resid"] <= 1e-8
        ep = np.linalg.norm(got[k]["p"][f] - ref[k].p[f]) / np.linalg.norm(ref[k].p[f])
        ex = np.abs(got[k]["pos"] - ref[k].pos).max() / scene.l0
        assert ep <= 1e-5, (k, ep)
        assert ex <= 1e-6, (k, ex)
        band = np.abs(ref[k].nstar - prm.beta * n0) <= 1e-7 * n0
        assert np.array_equal(got[k]["flags"][~band], ref[k].flags[~band]), k
    # the steps after tuning ran as one graph each, the bucket build merging its movers
    assert all(r["step_graph"] == 1 for r in reps[2:])
    assert all(r["bucket_merged"] == 1 for r in reps[3:])


def test_fullsize_fp64_trajectory_with_quadratic_guess(scene, oracle_trajectory):
    """FP64 with cg_x0 = 3 over five steps against the oracle (which starts every solve
    from zero) at max(1e-10, 4x the oracle's own one-ulp sensitivity over those steps)."""
    from _parity import ulp_sensitivity
    prm, ref = oracle_trajectory
    got, reps = _gpu_trajectory(scene, precision=0, cg_tol=PARITY_CG_TOL, cg_x0=3)
    sens = ulp_sensitivity(scene, TRAJ_STEPS, dt=5e-5, cg_tol=PARITY_CG_TOL)
    for name, key in (("p", "p"), ("vel", "vel")):
        tol = max(FP64_TOL, 4.0 * sens[name])
        err = rel_err(got[-1][key], getattr(ref[-1], name))
        assert err <= tol, (name, err, tol)
    for k in range(TRAJ_STEPS):
        assert np.array_equal(got[k]["flags"], ref[k].flags), k
        assert np.array_equal(got[k]["types"], ref[k].types), k
