"""Candidate lists kept across steps (list_every > 1) against the oracle, which defines every
neighbour set afresh at every step (Sec. 4.1).  A kept list is a superset gathered within
h = max(re)(1 + s) at r_b; while no particle has moved more than s max(re)/2 from r_b the
sets filtered out of it are the exact sets, so the kept and the every-step runs differ only
in summation order.  The tests also drive the three ways a kept list is given up: its age,
a predicted position r* beyond the skin (the step restarts with a fresh gather) and a
particle leaving the cell grid."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, oracle_params, rel_err,
                     small_3d, ulp_sensitivity)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _run_steps(scene, nsteps, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(scene, torch_alloc=True, use_torch_stream=True, **kw)
    gathered = []
    try:
        for _ in range(nsteps):
            rc, rep = sim.step(1)
            gathered.append(rep["list_gathered"])
        st = sim.read()
    finally:
        sim.close()
    return st, rep, gathered


def _oracle_steps(scene, nsteps, **kw):
    prm = oracle_params(scene, **kw)
    st = oracle.State.from_scene(scene)
    for _ in range(nsteps):
        oracle.step(prm, st)
    return st, prm


@pytest.mark.parametrize("seed", [1, 2])
def test_kept_lists_fp64_2d_matches_oracle(seed):
    sc = scenes.dam_break_2d(seed=seed)
    got, rep, gathered = _run_steps(sc, 9, **gpu_params(sc, cg_tol=PARITY_CG_TOL, list_every=4))
    assert gathered == [1, 0, 0, 0, 1, 0, 0, 0, 1]
    ost, prm = _oracle_steps(sc, 9, cg_tol=PARITY_CG_TOL)
    compare_step(sc, got, ost, prm)


def test_kept_lists_fp64_3d_same_as_every_step():
    sc = small_3d(seed=2)
    kw = gpu_params(sc, cg_tol=PARITY_CG_TOL)
    every, _, g1 = _run_steps(sc, 6, **kw)
    kept, _, g4 = _run_steps(sc, 6, list_every=4, **kw)
    assert g1 == [1] * 6 and g4 == [1, 0, 0, 0, 1, 0]
    for k in ("pos", "vel", "p", "n_star"):
        assert rel_err(kept[k], every[k]) <= 1e-11, k
    assert np.array_equal(kept["flags"], every["flags"])
    assert np.array_equal(kept["types"], every["types"])


def test_kept_lists_mixed_3d_bound():
    """Mixed precision over 4 steps (3 of them on kept lists) against the FP64 oracle: the
    single-step bound (p 1e-5 relative L2 over fluid, positions 1e-6 l0) times the steps."""
    sc = small_3d(seed=1)
    got, rep, gathered = _run_steps(sc, 4, **gpu_params(sc, precision=1, list_every=4))
    assert gathered == [1, 0, 0, 0]
    ost, prm = _oracle_steps(sc, 4, cg_tol=PARITY_CG_TOL)
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert ep <= 4e-5, ep
    assert ex <= 4e-6, ex
    assert np.array_equal(got["flags"], ost.flags)


def test_kept_lists_gather_afresh_when_skin_is_used_up():
    """Fluid moving at 4 m/s covers 0.04 l0 per step; a skin s = 0.05 allows s re_lap/2 =
    0.1 l0 from r_b, so r* of the third step after a gather is beyond it: that step restarts
    on a fresh gather although the list is far from its age of 10 steps."""
    sc = scenes.dam_break_2d(seed=1)
    f = sc.types == scenes.FLUID
    sc.vel[f] = [4.0, 0.0]
    kw = dict(cg_tol=PARITY_CG_TOL, cell_skin=0.05)
    got, rep, gathered = _run_steps(sc, 5, **gpu_params(sc, list_every=10, **kw))
    assert gathered == [1, 0, 1, 0, 1], gathered
    every, _, _ = _run_steps(sc, 5, **gpu_params(sc, **kw))
    for k in ("pos", "vel", "p", "n_star"):
        assert rel_err(got[k], every[k]) <= FP64_TOL, k
    ost, prm = _oracle_steps(sc, 5, **kw)
    # five steps of a moving column: one ulp in the fluid positions already moves the oracle's
    # own p by ~2e-10, so p takes four times that sensitivity (not less than 1e-10)
    compare_step(sc, got, ost, prm, fields=("n_star", "vel", "disp"))
    sens = ulp_sensitivity(sc, 5, **kw)
    assert rel_err(got["p"], ost.p) <= max(FP64_TOL, 4.0 * sens["p"])


def test_kept_lists_particle_leaving_grid():
    """A lone fluid particle just inside the last cell of the grid, moving out: the next step
    gathers afresh and the particle becomes a GHOST exactly when the oracle makes it one."""
    sc = scenes.dam_break_2d(seed=1)
    h = 4.0 * sc.l0 * 1.1
    ncell = np.floor((sc.box_max[0] - sc.box_min[0]) / h) + 1
    edge = sc.box_min[0] + ncell * h
    pos = np.vstack([sc.pos, [[edge - 1e-4, 0.45]]])
    vel = np.vstack([sc.vel, [[2.0, 0.0]]])
    types = np.concatenate([sc.types, np.array([scenes.FLUID], np.int8)])
    sc2 = scenes.Scene(2, sc.l0, pos, vel, types, sc.box_min.copy(), sc.box_max.copy())
    kw = dict(cg_tol=PARITY_CG_TOL)
    got, rep, gathered = _run_steps(sc2, 3, **gpu_params(sc2, list_every=4, **kw))
    assert gathered == [1, 1, 0], gathered
    ost, prm = _oracle_steps(sc2, 3, **kw)
    assert got["types"][-1] == scenes.GHOST == ost.types[-1]
    assert rep["n_ghost"] == 1
    compare_step(sc2, got, ost, prm)


def test_kept_lists_write_state_gathers_afresh():
    sc = scenes.dam_break_2d(seed=2)
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, list_every=8))
    try:
        sim.step(2)
        sim.write(sc.pos, sc.vel, sc.types)
        rc, rep = sim.step(1)
        assert rep["list_gathered"] == 1
        rc, rep = sim.step(1)
        assert rep["list_gathered"] == 0
    finally:
        sim.close()
