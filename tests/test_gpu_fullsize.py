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
