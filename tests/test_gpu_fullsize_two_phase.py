"""Parity at the two-phase workload's full size: the 3D dam break at l0 = 0.004 m
(1,125,000 fluid + 927,456 wall/dummy = 2,052,456 particles), light fluid (800 kg/m^3,
nu 5e-6) over water (1000, 1e-6), in the launch configuration bench.py times (library
defaults, dt = 5e-5, c0 = 20 m/s on the equation-of-state path).

One full FP64 oracle step per path on the host (cell-list neighbours, OpenMP over
particles); the PPE solves run to 1e-13 on both sides for the FP64 comparison."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, oracle_params, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    oracle.set_threads(0)
    sc = scenes.dam_break_3d(seed=1, l0=0.004)
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 800.0), nu=(1e-6, 5e-6))
    return sc, dict(rho_i=rho, nu_i=nu)


def _oracle(sc, **kw):
    prm = oracle_params(sc, **kw)
    st = oracle.State.from_scene(sc)
    _, rep = oracle.step(prm, st)
    return prm, st, rep


@pytest.fixture(scope="module")
def oracle_ppe(scene):
    sc, props = scene
    return _oracle(sc, dt=5e-5, cg_tol=PARITY_CG_TOL, **props)


def test_fullsize_two_phase_ppe_fp64(scene, oracle_ppe):
    sc, props = scene
    prm, ost, orep = oracle_ppe
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, dt=5e-5, cg_tol=PARITY_CG_TOL, **props))
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"] and rep["n_surface"] == orep["n_surface"]
    errs = compare_step(sc, got, ost, prm)
    assert max(errs.values()) <= FP64_TOL


def test_fullsize_two_phase_ppe_mixed_bound(scene, oracle_ppe):
    sc, props = scene
    prm, ost, orep = oracle_ppe
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, dt=5e-5, precision=1, cg_tol=1e-8, **props))
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert rep["cg_resid"] <= 1e-8
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)


def test_fullsize_two_phase_eos_fp64_and_mixed(scene):
    sc, props = scene
    prm, ost, orep = _oracle(sc, dt=5e-5, pressure_mode=1, c0=20.0, **props)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, dt=5e-5, pressure_mode=1, c0=20.0, **props))
    compare_step(sc, got, ost, prm)
    rc, rep, gm, _ = run_gpu(sc, **gpu_params(sc, dt=5e-5, pressure_mode=1, c0=20.0, precision=1,
                                              **props))
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(gm["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    assert ep <= 1e-5, ep
    assert np.abs(gm["pos"] - ost.pos).max() / sc.l0 <= 1e-6
    assert np.array_equal(gm["flags"], ost.flags)
