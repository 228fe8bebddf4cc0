"""Two-phase flow (Sec. 3.2.1) on the GPU against the oracle: per-particle density and
viscosity (light fluid over heavy fluid in the dam-break column), on the PPE and on the
equation-of-state paths, FP64 to the single-step bound and mixed precision to its bound."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, rel_err, run_gpu,
                     run_oracle, small_3d, ulp_sensitivity)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _props(sc):
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 800.0), nu=(1e-6, 5e-6))
    return dict(rho_i=rho, nu_i=nu)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_two_phase_fp64_2d(mode, seed):
    sc = scenes.dam_break_2d(seed=seed)
    kw = dict(pressure_mode=mode, cg_tol=PARITY_CG_TOL, **_props(sc))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("mode", [0, 1])
def test_two_phase_fp64_3d_small(mode):
    sc = small_3d(seed=1)
    kw = dict(pressure_mode=mode, cg_tol=PARITY_CG_TOL, **_props(sc))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"]
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("mode", [0, 1])
def test_two_phase_mixed_bound_3d_small(mode):
    sc = small_3d(seed=2)
    props = _props(sc)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=1, pressure_mode=mode, **props))
    orep, ost, prm = run_oracle(sc, pressure_mode=mode, cg_tol=PARITY_CG_TOL, **props)
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)


def test_two_phase_fp64_five_steps_2d():
    sc = scenes.dam_break_2d(seed=3)
    kw = dict(cg_tol=PARITY_CG_TOL, **_props(sc))
    rc, rep, got, _ = run_gpu(sc, nsteps=5, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, nsteps=5, **kw)
    compare_step(sc, got, ost, prm, fields=("n_star", "vel", "disp"))
    sens = ulp_sensitivity(sc, 5, **kw)
    assert rel_err(got["p"], ost.p) <= max(FP64_TOL, 4.0 * sens["p"])


def test_two_phase_properties_follow_write_state_and_reset():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    props = _props(sc)
    kw = gpu_params(sc, cg_tol=PARITY_CG_TOL)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **props, **kw)
    try:
        sim.step(1)
        sim.write(sc.pos, sc.vel, sc.types)   # back to the initial state, properties kept
        sim.step(1)
        got = sim.read()
        sim.set_fluid_properties(None, None)   # single phase again
        sim.write(sc.pos, sc.vel, sc.types)
        sim.step(1)
        single = sim.read()
    finally:
        sim.close()
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **props)
    compare_step(sc, got, ost, prm)
    orep1, ost1, prm1 = run_oracle(sc, cg_tol=PARITY_CG_TOL)
    compare_step(sc, single, ost1, prm1)


def test_two_phase_invalid_properties():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    sim = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc))
    try:
        rho, nu = scenes.two_phase(sc)
        bad = rho.copy()
        bad[3] = 0.0
        assert sim.set_fluid_properties(bad, None, check=False) == mps.EINVAL
        bad[3] = np.nan
        assert sim.set_fluid_properties(bad, None, check=False) == mps.EINVAL
        nub = nu.copy()
        nub[5] = -1e-6
        assert sim.set_fluid_properties(None, nub, check=False) == mps.EINVAL
        assert sim.set_fluid_properties(rho, nu, check=False) == mps.OK
    finally:
        sim.close()
    simf = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, precision=1, ppe_operator=1))
    try:
        assert simf.set_fluid_properties(rho, None, check=False) == mps.EINVAL
    finally:
        simf.close()
