"""Particles that outrun the cell skin within a step.

The candidate lists are gathered at r^k within max(re)(1 + s); a particle moving more than
s max(re)/2 in one step may then miss pairs at r*.  The library completes the lists of such
particles by a direct search at r* (and enters them into their neighbours' lists), so the
neighbour sets stay exact, and reports MPS_ESKIN only beyond max(64, n/256) of them -- the
oracle searches its sets at r* afresh and follows the same limit.  Cases: a few kicked
particles in 2D and 3D, FP64 to the parity tolerance and mixed to its bound, with the step
graph (which hands such a step to the host-driven path) and without, and the limit."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import PARITY_CG_TOL, compare_step, gpu_params, run_gpu, run_oracle, small_3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    oracle.set_threads(0)


def _kicked(dim):
    if dim == 2:
        sc = scenes.dam_break_2d(seed=4)
        f = np.flatnonzero(sc.types == scenes.FLUID)
        sc.vel[f[[5, 300, 700]]] = [[40.0, 0.0], [0.0, 35.0], [-30.0, 20.0]]   # 3-4 mm / step
        return sc, 1e-4
    sc = small_3d(seed=5)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    rng = np.random.default_rng(3)
    pick = rng.choice(f, size=12, replace=False)
    sc.vel[pick] = rng.uniform(-1.0, 1.0, size=(12, 3)) * 150.0               # up to 1.3 cm
    return sc, 5e-5


@pytest.mark.parametrize("step_graph", [1, 0])
@pytest.mark.parametrize("dim", [2, 3])
def test_fast_particles_fp64_parity(dim, step_graph):
    sc, dt = _kicked(dim)
    kw = dict(dt=dt, cg_tol=PARITY_CG_TOL)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, step_graph=step_graph, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    re_max = 4.0 * sc.l0
    assert rc == 0 and rep["max_disp"] > 0.5 * 0.1 * re_max   # beyond half the full skin
    assert rep["n_fast"] == 3 if dim == 2 else 1 <= rep["n_fast"] <= 12
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("dim", [2, 3])
def test_fast_particles_mixed_bound(dim):
    sc, dt = _kicked(dim)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, dt=dt, precision=1, cg_tol=1e-8))
    orep, ost, prm = run_oracle(sc, dt=dt, cg_tol=PARITY_CG_TOL)
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert rc == 0 and ep <= 1e-5 and ex <= 1e-6, (ep, ex)
    assert np.array_equal(got["flags"], ost.flags)


def test_more_fast_particles_than_the_limit_is_eskin():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=4)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    sc.vel[f[:65]] = [30.0, 0.0]
    for step_graph in (1, 0):
        rc, rep, got, _ = run_gpu(sc, check=False, **gpu_params(sc, step_graph=step_graph))
        assert rc == mps.ESKIN
    sc.vel[f[64]] = [0.0, 0.0]
    rc, rep, got, _ = run_gpu(sc, check=False, **gpu_params(sc))
    assert rc == 0
