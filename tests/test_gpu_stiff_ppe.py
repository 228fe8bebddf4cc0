"""GPU parity on the stiff PPE: Eq. 13 without the diagonal term of the PPE listing
(alpha_c = 0, allowed where every connected part of the system has a free-surface row, as
the dam break has).  Without alpha_c/dt^2 the diagonal is the Laplacian's alone and CG
needs 45-75 iterations on these scenes instead of 4-11, so these cases exercise the solver
(FP64 CG, and the FP32-inner / FP64-outer refinement of the mixed path) where its
iteration count matters.

FP64: relative error <= 1e-10 with both CG solves run to 1e-13.  Mixed: the stated bound
(p: relative L2 over fluid <= 1e-5, positions <= 1e-6 l0) against the FP64 oracle.

At the first step of the dam break the unclamped solution is negative everywhere (the
source term's deficit of number density near the surface), so the clamp would leave p = 0:
the single-step cases compare the unclamped solution, and a 2D case compares a step from
the oracle's state 30 clamped steps in, where 28% of the fluid has positive pressure."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, oracle_params, rel_err,
                     run_gpu, run_oracle, small_3d)

pytestmark = pytest.mark.gpu

STIFF = dict(alpha_c=0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    oracle.set_threads(0)


def _scene(dim):
    return (scenes.dam_break_2d(seed=1), 1e-4) if dim == 2 else (small_3d(seed=1), 5e-5)


@pytest.mark.parametrize("dim", [2, 3])
def test_stiff_step_fp64(dim):
    sc, dt = _scene(dim)
    kw = dict(dt=dt, cg_tol=PARITY_CG_TOL, clamp_negative_p=0, **STIFF)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, **kw))
    orep, ost, prm = run_oracle(sc, **kw)
    assert orep["cg_iters"] >= 40          # the stiff system, not the regularised one
    assert rep["cg_resid"] <= PARITY_CG_TOL
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("dim", [2, 3])
def test_stiff_step_mixed_bound(dim):
    sc, dt = _scene(dim)
    kw = dict(dt=dt, clamp_negative_p=0, **STIFF)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=1, cg_tol=1e-8, **kw))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **kw)
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert rep["cg_resid"] <= 1e-8
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)
    rows = ost.types <= oracle.WALL
    assert rel_err(got["n_star"][rows], ost.nstar[rows]) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_stiff_step_from_a_developed_state(precision):
    """The oracle runs 30 clamped steps of the 2D dam break on the stiff PPE; from its state
    both sides take one step (FP64 to the parity tolerance, mixed to its bound).

    The compared step leaves the solution unclamped.  Both solves stop at a residual of
    1e-13 |b|, which bounds their difference by ~kappa 1e-13 of the full solution (kappa ~200
    here); after the clamp only the positive part remains, whose largest value is ~70x
    smaller than the solution's (the suction below the free surface), so the same absolute
    difference would read ~70x larger against it.  The clamp itself (max(p, 0)) is
    1-Lipschitz and is compared by the regularised-system tests."""
    sc, dt = _scene(2)
    kw = dict(dt=dt, cg_tol=PARITY_CG_TOL, **STIFF)
    prm = oracle_params(sc, **kw)
    st = oracle.State.from_scene(sc)
    for _ in range(30):
        oracle.step(prm, st)
    start = scenes.Scene(2, sc.l0, st.pos.copy(), st.vel.copy(), st.types.copy(), sc.box_min,
                         sc.box_max)
    f = start.types == scenes.FLUID
    assert (st.p[f] > 0).mean() > 0.1      # a developed flow: positive pressure in the fluid
    kw = dict(kw, clamp_negative_p=0)
    prm = oracle_params(start, **kw)
    nxt = st.copy()
    oracle.step(prm, nxt)
    gkw = dict(kw, cg_tol=PARITY_CG_TOL if precision == 0 else 1e-8)
    rc, rep, got, _ = run_gpu(start, precision=precision, **gpu_params(start, **gkw))
    if precision == 0:
        compare_step(start, got, nxt, prm)
    else:
        ep = np.linalg.norm(got["p"][f] - nxt.p[f]) / np.linalg.norm(nxt.p[f])
        ex = np.abs(got["pos"] - nxt.pos).max() / sc.l0
        assert rep["cg_resid"] <= 1e-8
        assert ep <= 1e-5, ep
        assert ex <= 1e-6, ex
