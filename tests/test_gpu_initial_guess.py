"""The PPE started from the previous solves (cg_x0 = 1: the previous solution; 2, 3: its
linear and quadratic extrapolation): the same solution as a cold start to the tolerance,
oracle parity along a short trajectory, fewer iterations, the lower orders while the
history is short, identical results from the device-driven and host-driven loops, and a
written state that restarts cold."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, compare_step, gpu_params, rel_err, run_gpu,
                     run_oracle, small_3d, ulp_sensitivity)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _scene(name):
    return scenes.dam_break_2d(seed=2) if name == "2d" else small_3d(seed=2)


def _steps(sc, nsteps, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, **kw))
    try:
        reps = [sim.step(1)[1] for _ in range(nsteps)]
        st = sim.read()
    finally:
        sim.close()
    return reps, st


@pytest.mark.parametrize("host_loop", [0, 1])
def test_first_step_is_the_cold_start_bitwise(host_loop):
    """Before any solve the guess is zero: the mixed solve from it is the cold solve bit for
    bit (r = b - A 0 = b exactly, the same reductions in the same order)."""
    sc = small_3d(seed=1)
    kw = dict(precision=1, dt=5e-5, ppe_host_loop=host_loop)
    r0, s0 = _steps(sc, 1, cg_x0=0, **kw)
    r1, s1 = _steps(sc, 1, cg_x0=1, **kw)
    assert (r0[0]["cg_iters"], r0[0]["cg_outer"], r0[0]["cg_resid"]) == \
        (r1[0]["cg_iters"], r1[0]["cg_outer"], r1[0]["cg_resid"])
    for k in ("pos", "vel", "p", "n_star", "flags"):
        assert np.array_equal(s0[k], s1[k]), k


@pytest.mark.parametrize("scene,x0", [("2d", 1), ("3d", 1), ("2d", 3), ("3d", 2)])
def test_guess_trajectory_matches_oracle(scene, x0):
    """FP64, four steps at the parity tolerance: every solve after the first starts from the
    previous solutions (or their extrapolation); the oracle starts every solve from zero.
    The bound is the oracle's own sensitivity to one-ulp changes of the positions over the
    same steps."""
    sc = _scene(scene)
    nsteps = 4
    dt = 1e-4 if sc.dim == 2 else 5e-5
    kw = dict(cg_tol=PARITY_CG_TOL, dt=dt)
    rc, rep, got, _ = run_gpu(sc, nsteps=nsteps, **gpu_params(sc, cg_x0=x0, **kw))
    orep, ost, prm = run_oracle(sc, nsteps=nsteps, **kw)
    sens = ulp_sensitivity(sc, nsteps, **kw)
    tol = max(FP64_TOL, 10.0 * max(sens.values()))
    compare_step(sc, got, ost, prm, tol=tol, fields=("p", "n_star", "vel"))
    assert rep["cg_resid"] <= PARITY_CG_TOL


@pytest.mark.parametrize("precision,x0", [(0, 1), (1, 1), (1, 2), (1, 3), (0, 3), (1, 4), (0, 4)])
def test_guess_agrees_with_cold_start_and_cuts_iterations(precision, x0):
    sc = small_3d(seed=3)
    kw = dict(precision=precision, dt=5e-5, cg_tol=1e-8)
    rc_, sc_ = _steps(sc, 6, cg_x0=0, **kw)
    rw_, sw_ = _steps(sc, 6, cg_x0=x0, **kw)
    assert all(r["cg_resid"] <= 1e-8 for r in rc_ + rw_)
    cold = sum(r["cg_iters"] for r in rc_[1:])
    warm = sum(r["cg_iters"] for r in rw_[1:])
    assert warm < cold, (warm, cold)
    # both are solutions to 1e-8: the states agree to what that tolerance leaves
    assert rel_err(sw_["p"], sc_["p"]) <= 1e-5
    assert rel_err(sw_["vel"], sc_["vel"]) <= 1e-5
    assert np.array_equal(sw_["flags"], sc_["flags"])


@pytest.mark.parametrize("scene,nsteps,x0", [("2d", 5, 1), ("3d", 3, 1), ("2d", 5, 3), ("2d", 6, 4)])
def test_graph_equals_host_loop_with_guess(scene, nsteps, x0):
    sc = _scene(scene)
    dt = 1e-4 if sc.dim == 2 else 5e-5
    out = [_steps(sc, nsteps, precision=1, dt=dt, cg_x0=x0, ppe_host_loop=h) for h in (0, 1)]
    (rg, sg), (rh, sh) = out
    for a, b in zip(rg, rh):
        assert (a["cg_iters"], a["cg_outer"], a["cg_resid"]) == (b["cg_iters"], b["cg_outer"], b["cg_resid"])
    for k in ("pos", "vel", "p", "n_star", "flags", "types"):
        assert np.array_equal(sg[k], sh[k]), k


def test_graph_equals_host_loop_with_guess_ensemble():
    from paper_2105_01677_gb300 import mps
    E = scenes.ensemble_2d(count=5, seed=6, fluid=(150, 1200))
    out = []
    for host_loop in (0, 1):
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1,
                           cg_tol=1e-9, ppe_host_loop=host_loop, cg_x0=2)
        try:
            reps = [ens.step(1)[1] for _ in range(4)]
            out.append((reps, ens.read(), ens.residuals()))
        finally:
            ens.close()
    (rg, sg, resg), (rh, sh, resh) = out
    for a, b in zip(rg, rh):
        assert (a["cg_iters"], a["cg_outer"], a["cg_resid"]) == (b["cg_iters"], b["cg_outer"], b["cg_resid"])
    assert np.array_equal(resg, resh) and np.all(resg <= 1e-9)
    for a, b in zip(sg, sh):
        for k in ("pos", "vel", "p", "n_star", "flags"):
            assert np.array_equal(a[k], b[k]), k


def test_written_state_restarts_cold():
    """mps_write_state of a new state clears the guess: stepping the same written state twice
    gives the same bits, although the guess after the first of them would differ."""
    from paper_2105_01677_gb300 import mps
    sc = _scene("2d")
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, precision=1, cg_x0=3))
    try:
        sim.step(3)
        s = sim.read()
        f = np.flatnonzero(s["types"] == 0)[0]
        moved = s["pos"].copy()
        moved[f, 0] = np.nextafter(moved[f, 0], 1.0)   # another state than the context's
        outs = []
        for _ in range(2):
            sim.write(moved, s["vel"], s["types"])
            rep = sim.step(1)[1]
            outs.append((rep, sim.read()))
    finally:
        sim.close()
    (ra, a), (rb, b) = outs
    assert (ra["cg_iters"], ra["cg_resid"]) == (rb["cg_iters"], rb["cg_resid"])
    for k in ("pos", "vel", "p", "n_star", "flags"):
        assert np.array_equal(a[k], b[k]), k


def test_writing_back_the_same_state_changes_nothing():
    """Reading the state and writing it back unchanged is a no-op: the next step (with its
    guess from the history) is bit for bit the step without the write; clear_history then
    restarts cold like a new state."""
    from paper_2105_01677_gb300 import mps
    sc = _scene("2d")
    outs = []
    for mode in ("plain", "write-back", "clear"):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, cg_x0=3))
        try:
            sim.step(3)
            if mode != "plain":
                s = sim.read()
                sim.write(s["pos"], s["vel"], s["types"])
            if mode == "clear":
                sim.clear_history()
            rep = sim.step(1)[1]
            outs.append((rep, sim.read()))
        finally:
            sim.close()
    (r0, a), (r1, b), (r2, c) = outs
    assert (r0["cg_iters"], r0["cg_resid"]) == (r1["cg_iters"], r1["cg_resid"])
    for k in ("pos", "vel", "p", "n_star", "flags"):
        assert np.array_equal(a[k], b[k]), k
    assert r2["cg_iters"] > r0["cg_iters"]      # from zero: more inner iterations


@pytest.mark.parametrize("precision", [0, 1])
def test_short_history_uses_the_lower_orders(precision):
    """With k solutions in the history the guess is of order min(k, cg_x0): the first two
    steps of cg_x0 = 2 are those of cg_x0 = 1, the first three of cg_x0 = 3 those of
    cg_x0 = 2 and the first four of cg_x0 = 4 those of cg_x0 = 3, bit for bit (the same
    weights over the same buffers); the next step differs."""
    sc = small_3d(seed=4)
    kw = dict(precision=precision, dt=5e-5)
    runs = {x0: _steps(sc, k, cg_x0=x0, **kw) for x0, k in ((1, 3), (2, 4), (3, 5), (4, 5))}
    for lo, hi, same in ((1, 2, 2), (2, 3, 3), (3, 4, 4)):
        a, b = runs[lo][0], runs[hi][0]
        for t in range(same):
            assert (a[t]["cg_iters"], a[t]["cg_resid"]) == (b[t]["cg_iters"], b[t]["cg_resid"]), (lo, hi, t)
    # one more step: the higher order changes the iterate path (not the solution's tolerance)
    a, b = runs[1][0][2], runs[2][0][2]
    assert a["cg_resid"] != b["cg_resid"]
