"""The device-driven mixed PPE solve (one CUDA graph with conditional WHILE nodes for the
refinement sweeps and the inner FP32 CG) against the host-driven loop over the same
kernels: identical results bit for bit, identical iteration counts, the same error when the
iteration cap is hit, and a context that stays usable afterwards."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import gpu_params, small_3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _run(sc, nsteps, host_loop, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, precision=1, ppe_host_loop=host_loop, **kw))
    try:
        reps = [sim.step(1)[1] for _ in range(nsteps)]
        st = sim.read()
    finally:
        sim.close()
    return reps, st


@pytest.mark.parametrize("scene,nsteps,kw", [
    ("2d", 6, dict(cg_tol=1e-8)),
    ("2d", 3, dict(cg_tol=1e-11)),
    ("3d", 3, dict(cg_tol=1e-8, dt=5e-5)),
    ("3d-free", 2, dict(cg_tol=1e-8, dt=5e-5, ppe_operator=1)),
])
def test_graph_solve_equals_host_loop(scene, nsteps, kw):
    sc = scenes.dam_break_2d(seed=3) if scene == "2d" else small_3d(seed=2)
    r_graph, s_graph = _run(sc, nsteps, 0, **kw)
    r_host, s_host = _run(sc, nsteps, 1, **kw)
    for a, b in zip(r_graph, r_host):
        assert (a["cg_iters"], a["cg_outer"]) == (b["cg_iters"], b["cg_outer"])
        assert a["cg_resid"] == b["cg_resid"]
    for k in ("pos", "vel", "p", "n_star", "flags", "types"):
        assert np.array_equal(s_graph[k], s_host[k]), k


def test_graph_solve_iteration_cap_and_recovery():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=4)
    for host_loop in (0, 1):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, ppe_host_loop=host_loop, cg_tol=1e-12,
                                          cg_max_iter=3))
        try:
            rc, rep = sim.step(1, check=False)
            assert rc == mps.ECG_NOCONV
            assert rep["cg_iters"] <= 3 and rep["cg_resid"] > 1e-12
        finally:
            sim.close()
    # a converging solve on a fresh context after a capped one
    reps, st = _run(sc, 2, 0, cg_tol=1e-8)
    assert all(r["cg_resid"] <= 1e-8 for r in reps)
    assert np.all(np.isfinite(st["p"]))


def test_time_kernel_leaves_the_state_and_counts_bytes():
    from paper_2105_01677_gb300 import mps
    sc = small_3d(seed=3)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, precision=1, dt=5e-5))
    try:
        rc, rep = sim.step(1)
        before = sim.read()
        ms, by = mps.mps_time_kernel(sim.h, mps.KERNEL_SPMV32, 3)
        ms2, by2 = mps.mps_time_kernel(sim.h, mps.KERNEL_RESID_FF, 2)
        after = sim.read()
        with pytest.raises(mps.MPSError):
            mps.mps_time_kernel(sim.h, mps.KERNEL_SPMV64, 1)   # FP64 kernel of a mixed context
        sim.step(1)                                           # still steps afterwards
    finally:
        sim.close()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    # 8 bytes per stored coefficient of the system's rows (free-surface rows, whose
    # coefficients are stored but not in the system, are a large share of this small scene),
    # 12 for the float-float residual
    assert ms > 0 and ms2 > 0
    assert 8 * rep["pairs_ppe"] * 0.4 <= by <= 8 * rep["pairs_ppe"] + 12 * sc.n
    assert abs(by2 / by - 1.5) < 0.1


def test_graph_solve_equals_host_loop_ensemble():
    """An ensemble's per-scene convergence decided on the device inside the graph: the
    same sweeps, iterations, per-scene residuals and states as the host-driven loop."""
    from paper_2105_01677_gb300 import mps
    E = scenes.ensemble_2d(count=6, seed=4, fluid=(150, 1500))
    out = []
    for host_loop in (0, 1):
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1,
                           cg_tol=1e-9, ppe_host_loop=host_loop)
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
