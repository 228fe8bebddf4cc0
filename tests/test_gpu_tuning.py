"""The tunable forms of the mixed PPE solve and the autotuner that picks them.

- The fused inner CG (inner_cg = 1: two kernels per iteration by the recurrences of
  Chronopoulos and Gear) and the 256-thread FP32 SpMV round differently from the defaults,
  so they are held to the mixed-precision bound against the FP64 oracle (p: relative L2 over
  fluid <= 1e-5, positions <= 1e-6 l0), on the regularised and on the stiff PPE, one scene
  and an ensemble, and must reach the same FP64 residual.
- The row build's block (64, 128 or 256 threads) changes nothing: every row is one thread's
  walk over its candidate list, so results are bit-identical.
- The cell side h = max(re)(1 + s) changes the candidates' order, not the neighbour sets:
  FP64 parity with the oracle at other cell skins.
- mps_autotune returns a valid choice with its times (cell side, gather block, build block,
  SpMV block, inner-CG form); a scene or an ensemble stepped after tuning keeps its
  tolerance and stays within the mixed bound of the oracle, and the grid in force is the one
  of the chosen cell skin."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import (FP64_TOL, PARITY_CG_TOL, gpu_params, oracle_params, rel_err, run_gpu,
                     run_oracle, small_3d)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    oracle.set_threads(0)


def _mixed_bound(sc, got, ref):
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ref.p[f]) / np.linalg.norm(ref.p[f])
    ex = np.abs(got["pos"] - ref.pos).max() / sc.l0
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex


@pytest.mark.parametrize("form", [dict(inner_cg=1), dict(spmv_block=256),
                                  dict(inner_cg=1, spmv_block=256)])
@pytest.mark.parametrize("case", ["2d", "3d", "2d-stiff"])
def test_tunable_forms_within_the_mixed_bound(case, form):
    if case == "2d":
        sc, kw = scenes.dam_break_2d(seed=1), {}
    elif case == "3d":
        sc, kw = small_3d(seed=2), dict(dt=5e-5)
    else:
        sc, kw = scenes.dam_break_2d(seed=3), dict(alpha_c=0.0, clamp_negative_p=0)
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=1, cg_tol=1e-8, cg_x0=0, **kw,
                                               **form))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **kw)
    assert rc == 0 and rep["cg_resid"] <= 1e-8
    _mixed_bound(sc, got, ost)
    assert np.array_equal(got["flags"], ost.flags)


def test_fused_cg_along_a_trajectory_with_the_guess():
    """Five steps of the 3D small dam break with the quadratic guess: the fused inner CG
    and the default reach the same residual and stay within the mixed bound of each other."""
    sc = small_3d(seed=4)
    outs = []
    for form in (0, 1):
        from paper_2105_01677_gb300 import mps
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, dt=5e-5, cg_x0=3, inner_cg=form))
        try:
            reps = [sim.step(1)[1] for _ in range(5)]
            outs.append((reps, sim.read()))
        finally:
            sim.close()
    (r0, s0), (r1, s1) = outs
    assert all(r["cg_resid"] <= 1e-8 for r in r0 + r1)
    f = sc.types == scenes.FLUID
    assert np.linalg.norm(s1["p"][f] - s0["p"][f]) / np.linalg.norm(s0["p"][f]) <= 1e-5
    assert np.abs(s1["pos"] - s0["pos"]).max() / sc.l0 <= 1e-6


def test_autotune_mixed_ensemble():
    from paper_2105_01677_gb300 import mps
    E = scenes.ensemble_2d(count=8, seed=9, fluid=(500, 3000))
    ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                       cg_tol=1e-8, cg_x0=3)
    try:
        ens.step(2)
        t = ens.autotune(2)
        assert t["gather_block"] in (32, 64, 96, 128)
        assert t["spmv_block"] in (256, 512)
        assert t["cg_fused"] in (0, 1) and t["cg_unroll"] in (1, 2, 4)
        assert t["predict_tpr"] in (1, 2, 4) and t["predict_ms"] > 0
        assert t["gather_ms"] > 0 and t["spmv_ms"] > 0 and t["solve_ms"] > 0
        assert t["build_block"] in (64, 128, 256) and t["build_ms"] > 0
        assert t["cell_skin"] in (0.1, 0.05, 0.15, 0.2) and t["cell_ms"] > 0
        for _ in range(3):
            rc, rep = ens.step(1)
            assert rc == 0 and rep["step_graph"] == 1
            assert np.all(ens.residuals() <= 1e-8)
        got = ens.read()
        before = [sc.copy() for sc in E]
    finally:
        ens.close()
    # every scene's state after tuning within the mixed bound of the oracle run on that scene
    # alone for the same five steps (two before tuning, three after)
    for k in (0, len(E) - 1):
        sc = E[k]
        prm = oracle_params(sc, dt=1e-4, cg_tol=PARITY_CG_TOL)
        st = oracle.State.from_scene(sc)
        for _ in range(5):
            oracle.step(prm, st)
        f = sc.types == scenes.FLUID
        ep = np.linalg.norm(got[k]["p"][f] - st.p[f]) / np.linalg.norm(st.p[f])
        ex = np.abs(got[k]["pos"] - st.pos).max() / sc.l0
        assert ep <= 1e-4, (k, ep)     # five steps of drift at the mixed bound
        assert ex <= 1e-6, (k, ex)
    del before


@pytest.mark.parametrize("bb", [64, 128, 256])
@pytest.mark.parametrize("case", ["2d-fp64", "3d-mixed", "3d-eos-mixed"])
def test_build_block_changes_nothing(case, bb):
    if case == "2d-fp64":
        sc, kw = scenes.dam_break_2d(seed=1), dict(precision=0)
    elif case == "3d-mixed":
        sc, kw = small_3d(seed=2), dict(precision=1, dt=5e-5)
    else:
        sc, kw = small_3d(seed=3), dict(precision=1, dt=5e-5, pressure_mode=1)
    outs = []
    for b in (0, bb):
        rc, rep, st, _ = run_gpu(sc, nsteps=2, **gpu_params(sc, cg_x0=0, build_block=b, **kw))
        assert rc == 0
        outs.append(st)
    for key in ("p", "n_star", "pos", "vel", "flags"):
        assert np.array_equal(outs[0][key], outs[1][key]), key


@pytest.mark.parametrize("skin", [0.05, 0.2])
def test_other_cell_side_fp64_parity(skin):
    sc = small_3d(seed=5)
    rc, rep, got, consts = run_gpu(sc, **gpu_params(sc, precision=0, cg_tol=PARITY_CG_TOL,
                                                     dt=5e-5, cell_skin=skin))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, dt=5e-5)
    assert rc == 0
    assert consts["h"] == pytest.approx(4.0 * sc.l0 * (1.0 + skin), rel=1e-12)
    for key, ref in (("p", ost.p), ("vel", ost.vel)):
        assert rel_err(got[key], ref) <= FP64_TOL, key
    assert np.array_equal(got["flags"], ost.flags)


def test_autotune_single_scene_cell_side_and_build_block():
    """Created with cell skin 0.3 (not among the tuner's own candidates, so the tuner derives
    other grids and comes back to one of them); the grid afterwards is that of the choice."""
    from paper_2105_01677_gb300 import mps
    sc = small_3d(seed=6)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, precision=1, dt=5e-5, cg_tol=1e-8, cg_x0=3,
                                      cell_skin=0.3))
    try:
        sim.step(2)
        t = sim.autotune(2)
        assert t["cell_skin"] in (0.3, 0.05, 0.1, 0.15, 0.2)
        assert t["build_block"] in (64, 128, 256)
        assert t["cell_ms"] > 0 and t["build_ms"] > 0 and t["gather_ms"] > 0
        c = sim.constants()
        assert c["h"] == pytest.approx(4.0 * sc.l0 * (1.0 + t["cell_skin"]), rel=1e-12)
        for _ in range(3):
            rc, rep = sim.step(1)
            assert rc == 0 and rep["cg_resid"] <= 1e-8
        got = sim.read()
    finally:
        sim.close()
    prm = oracle_params(sc, dt=5e-5, cg_tol=PARITY_CG_TOL)
    st = oracle.State.from_scene(sc)
    for _ in range(5):
        oracle.step(prm, st)
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - st.p[f]) / np.linalg.norm(st.p[f])
    ex = np.abs(got["pos"] - st.pos).max() / sc.l0
    assert ep <= 1e-4, ep
    assert ex <= 1e-6, ex


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("case", ["3d-guess", "2d-stiff"])
def test_cg_unroll_changes_nothing(case, fused):
    """Several inner CG iterations per pass of the device-driven loop: the iterations after
    convergence return at once, so every field and the iteration counts are bit-identical."""
    if case == "3d-guess":
        sc, kw = small_3d(seed=7), dict(dt=5e-5, cg_x0=3)
    else:
        sc, kw = scenes.dam_break_2d(seed=8), dict(alpha_c=0.0, clamp_negative_p=0, cg_x0=0)
    outs = []
    for u in (1, 2, 4):
        from paper_2105_01677_gb300 import mps
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, cg_tol=1e-8, inner_cg=fused,
                                          cg_unroll=u, **kw))
        try:
            reps = [sim.step(1)[1] for _ in range(3)]
            outs.append((reps, sim.read()))
        finally:
            sim.close()
    (r1, s1) = outs[0]
    for reps, st in outs[1:]:
        for key in ("p", "n_star", "pos", "vel", "flags"):
            assert np.array_equal(st[key], s1[key]), key
        for a, b in zip(reps, r1):
            assert a["cg_iters"] == b["cg_iters"] and a["cg_outer"] == b["cg_outer"]
            assert a["cg_resid"] == b["cg_resid"]


@pytest.mark.parametrize("tpr", [2, 4])
@pytest.mark.parametrize("case", ["2d-fp64", "3d-fp64", "3d-mixed", "ensemble-mixed"])
def test_prediction_threads_per_row_parity(case, tpr):
    """Two or four threads per FLUID row in the prediction: its viscosity sums are added in
    another order, so the step stays within the oracle parity bounds (FP64: 1e-10 relative;
    mixed: the mixed bound); neighbour sets, and so the flags, are unchanged."""
    from paper_2105_01677_gb300 import mps
    if case == "ensemble-mixed":
        E = scenes.ensemble_2d(count=4, seed=12, fluid=(500, 2000))
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                           cg_tol=1e-8, predict_tpr=tpr)
        try:
            rc, rep = ens.step(1)
            got = ens.read()
        finally:
            ens.close()
        assert rc == 0
        for k in (0, len(E) - 1):
            orep, ost, prm = run_oracle(E[k], dt=1e-4, cg_tol=PARITY_CG_TOL)
            _mixed_bound(E[k], got[k], ost)
            assert np.array_equal(got[k]["flags"], ost.flags)
        return
    if case == "2d-fp64":
        sc, kw = scenes.dam_break_2d(seed=1), dict(precision=0, dt=1e-4)
    elif case == "3d-fp64":
        sc, kw = small_3d(seed=2), dict(precision=0, dt=5e-5)
    else:
        sc, kw = small_3d(seed=3), dict(precision=1, dt=5e-5)
    tol = PARITY_CG_TOL if kw["precision"] == 0 else 1e-8
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, cg_tol=tol, predict_tpr=tpr, **kw))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, dt=kw["dt"])
    assert rc == 0
    if kw["precision"] == 0:
        for key, ref in (("p", ost.p), ("vel", ost.vel)):
            assert rel_err(got[key], ref) <= FP64_TOL, key
    else:
        _mixed_bound(sc, got, ost)
    assert np.array_equal(got["flags"], ost.flags)
