"""Whole steps as one CUDA graph (step_graph = 1, the default) against the same steps launched
one by one (step_graph = 0; 2 launches the bucket build kernel by kernel as well): the
kernels are the same, so every field must agree bit for bit, over several steps (which
exercises both state-buffer parities of the graph, the guess history and the adaptive list
skin), for one scene and for an ensemble, on the mixed PPE path and the equation-of-state
path; the retry with the full skin, MPS_ESKIN and the device errors must come out as on the
host-driven path. The parity of either path with the oracle is covered by the other GPU
tests, which run the graph by default."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import gpu_params, small_3d

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "vel", "p", "n_star", "flags", "types")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _run(sc, steps, step_graph, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, step_graph=step_graph, **kw))
    reps, states = [], []
    try:
        for _ in range(steps):
            rc, rep = sim.step(1)
            reps.append(rep)
            states.append(sim.read())
    finally:
        sim.close()
    return reps, states


def _same(a, b):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("case", ["2d-mixed", "3d-mixed-guess", "2d-eos-mixed", "3d-eos-fp64",
                                  "2d-mixed-two-phase"])
def test_step_graph_equals_launch_by_launch(case):
    kw = {}
    rho_i = nu_i = None
    if case == "2d-mixed":
        sc, kw = scenes.dam_break_2d(seed=1), dict(precision=1)
    elif case == "3d-mixed-guess":
        sc, kw = small_3d(seed=2), dict(precision=1, dt=5e-5, cg_x0=3)
    elif case == "2d-eos-mixed":
        sc, kw = scenes.dam_break_2d(seed=3), dict(precision=1, pressure_mode=1, c0=20.0)
    elif case == "3d-eos-fp64":
        sc, kw = small_3d(seed=4), dict(precision=0, pressure_mode=1, c0=20.0, dt=5e-5)
    else:
        sc = scenes.dam_break_2d(seed=5)
        kw = dict(precision=1, cg_x0=2)
    if case == "2d-mixed-two-phase":
        rho_i, nu_i = scenes.two_phase(sc, rho=(1000.0, 800.0), nu=(1e-6, 5e-6))
        kw.update(rho_i=rho_i, nu_i=nu_i)
    rg, sg = _run(sc, 6, 1, **kw)
    rh, sh = _run(sc, 6, 0, **kw)
    # step_graph = 2: the bucket build launched kernel by kernel too (its radix sort every step)
    rn, sn = _run(sc, 6, 2, **kw)
    assert all(r["step_graph"] == 1 for r in rg)
    assert all(r["step_graph"] == 0 for r in rh + rn)
    for k in range(6):
        _same(sg[k], sh[k])
        _same(sg[k], sn[k])
        for f in ("cg_iters", "cg_outer", "cg_resid", "n_surface", "n_ppe_rows", "max_disp",
                  "cand_tests", "pairs_ppe", "pairs_pnd", "list_tests"):
            assert rg[k][f] == rh[k][f] == rn[k][f], (k, f)


@pytest.mark.parametrize("list_every", [1, 3])
def test_step_graph_ensemble_equals_launch_by_launch(list_every):
    from paper_2105_01677_gb300 import mps
    E = scenes.ensemble_2d(count=12, seed=3, fluid=(500, 3000))
    out = []
    nsteps = 5 if list_every == 1 else 8
    for sgflag in (1, 0):
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                           cg_tol=1e-8, cg_x0=3, step_graph=sgflag, list_every=list_every)
        try:
            reps, states, res = [], [], []
            for _ in range(nsteps):
                rc, rep = ens.step(1)
                reps.append(rep)
                states.append(ens.read())
                res.append(ens.residuals())
        finally:
            ens.close()
        out.append((reps, states, res))
    (rg, sg, qg), (rh, sh, qh) = out
    assert all(r["step_graph"] == 1 for r in rg) and all(r["step_graph"] == 0 for r in rh)
    assert [r["list_gathered"] for r in rg] == [r["list_gathered"] for r in rh]
    if list_every > 1:
        assert 0 in [r["list_gathered"] for r in rg]
    for k in range(nsteps):
        assert np.array_equal(qg[k], qh[k])
        assert rg[k]["cg_iters"] == rh[k]["cg_iters"]
        for a, b in zip(sg[k], sh[k]):
            _same(a, b)


def test_step_graph_retries_with_the_full_skin():
    """A calm first step leaves a small adaptive list skin; the state is then given velocities
    that move particles beyond it but within the full cell skin: both paths gather again with
    the full skin, and agree bit for bit."""
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=6)
    f = sc.types == scenes.FLUID
    rng = np.random.default_rng(7)
    kick = np.zeros_like(sc.vel)
    # up to 1.4 mm in one 1e-4 s step: past half a list skin of 0.02 (0.4 mm at
    # re = 0.04 m), within half the full skin of 0.1 (2 mm)
    kick[f] = rng.uniform(-1.0, 1.0, size=(int(f.sum()), 2)) * 10.0
    states = []
    for sgflag in (1, 0):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, step_graph=sgflag))
        try:
            sim.step(2)
            st = sim.read()
            sim.write(st["pos"], kick, st["types"])
            rc, rep = sim.step(1)
            assert rc == 0 and rep["max_disp"] > 0.4e-3, rep["max_disp"]
            states.append(sim.read())
        finally:
            sim.close()
    _same(states[0], states[1])


def test_step_graph_reports_skin_and_coincidence_errors():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=8)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    fast = sc.copy()
    fast.vel[f[:65]] = [300.0, 0.0]    # 65 particles beyond the skin: more than the direct
                                       # search completes (max(64, n/256))
    coinc = sc.copy()
    coinc.pos[f[1]] = coinc.pos[f[0]]
    for sgflag in (1, 0):
        for scene, code in ((fast, mps.ESKIN), (coinc, mps.ECOINCIDENT)):
            sim = mps.Simulation(scene, torch_alloc=True, use_torch_stream=True,
                                 **gpu_params(scene, precision=1, step_graph=sgflag))
            try:
                rc, rep = sim.step(1, check=False)
                assert rc == code, (sgflag, rc, code)
            finally:
                sim.close()


@pytest.mark.parametrize("case", ["3d-mixed-kept", "2d-eos-kept", "2d-mixed-kept-fast"])
def test_step_graph_kept_lists_equals_launch_by_launch(case):
    """Candidate lists kept across steps (list_every > 1): the steps on kept lists run a graph
    without bucket build and gather, those whose lists are due the full graph; a kept step
    whose lists fall short (fluid at 4 m/s against a skin of 0.05) is taken again on fresh
    lists.  Every field, and which steps gathered, as launched one by one."""
    if case == "3d-mixed-kept":
        sc, kw = small_3d(seed=5), dict(precision=1, dt=5e-5, cg_x0=3, list_every=4)
    elif case == "2d-eos-kept":
        sc, kw = scenes.dam_break_2d(seed=6), dict(precision=1, pressure_mode=1, c0=20.0,
                                                   list_every=4)
    else:
        sc = scenes.dam_break_2d(seed=1)
        f = sc.types == scenes.FLUID
        sc.vel[f] = [4.0, 0.0]
        kw = dict(precision=1, cell_skin=0.05, list_every=10)
    steps = 10
    rg, sg = _run(sc, steps, 1, **kw)
    rh, sh = _run(sc, steps, 0, **kw)
    assert all(r["step_graph"] == 1 for r in rg)
    gathered = [r["list_gathered"] for r in rg]
    assert gathered == [r["list_gathered"] for r in rh]
    assert 0 in gathered and gathered.count(1) >= 2
    if case == "2d-mixed-kept-fast":
        assert gathered[:5] == [1, 0, 1, 0, 1], gathered
    for k in range(steps):
        _same(sg[k], sh[k])
        for f in ("cg_iters", "cg_outer", "cg_resid", "n_surface", "n_ppe_rows", "max_disp",
                  "pairs_ppe", "pairs_pnd", "list_tests", "bucket_merged"):
            assert rg[k][f] == rh[k][f], (k, f)
