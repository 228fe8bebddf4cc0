"""Batched ensembles of independent scenes in one context against the oracle run on each
scene alone: seeded 2D dam breaks of different sizes, aspects and particle spacings."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import PARITY_CG_TOL, compare_step, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _ensemble(count=6, seed=4):
    return scenes.ensemble_2d(count=count, seed=seed, fluid=(150, 1500))


def _run(scene_list, nsteps=1, **kw):
    from paper_2105_01677_gb300 import mps
    ens = mps.Ensemble(scene_list, torch_alloc=True, use_torch_stream=True, **kw)
    try:
        rc, rep = ens.step(nsteps)
        got = ens.read()
        res = ens.residuals()
    finally:
        ens.close()
    return rep, got, res


def _oracle(sc, nsteps=1, **kw):
    prm = oracle_params(sc, **kw)
    st = oracle.State.from_scene(sc)
    for _ in range(nsteps):
        oracle.step(prm, st)
    return prm, st


@pytest.mark.parametrize("mode", [0, 1])
def test_ensemble_fp64_each_scene_matches_oracle(mode):
    E = _ensemble()
    assert len({sc.l0 for sc in E}) == len(E)          # every scene has its own spacing
    kw = dict(pressure_mode=mode, cg_tol=PARITY_CG_TOL)
    rep, got, res = _run(E, **kw)
    for sc, g in zip(E, got):
        prm, ost = _oracle(sc, **kw)
        compare_step(sc, g, ost, prm)
    if mode == 0:
        assert np.all(res <= PARITY_CG_TOL) and res.max() > 0


def test_ensemble_mixed_bound_per_scene():
    E = _ensemble(seed=5)
    rep, got, res = _run(E, precision=1, cg_tol=1e-8)
    assert np.all(res <= 1e-8)
    assert rep["cg_resid"] == pytest.approx(res.max())
    for sc, g in zip(E, got):
        prm, ost = _oracle(sc, cg_tol=PARITY_CG_TOL)
        f = sc.types == scenes.FLUID
        ep = np.linalg.norm(g["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
        assert ep <= 1e-5, ep
        assert np.abs(g["pos"] - ost.pos).max() / sc.l0 <= 1e-6
        assert np.array_equal(g["flags"], ost.flags)


def test_ensemble_of_one_equals_single_context():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=2)
    rep1, got1, _ = _run([sc], nsteps=3, cg_tol=1e-10)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, cg_tol=1e-10)
    try:
        sim.step(3)
        got = sim.read()
    finally:
        sim.close()
    for k in ("pos", "vel", "p", "n_star", "flags", "types"):
        assert np.array_equal(got1[0][k], got[k]), k


def test_ensemble_scenes_do_not_interact_and_ghosts_per_scene():
    """Two scenes in overlapping coordinates (both tanks start at the origin): a particle
    sitting inside the other scene's grid but outside its own becomes a GHOST, as the oracle
    of its own scene decides, and neither scene sees the other's particles."""
    a = scenes.tank_scene(2, 0.01, (120, 50), (20, 40), seed=1)
    b = scenes.dam_break_2d(seed=2, l0=0.008).copy()
    hb = 4.0 * b.l0 * 1.1
    b_end = b.box_min[0] + (np.floor((b.box_max[0] - b.box_min[0]) / hb) + 1) * hb
    far = 1.0
    assert b_end < far < a.box_max[0]   # outside b's own grid, inside a's
    b.pos[0] = [far, 0.3]
    kw = dict(cg_tol=PARITY_CG_TOL)
    rep, got, res = _run([a, b], **kw)
    for sc, g in zip((a, b), got):
        prm, ost = _oracle(sc, **kw)
        compare_step(sc, g, ost, prm)
    assert got[1]["types"][0] == scenes.GHOST


def _degenerate_scenes():
    """A normal dam break beside a lone particle, the tank without its fluid, a compressed
    fluid block without walls and a scene whose particles are all GHOST."""
    l0 = 0.01
    normal = scenes.dam_break_2d(seed=3)
    lone = scenes.Scene(2, l0, np.array([[0.3, 0.3]]), np.array([[0.2, -0.1]]),
                        np.zeros(1, np.int8), np.zeros(3), np.array([1.0, 1.0, 0.0]))
    full = scenes.dam_break_2d(seed=1)
    keep = full.types != scenes.FLUID
    walls = scenes.Scene(2, l0, full.pos[keep].copy(), full.vel[keep].copy(),
                         full.types[keep].copy(), full.box_min, full.box_max)
    g = np.meshgrid(np.arange(20), np.arange(12), indexing="ij")
    blk = np.stack([a.reshape(-1) for a in g], axis=1).astype(np.float64) * (0.98 * l0) + 0.2
    block = scenes.Scene(2, l0, blk, np.zeros_like(blk), np.zeros(len(blk), np.int8),
                         np.zeros(3), np.array([1.0, 1.0, 0.0]))
    ghosts = scenes.dam_break_2d(seed=5)
    ghosts.types[:] = scenes.GHOST
    return [normal, lone, walls, block, ghosts]


@pytest.mark.parametrize("precision", [0, 1])
def test_ensemble_with_degenerate_scenes(precision):
    """Each scene of the ensemble matches the oracle of that scene alone, and each PPE is
    solved to its own tolerance, whether it has rows with a nonzero right-hand side (the
    dam break, the wall-less block), rows with a negative one (the walls), or none at all
    (the lone particle, the GHOST scene)."""
    E = _degenerate_scenes()
    tol = PARITY_CG_TOL if precision == 0 else 1e-8
    rep, got, res = _run(E, precision=precision, cg_tol=tol)
    assert np.all(res <= tol)
    for k, (sc, g) in enumerate(zip(E, got)):
        prm, ost = _oracle(sc, cg_tol=PARITY_CG_TOL)
        if k == 4:
            assert np.array_equal(g["pos"], sc.pos) and np.all(g["types"] == scenes.GHOST)
            continue
        if precision == 0:
            compare_step(sc, g, ost, prm)
            continue
        f = sc.types == scenes.FLUID
        if ost.p[f].size and np.linalg.norm(ost.p[f]) > 0:
            ep = np.linalg.norm(g["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
            assert ep <= 1e-5, (k, ep)
        assert np.abs(g["pos"] - ost.pos).max() / sc.l0 <= 1e-6, k
        assert np.array_equal(g["flags"], ost.flags), k


def test_ensemble_multi_step_mixed_runs_and_converges():
    E = _ensemble(count=12, seed=6)
    rep, got, res = _run(E, nsteps=10, precision=1, cg_tol=1e-8)
    assert rep["steps_done"] == 10 and np.all(res <= 1e-8)
    for g in got:
        assert np.all(np.isfinite(g["pos"])) and np.all(np.isfinite(g["p"]))


def test_autotune_keeps_results_bitwise():
    """On the FP64 path the tuned launch shapes (gather block, build block) change no bit;
    the prediction's threads per row change the order of its sums, so the untuned run takes
    the tuner's choice of those."""
    from paper_2105_01677_gb300 import mps
    E = _ensemble(count=4, seed=7)
    outs = []
    tpr = 1
    for tune in (True, False):
        ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, cg_tol=1e-10,
                           predict_tpr=tpr)
        try:
            if tune:
                t = ens.autotune(2)
                assert t["gather_block"] in (32, 64, 96, 128)
                tpr = t["predict_tpr"]
            ens.step(2)
            outs.append(ens.read())
        finally:
            ens.close()
    for a, b in zip(*outs):
        for k in ("pos", "vel", "p", "n_star", "flags"):
            assert np.array_equal(a[k], b[k]), k
