"""Candidate lists gathered every step use a skin sized from the last step's motion (the
grid keeps the full skin).  A step whose predicted motion exceeds that skin is gathered
again with the full skin, so the neighbour sets, and the results, match the oracle either
way."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import PARITY_CG_TOL, compare_step, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def test_sudden_motion_after_rest_regathers_with_the_full_skin():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    kw = dict(cg_tol=PARITY_CG_TOL)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, **kw))
    try:
        sim.step(3)                       # near rest: the list skin shrinks to its minimum
        st = sim.read()
        fast = st["vel"].copy()
        f = st["types"] == scenes.FLUID
        fast[f] += [6.0, 0.0]             # 6e-4 m per step, beyond the shrunk skin (4e-4 m)
        sim.write(st["pos"], fast, st["types"])
        sim.step(1)
        got = sim.read()
    finally:
        sim.close()
    ref = scenes.Scene(2, sc.l0, st["pos"], fast, st["types"], sc.box_min, sc.box_max)
    prm = oracle_params(ref, **kw)
    ost = oracle.State.from_scene(ref)
    oracle.step(prm, ost)
    compare_step(ref, got, ost, prm)
