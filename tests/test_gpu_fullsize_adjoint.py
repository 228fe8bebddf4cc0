"""The reverse step at full size: the 3D sloshing tank (85,564 particles, l0 = 0.008 m) under
its tank-frame forcing, FP64, in the configuration the bench times (dt 5e-5 s).

Parity: the oracle's reverse step at the same state, every cotangent compared (the state is
the oracle's own, five oracle steps into the forcing, so nothing the oracle sees comes from
the CUDA path).  Central differences are checked on the equation-of-state path only: the PPE
path's p_hat_i = min_j p_j has kinks wherever neighbours at one depth share nearly the same
hydrostatic pressure, and at this size a finite-difference step crosses some of them; the
equation-of-state path has no minimum and is smooth in the velocities."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

DT = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _forcing(t):
    return (float(scenes.sloshing_forcing(t * DT)), 0.0, -9.81)


@pytest.fixture(scope="module")
def sloshing_state():
    sc = scenes.sloshing_3d()
    assert sc.n == 85564
    st = oracle.State.from_scene(sc)
    for t in range(5):
        oracle.step(oracle_params(sc, dt=DT, cg_tol=1e-13, g=_forcing(t)), st)
    s = sc.copy()
    s.pos, s.vel, s.types = st.pos.copy(), st.vel.copy(), st.types.copy()
    return s


def _sim(sc, **kw):
    from paper_2105_01677_gb300 import mps
    return mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, **kw))


def test_sloshing_vjp_matches_oracle_full_size(sloshing_state):
    sc = sloshing_state
    kw = dict(dt=DT, cg_tol=1e-13, g=_forcing(5))
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal(sc.pos.shape), rng.standard_normal(sc.vel.shape)
    sim = _sim(sc, **kw)
    try:
        rc, gr, gu, gg, rep = sim.step_vjp(a, b)
        _, gr2, gu2, _, _ = sim.step_vjp(2.0 * a, 2.0 * b)
    finally:
        sim.close()
    assert rep["cg_resid"] <= 1e-13 and rep["forward"]["n_ppe_rows"] > 0
    ogr, ogu, ogg = oracle.step_vjp(oracle_params(sc, **kw), oracle.State.from_scene(sc), a, b)
    for name, val, ref in (("dL/dr", gr, ogr), ("dL/du", gu, ogu), ("dL/dg", gg, ogg)):
        err = np.abs(val - ref).max() / np.abs(ref).max()
        assert err <= 1e-8, (name, err)
    # linear in the cotangent
    assert np.abs(gr2 - 2.0 * gr).max() <= 1e-9 * np.abs(gr).max()
    assert np.abs(gu2 - 2.0 * gu).max() <= 1e-9 * np.abs(gu).max()


def test_sloshing_eos_vjp_matches_central_differences(sloshing_state):
    sc = sloshing_state
    kw = dict(dt=DT, pressure_mode=1, c0=20.0, g=_forcing(5))
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(sc.pos.shape), rng.standard_normal(sc.vel.shape)
    v = rng.standard_normal(sc.vel.shape)
    h = 1e-6
    sim = _sim(sc, **kw)
    try:
        outs = []
        for sgn in (1.0, -1.0):
            sim.write(sc.pos, sc.vel + sgn * h * v, sc.types)
            sim.step(1)
            s = sim.read(want=("pos", "vel"))
            outs.append((s["pos"], s["vel"]))
        sim.write(sc.pos, sc.vel, sc.types)
        _, gr, gu, _, _ = sim.step_vjp(a, b)
    finally:
        sim.close()
    fd = float(((outs[0][0] - outs[1][0]) * a + (outs[0][1] - outs[1][1]) * b).sum()) / (2 * h)
    adj = float((gu * v).sum())
    assert abs(fd - adj) <= 1e-6 * abs(adj), (fd, adj)
