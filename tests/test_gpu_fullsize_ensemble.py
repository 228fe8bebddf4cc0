"""Parity at the ensemble workload's full size: the 256 seeded 2D dam breaks of the bench
(3,355,770 particles, l0 0.005-0.01 m, dt = 1e-4) stepped together in one context, FP64
and mixed; a sample of scenes (the largest, the smallest and six drawn by index) is
compared with the oracle run on each scene alone."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import PARITY_CG_TOL, compare_step, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ensemble():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    E = scenes.ensemble_2d(count=256, seed=1)
    sizes = np.array([sc.n for sc in E])
    sample = sorted({int(sizes.argmax()), int(sizes.argmin()), 3, 57, 101, 150, 199, 255})
    return E, sample


def _run(E, **kw):
    from paper_2105_01677_gb300 import mps
    ens = mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, dt=1e-4, **kw)
    try:
        ens.autotune(1)
        rc, rep = ens.step(1)
        return rep, ens.read(), ens.residuals()
    finally:
        ens.close()


def _oracle(sc, **kw):
    prm = oracle_params(sc, dt=1e-4, **kw)
    st = oracle.State.from_scene(sc)
    oracle.step(prm, st)
    return prm, st


def test_fullsize_ensemble_fp64_sampled_scenes(ensemble):
    E, sample = ensemble
    rep, got, res = _run(E, cg_tol=PARITY_CG_TOL)
    assert np.all(res <= PARITY_CG_TOL)
    for s in sample:
        prm, ost = _oracle(E[s], cg_tol=PARITY_CG_TOL)
        compare_step(E[s], got[s], ost, prm)


def test_fullsize_ensemble_mixed_sampled_scenes(ensemble):
    E, sample = ensemble
    rep, got, res = _run(E, precision=1, cg_tol=1e-8)
    assert np.all(res <= 1e-8)
    for s in sample:
        sc = E[s]
        prm, ost = _oracle(sc, cg_tol=PARITY_CG_TOL)
        f = sc.types == scenes.FLUID
        ep = np.linalg.norm(got[s]["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
        assert ep <= 1e-5, (s, ep)
        assert np.abs(got[s]["pos"] - ost.pos).max() / sc.l0 <= 1e-6
        assert np.array_equal(got[s]["flags"], ost.flags)
