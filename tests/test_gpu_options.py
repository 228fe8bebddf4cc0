"""The paper's numerical options on the GPU against the oracle: the cubic weight of the
equation-of-state path (Sec. 3.1), the CMPS gradient (Eq. 18), the HS source (Eq. 21) and
the error-compensating source (Eq. 24-25), alone and combined, FP64 to the single-step
bound and mixed precision to its bound."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import PARITY_CG_TOL, compare_step, gpu_params, run_gpu, run_oracle, small_3d

pytestmark = pytest.mark.gpu

OPTIONS = [
    dict(kernel=1, pressure_mode=1, c0=20.0),
    dict(kernel=1, pressure_mode=0),
    dict(gradient_form=1, pressure_mode=0),
    dict(gradient_form=1, pressure_mode=1, c0=20.0),
    dict(source_term=1, pressure_mode=0),
    dict(source_term=1, gradient_form=1, pressure_mode=0),
    dict(kernel=1, gradient_form=1, pressure_mode=1, c0=20.0),
    dict(source_term=2, pressure_mode=0),
    dict(source_term=2, gradient_form=1, pressure_mode=0),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _oracle_kw(opt):
    kw = dict(opt)
    kw["grad_form"] = kw.pop("gradient_form", 0)
    kw["source"] = kw.pop("source_term", 0)
    return kw


def _moving(sc):
    """A smooth velocity field on the fluid, so that the HS source is not trivially zero."""
    sc = sc.copy()
    f = sc.types == scenes.FLUID
    x = sc.pos[:, 0]
    y = sc.pos[:, 1]
    sc.vel[f, 0] = 0.2 * np.sin(9.0 * y[f])
    sc.vel[f, 1] = 0.1 * np.cos(7.0 * x[f])
    return sc


@pytest.mark.parametrize("opt", OPTIONS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_option_fp64_2d(opt):
    sc = _moving(scenes.dam_break_2d(seed=1))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, cg_tol=PARITY_CG_TOL, **opt))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **_oracle_kw(opt))
    assert rep["n_ppe_rows"] == orep["n_ppe_rows"]
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("opt", OPTIONS[:3] + OPTIONS[4:5] + OPTIONS[7:8],
                         ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_option_fp64_3d_small(opt):
    sc = _moving(small_3d(seed=2))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, cg_tol=PARITY_CG_TOL, **opt))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **_oracle_kw(opt))
    compare_step(sc, got, ost, prm)


@pytest.mark.parametrize("opt", OPTIONS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_option_mixed_bound_3d_small(opt):
    sc = _moving(small_3d(seed=1))
    rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, precision=1, **opt))
    orep, ost, prm = run_oracle(sc, cg_tol=PARITY_CG_TOL, **_oracle_kw(opt))
    f = sc.types == scenes.FLUID
    ep = np.linalg.norm(got["p"][f] - ost.p[f]) / np.linalg.norm(ost.p[f])
    ex = np.abs(got["pos"] - ost.pos).max() / sc.l0
    assert ep <= 1e-5, ep
    assert ex <= 1e-6, ex
    assert np.array_equal(got["flags"], ost.flags)


def test_cmps_conserves_momentum_on_gpu():
    """Equation of state, CMPS, no gravity, an isolated fluid block: the pressure forces sum
    to zero, so the total momentum of the fluid stays where the viscosity leaves it."""
    from test_oracle_pins import lattice_block
    pos, t = lattice_block(2, 24, spacing=0.0098)   # compressed: positive pressure
    pos = pos + 0.1
    u = scenes.splitmix_uniform(5, np.arange(pos.size, dtype=np.uint64)).reshape(pos.shape)
    pos = pos + (u - 0.5) * 2e-4
    sc = scenes.Scene(2, 0.01, pos, np.zeros_like(pos), t, np.zeros(3), np.array([0.5, 0.5, 0.0]))
    mom = {}
    for form in (0, 1):
        rc, rep, got, _ = run_gpu(sc, **gpu_params(sc, pressure_mode=1, c0=20.0, nu=0.0,
                                                   g=(0.0, 0.0, 0.0), gradient_form=form))
        mom[form] = np.abs(got["vel"].sum(0)).max() / np.abs(got["vel"]).sum()
    assert mom[1] <= 1e-12
    assert mom[0] > 1e-6


def test_hs_rejects_cubic_kernel():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    with pytest.raises(mps.MPSError):
        mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, source_term=1, kernel=1))
