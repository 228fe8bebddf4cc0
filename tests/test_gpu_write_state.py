"""mps_write_state validates the uploaded state on the device: non-finite values or unknown
kinds are rejected with the context's state left as it was."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def test_invalid_upload_is_rejected_and_state_kept():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    sim = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, cg_tol=1e-10))
    ref = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, cg_tol=1e-10))
    try:
        bad = sc.pos.copy()
        bad[7, 1] = np.nan
        L = mps.lib()
        for pos, vel, types, expect in (
                (bad, sc.vel, sc.types, mps.ENONFINITE),
                (sc.pos, np.where(np.arange(sc.n)[:, None] == 3, np.inf, sc.vel), sc.types,
                 mps.ENONFINITE),
                (sc.pos, sc.vel, np.where(np.arange(sc.n) == 5, 9, sc.types).astype(np.int8),
                 mps.EINVAL)):
            pos = np.ascontiguousarray(pos, np.float64)
            vel = np.ascontiguousarray(vel, np.float64)
            types = np.ascontiguousarray(types, np.int8)
            rc = L.mps_write_state(sim.h, mps._ptr(pos, mps.C.c_double),
                                   mps._ptr(vel, mps.C.c_double), mps._ptr(types, mps.C.c_int8))
            assert rc == expect, mps.mps_strerror(rc)
        sim.step(2)
        ref.step(2)
        a, b = sim.read(), ref.read()
        for k in ("pos", "vel", "p", "n_star", "flags", "types"):
            assert np.array_equal(a[k], b[k]), k
    finally:
        sim.close()
        ref.close()
