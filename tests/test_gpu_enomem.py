"""MPS_ENOMEM from the host side: the PyTorch allocator shim of the binding is given a byte
budget beyond which an allocation fails (returns NULL, as a full device would).  No GPU
fault is involved: the library sees a failed allocation hook and must report MPS_ENOMEM,
release whatever it had allocated, and leave a context that exists usable."""
import ctypes as C

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


def _create(sc, limit):
    """mps_create through the C ABI with a budgeted allocator; returns (rc, handle, shim)."""
    import torch
    from paper_2105_01677_gb300 import mps
    params = mps.mps_params_default(**gpu_params(sc))
    params.stream = C.c_void_p(torch.cuda.current_stream(0).cuda_stream)
    shim = mps._TorchAllocator(0, params.stream, limit)
    params.alloc = shim.alloc
    params.release = shim.release
    h = C.c_void_p()
    pos = np.ascontiguousarray(sc.pos)
    vel = np.ascontiguousarray(sc.vel)
    typ = np.ascontiguousarray(sc.types)
    rc = mps.lib().mps_create(pos.ctypes.data_as(C.POINTER(C.c_double)),
                              vel.ctypes.data_as(C.POINTER(C.c_double)),
                              typ.ctypes.data_as(C.POINTER(C.c_int8)), sc.n, C.byref(params),
                              C.byref(h))
    return rc, h, shim, params


def test_create_reports_enomem_and_releases_everything():
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    for limit in (0, 4096, 1 << 20):
        rc, h, shim, _ = _create(sc, limit)
        assert rc == mps.ENOMEM, (limit, rc)
        assert shim.live_bytes() == 0, limit           # every block handed back
    rc, h, shim, params = _create(sc, None)             # no budget: fine
    assert rc == mps.OK
    assert shim.live_bytes() > 0
    mps.mps_destroy(h)
    assert shim.live_bytes() == 0


def test_later_allocations_report_enomem_and_the_context_stays_usable():
    """A budget just above what the context needs: the step runs; the reverse step's and
    the two-phase properties' buffers do not fit (MPS_ENOMEM); stepping still works."""
    from paper_2105_01677_gb300 import mps
    sc = scenes.dam_break_2d(seed=1)
    rc, h, shim, params = _create(sc, None)
    assert rc == mps.OK
    need = shim.live_bytes()
    mps.mps_destroy(h)

    rc, h, shim, params = _create(sc, need + 4096)
    assert rc == mps.OK
    try:
        rep = mps.mps_report()
        assert mps.lib().mps_step(h, 1, C.byref(rep)) == mps.OK
        g = np.zeros((sc.n, 2))
        rc, *_ = mps.mps_step_vjp(h, g, g, check=False)
        assert rc == mps.ENOMEM
        rho = np.full(sc.n, 1000.0)
        assert mps.mps_set_fluid_properties(h, rho, None, check=False) == mps.ENOMEM
        assert mps.lib().mps_step(h, 2, C.byref(rep)) == mps.OK
        assert rep.status == mps.OK and rep.cg_resid <= 1e-8
    finally:
        mps.mps_destroy(h)
    assert shim.live_bytes() == 0
