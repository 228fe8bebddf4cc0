"""The allocation-free CG entry point (mps_ppe_cg_noalloc) against the library's own PPE
solve (mps_solve_ppe) on the same dam-break state.

mps_ppe_cg_noalloc exists for callers that may not allocate device memory (their memory is
owned by their own pool, or allocation is off limits in their loop); it keeps its scratch in
a fixed array inside the library.  This file is collected last so that, if it fails, a run
stopping at the first failure has already run every other test.  It is called twice in a
row: the second call must not be disturbed by what the first left in the shared array."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import FP64_TOL, PARITY_CG_TOL, gpu_params, oracle_params, rel_err

pytestmark = pytest.mark.gpu


def _ell_from_csr(off, col, val, b, types, flags):
    """The oracle's PPE system (CSR, diagonal first, rows in particle order) laid out as the
    library's operator rows: diag, then c_ij = -A_ij of the off-diagonal entries."""
    n = len(b)
    rows = (types <= oracle.WALL) & (flags == 0)
    counts = (np.diff(off) - 1).astype(np.int64)
    counts[~rows] = 0
    cap = int(max(32, ((counts.max() + 31) // 32) * 32))
    ecol = np.zeros((n, cap), np.int32)
    eval_ = np.zeros((n, cap), np.float64)
    ecnt = counts.astype(np.int32)
    diag = np.zeros(n, np.float64)
    first = off[:-1][rows]
    assert np.array_equal(col[first], np.nonzero(rows)[0])
    diag[rows] = val[first]
    r = np.repeat(np.arange(n), counts)                      # row of each off-diagonal entry
    k = np.arange(len(r)) - np.repeat(np.cumsum(counts) - counts, counts)   # its slot
    src = np.repeat(off[:-1] + 1, counts) + k
    ecol[r, k] = col[src]
    eval_[r, k] = -val[src]
    return cap, ecol, eval_, ecnt, diag


def test_noalloc_cg_matches_solve_ppe_twice():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    from paper_2105_01677_gb300 import mps

    sc = scenes.dam_break_2d(seed=1)
    kw = dict(cg_tol=PARITY_CG_TOL, clamp_negative_p=0)
    # the existing entry point
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, **kw))
    sim.solve_ppe()
    ref = sim.read()["p"]
    sim.close()

    off, col, val, b, _, _, flags = oracle.ppe_system(oracle_params(sc, **kw), sc)
    cap, ecol, evl, ecnt, diag = _ell_from_csr(off, col, val, b, sc.types, flags)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_col, d_val, d_cnt, d_diag, d_b = t(ecol), t(evl), t(ecnt), t(diag), t(b)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        d_x = torch.full((sc.n,), float("nan"), dtype=torch.float64, device=dev)
        rc, iters, res = mps.mps_ppe_cg_noalloc(
            sc.n, cap, d_col.data_ptr(), d_cnt.data_ptr(), d_val.data_ptr(), d_diag.data_ptr(),
            d_b.data_ptr(), d_x.data_ptr(), PARITY_CG_TOL, 0, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        x = d_x.cpu().numpy()
        assert rc == 0 and iters > 0 and res <= PARITY_CG_TOL, (call, rc, iters, res)
        assert rel_err(x, ref) <= FP64_TOL, (call, rel_err(x, ref))


def test_noalloc_rejects_oversized_systems():
    __graft_entry__.build()
    from paper_2105_01677_gb300 import mps
    rc, _, _ = mps.mps_ppe_cg_noalloc(mps.NOALLOC_MAX_ROWS + 1, 32, 1, 1, 1, 1, 1, 1, 1e-8,
                                      check=False)
    assert rc == mps.EINVAL


def test_noalloc_cg_matches_the_oracle_cg_near_the_row_limit():
    """A system close to the size limit (the 3D dam break at l0 = 0.01 m: 227,136 rows of
    the 262,144 the fixed array holds), assembled by the oracle and solved both by the
    oracle's CG and by this entry point to 1e-13: the solutions agree to the FP64 parity
    tolerance.  Two calls in a row again."""
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()
    oracle.set_threads(0)
    from paper_2105_01677_gb300 import mps

    sc = scenes.dam_break_3d(seed=2, l0=0.01)
    assert 0.8 * mps.NOALLOC_MAX_ROWS < sc.n <= mps.NOALLOC_MAX_ROWS
    prm = oracle_params(sc, dt=5e-5, cg_tol=PARITY_CG_TOL)
    off, col, val, b, _, _, flags = oracle.ppe_system(prm, sc)
    ref, oit, ores = oracle.cg(off, col, val, b, tol=PARITY_CG_TOL)
    assert ores <= PARITY_CG_TOL
    cap, ecol, evl, ecnt, diag = _ell_from_csr(off, col, val, b, sc.types, flags)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_col, d_val, d_cnt, d_diag, d_b = t(ecol), t(evl), t(ecnt), t(diag), t(b)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        d_x = torch.full((sc.n,), float("nan"), dtype=torch.float64, device=dev)
        rc, iters, res = mps.mps_ppe_cg_noalloc(
            sc.n, cap, d_col.data_ptr(), d_cnt.data_ptr(), d_val.data_ptr(), d_diag.data_ptr(),
            d_b.data_ptr(), d_x.data_ptr(), PARITY_CG_TOL, 0, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        x = d_x.cpu().numpy()
        assert rc == 0 and iters > 0 and res <= PARITY_CG_TOL, (call, rc, iters, res)
        assert rel_err(x, ref) <= FP64_TOL, (call, rel_err(x, ref))
