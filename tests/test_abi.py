"""The C-ABI library loads, exports every symbol include/mps.h declares, and its structs
match the Python binding's ctypes mirror (checked against gcc's own offsetof).  No GPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

import __graft_entry__
from paper_2105_01677_gb300 import mps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mps.h")


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return mps.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(mps_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mps_create", "mps_step", "mps_solve_ppe", "mps_read_state", "mps_destroy",
                     "mps_debug_cells", "mps_debug_neighbors", "mps_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    names = declared_functions()
    assert names
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(mps.EXPORTS)


def test_library_links_no_torch(L):
    out = subprocess.run(["ldd", mps.lib_path()], capture_output=True, text=True).stdout
    assert "torch" not in out and "c10" not in out


def _c_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "mps.h"
#define P(s, f) printf(#s " " #f " %zu\n", offsetof(s, f));
int main(void) {
  printf("mps_params size %zu\n", sizeof(mps_params));
  printf("mps_report size %zu\n", sizeof(mps_report));
  printf("mps_vjp_report size %zu\n", sizeof(mps_vjp_report));
  printf("mps_tuning size %zu\n", sizeof(mps_tuning));
  P(mps_params, dim) P(mps_params, l0) P(mps_params, g) P(mps_params, cg_max_iter)
  P(mps_params, precision) P(mps_params, nbr_cap) P(mps_params, cell_skin) P(mps_params, box_min)
  P(mps_params, box_max) P(mps_params, inner_tol) P(mps_params, ppe_operator) P(mps_params, stream)
  P(mps_params, alloc) P(mps_params, release) P(mps_params, alloc_user) P(mps_params, list_every)
  P(mps_params, gather_block) P(mps_params, kernel) P(mps_params, source_term)
  P(mps_params, ppe_host_loop) P(mps_params, cg_x0) P(mps_params, spmv_block)
  P(mps_params, build_block) P(mps_params, bucket_sort) P(mps_params, cg_unroll)
  P(mps_params, predict_tpr)
  P(mps_tuning, build_block) P(mps_tuning, cg_unroll) P(mps_tuning, predict_tpr) P(mps_tuning, gather_ms) P(mps_tuning, build_ms)
  P(mps_tuning, cell_skin) P(mps_tuning, cell_ms) P(mps_tuning, predict_ms)
  P(mps_report, list_gathered)
  P(mps_report, cg_resid) P(mps_report, n_surface) P(mps_report, max_disp) P(mps_report, lambda)
  P(mps_report, steps_done) P(mps_report, cand_tests) P(mps_report, pairs_pnd)
  P(mps_report, list_tests) P(mps_report, bucket_merged) P(mps_report, n_moved)
  P(mps_vjp_report, cg_iters) P(mps_vjp_report, cg_resid) P(mps_vjp_report, forward)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        out = subprocess.check_output([exe], text=True)
    res = {}
    for line in out.splitlines():
        s, f, v = line.split()
        res[(s, f)] = int(v)
    return res


def test_struct_layout_matches_binding():
    lay = _c_layout()
    assert lay[("mps_params", "size")] == C.sizeof(mps.mps_params)
    assert lay[("mps_report", "size")] == C.sizeof(mps.mps_report)
    assert lay[("mps_vjp_report", "size")] == C.sizeof(mps.mps_vjp_report)
    assert lay[("mps_tuning", "size")] == C.sizeof(mps.mps_tuning)
    classes = {"mps_params": mps.mps_params, "mps_report": mps.mps_report,
               "mps_vjp_report": mps.mps_vjp_report, "mps_tuning": mps.mps_tuning}
    for (s, f), off in lay.items():
        if f == "size":
            continue
        cls = classes[s]
        name = "lambda_" if f == "lambda" else f
        assert getattr(cls, name).offset == off, (s, f)


def test_defaults_follow_the_paper(L):
    P = mps.mps_params_default()
    assert P.beta == 0.97 and P.gamma == 7.0 and P.alpha_c == 1e-7
    assert P.re_n == pytest.approx(2.1 * P.l0) and P.re_lap == pytest.approx(4.0 * P.l0)
    assert P.cg_tol == 1e-8 and P.clamp_negative_p == 1 and P.precision == 0


def test_invalid_arguments_rejected_before_device_use(L):
    import numpy as np
    pos = np.zeros((3, 2))
    t = np.zeros(3, np.int8)
    h = C.c_void_p()
    for kw in (dict(dim=4), dict(re_n=0.0), dict(dt=-1.0), dict(precision=2),
               dict(box_max=(0.0, 0.0, 0.0)), dict(list_every=-1), dict(kernel=2),
               dict(gradient_form=3), dict(source_term=1, kernel=1), dict(source_term=3),
               dict(precision=1, ppe_operator=1, kernel=1), dict(cg_x0=5), dict(cg_x0=-1), dict(ppe_host_loop=2),
               dict(build_block=96), dict(build_block=512), dict(spmv_block=128),
               dict(gather_block=48), dict(bucket_sort=2), dict(cg_unroll=3), dict(predict_tpr=3),
               dict(step_graph=3)):
        P = mps.mps_params_default(**kw)
        rc = L.mps_create(pos.ctypes.data_as(C.POINTER(C.c_double)), None,
                          t.ctypes.data_as(C.POINTER(C.c_int8)), 3, C.byref(P), C.byref(h))
        assert rc == mps.EINVAL, kw
    P = mps.mps_params_default()
    rc = L.mps_create(None, None, None, 3, C.byref(P), C.byref(h))
    assert rc == mps.EINVAL
    bad = np.array([[0.0, np.nan], [0.1, 0.1], [0.2, 0.2]])
    rc = L.mps_create(bad.ctypes.data_as(C.POINTER(C.c_double)), None,
                      t.ctypes.data_as(C.POINTER(C.c_int8)), 3, C.byref(P), C.byref(h))
    assert rc == mps.ENONFINITE
    t2 = np.array([0, 7, 1], np.int8)
    rc = L.mps_create(pos.ctypes.data_as(C.POINTER(C.c_double)), None,
                      t2.ctypes.data_as(C.POINTER(C.c_int8)), 3, C.byref(P), C.byref(h))
    assert rc == mps.EINVAL
    assert L.mps_step(None, 1, None) == mps.EINVAL
    assert L.mps_step_vjp(None, None, None, None, None, None, None, None) == mps.EINVAL
    g = np.zeros(3)
    assert L.mps_set_gravity(None, g.ctypes.data_as(C.POINTER(C.c_double))) == mps.EINVAL


def test_strerror_names_every_code(L):
    for code in range(0, -9, -1):
        s = mps.mps_strerror(code)
        assert s.startswith("MPS_")
