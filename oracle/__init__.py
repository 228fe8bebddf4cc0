"""ctypes wrapper of the plain FP64 CPU oracle (``mps_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  The GB300 library never imports, links or calls it, and it
never calls the GB300 library.

``build()`` compiles the C source with gcc (-O2 -ffp-contract=off -fopenmp) in-tree under
``oracle/_build/``; ``lib()`` loads it, building on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mps_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

FLUID, WALL, DUMMY, GHOST = 0, 1, 2, 3
ERRORS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECG_NOCONV", -4: "ENONFINITE",
          -5: "ESKIN", -6: "ECOINCIDENT", -7: "ECAP"}


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where}: {ERRORS.get(code, code)}")
        self.code = code


# A test that plants a mistake in the oracle (tests/test_oracle_mutations.py) points this
# at a library compiled from a mutated copy of the source.
_OVERRIDE = os.environ.get("MPS_ORACLE_LIB")


def build(force: bool = False) -> str:
    if _OVERRIDE:
        return _OVERRIDE
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-std=c11", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("pressure_mode", C.c_int32),
                ("l0", C.c_double), ("re_n", C.c_double), ("re_lap", C.c_double),
                ("rho", C.c_double), ("nu", C.c_double), ("dt", C.c_double),
                ("beta", C.c_double), ("g", C.c_double * 3), ("c0", C.c_double),
                ("gamma", C.c_double), ("alpha_c", C.c_double), ("cg_tol", C.c_double),
                ("cg_max_iter", C.c_int32), ("clamp_negative_p", C.c_int32),
                ("cell_skin", C.c_double), ("box_min", C.c_double * 3),
                ("box_max", C.c_double * 3), ("rho_i", C.POINTER(C.c_double)),
                ("nu_i", C.POINTER(C.c_double)), ("kernel", C.c_int32), ("grad_form", C.c_int32),
                ("source", C.c_int32), ("pad0", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("cg_iters", C.c_int32), ("cg_restarts", C.c_int32), ("cg_resid", C.c_double),
                ("n0_pnd", C.c_double), ("n0_lap", C.c_double), ("lambda_", C.c_double),
                ("max_disp", C.c_double), ("n_surface", C.c_int64), ("n_ghost", C.c_int64),
                ("n_ppe_rows", C.c_int64)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i64, i32, vp = C.POINTER(C.c_double), C.c_int64, C.c_int32, C.c_void_p
        L.orc_lattice.argtypes = [i32, C.c_double, C.c_double, d, d, i32]
        L.orc_cell_keys.argtypes = [C.POINTER(Params), i64, d, C.POINTER(C.c_int8),
                                    C.POINTER(C.c_uint32), C.POINTER(C.c_int32)]
        L.orc_neighbors.argtypes = [i32, i64, d, C.POINTER(C.c_int8), C.c_double, i32,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int32), i64]
        L.orc_pnd.argtypes = [i32, i64, d, C.POINTER(C.c_int8), C.c_double, i32, d, i32]
        L.orc_laplacian.argtypes = [i32, i64, d, C.POINTER(C.c_int8), C.c_double, C.c_double,
                                    C.c_double, d, i32, d, i32]
        L.orc_gradient.argtypes = [i32, i64, d, C.POINTER(C.c_int8), C.c_double, C.c_double,
                                   d, d, d, i32, i32]
        L.orc_step.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int8), d, d,
                               C.POINTER(C.c_uint8), C.POINTER(Report), i32, i32]
        L.orc_ppe_system.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int8),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int32), d, d, d, d,
                                     C.POINTER(C.c_uint8)]
        L.orc_cg.argtypes = [i64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), d, d, d,
                             C.c_double, i32, C.POINTER(C.c_int32), d]
        L.orc_dense_spd_solve.argtypes = [i64, d, d, d]
        L.orc_step_vjp.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int8), d, d, d, d,
                                   d, d, C.POINTER(Report), i32]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        for f in ("orc_lattice", "orc_cell_keys", "orc_neighbors", "orc_pnd", "orc_laplacian",
                  "orc_gradient", "orc_step", "orc_ppe_system", "orc_cg", "orc_dense_spd_solve",
                  "orc_step_vjp"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise OracleError(rc, where)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


@dataclass
class StepParams:
    """MPS parameters (same meaning as the library's mps_params)."""
    dim: int = 2
    l0: float = 0.01
    re_n_l0: float = 2.1
    re_lap_l0: float = 4.0
    rho: float = 1000.0
    nu: float = 1e-6
    dt: float = 1e-4
    beta: float = 0.97
    g: tuple = (0.0, -9.81, 0.0)
    pressure_mode: int = 0
    c0: float = 20.0
    gamma: float = 7.0
    alpha_c: float = 1e-7
    cg_tol: float = 1e-8
    cg_max_iter: int = 0          # 0 -> 10 * N
    clamp_negative_p: int = 1
    cell_skin: float = 0.1
    box_min: tuple = (0.0, 0.0, 0.0)
    box_max: tuple = (1.0, 1.0, 0.0)
    # two-phase flow (Sec. 3.2.1): per-particle density / viscosity in particle order
    rho_i: np.ndarray | None = None
    nu_i: np.ndarray | None = None
    # numerical options: kernel 0 (Eq. 4) / 1 (cubic WC kernel); gradient 0 (difference
    # form) / 1 (CMPS, Eq. 18); PPE source 0 (Eq. 13) / 1 (HS, Eq. 21)
    kernel: int = 0
    grad_form: int = 0
    source: int = 0

    @property
    def re_n(self):
        return self.re_n_l0 * self.l0

    @property
    def re_lap(self):
        return self.re_lap_l0 * self.l0

    def c_struct(self, n: int) -> Params:
        P = Params()
        P.dim, P.pressure_mode = self.dim, self.pressure_mode
        P.l0, P.re_n, P.re_lap = self.l0, self.re_n, self.re_lap
        P.rho, P.nu, P.dt, P.beta = self.rho, self.nu, self.dt, self.beta
        for a in range(3):
            P.g[a] = self.g[a]
            P.box_min[a] = self.box_min[a]
            P.box_max[a] = self.box_max[a]
        P.c0, P.gamma, P.alpha_c = self.c0, self.gamma, self.alpha_c
        P.cg_tol = self.cg_tol
        P.cg_max_iter = self.cg_max_iter if self.cg_max_iter > 0 else 10 * n
        P.clamp_negative_p = self.clamp_negative_p
        P.cell_skin = self.cell_skin
        P.kernel, P.grad_form, P.source = self.kernel, self.grad_form, self.source
        # the arrays stay referenced by this StepParams while the struct is in use
        for name in ("rho_i", "nu_i"):
            a = getattr(self, name)
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64)
                if a.shape != (n,):
                    raise ValueError(f"{name} must have one value per particle")
                setattr(self, name, a)
                setattr(P, name, _p(a, C.c_double))
        return P


def params_for(scene, **kw) -> StepParams:
    g = (0.0, -9.81, 0.0) if scene.dim == 2 else (0.0, 0.0, -9.81)
    base = dict(dim=scene.dim, l0=scene.l0, g=g, box_min=tuple(scene.box_min),
                box_max=tuple(scene.box_max))
    base.update(kw)
    return StepParams(**base)


def lattice(dim: int, l0: float, re: float, kernel: int = 0):
    n0, lam = C.c_double(), C.c_double()
    _check(lib().orc_lattice(dim, l0, re, C.byref(n0), C.byref(lam), kernel), "lattice")
    return n0.value, lam.value


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def cell_keys(prm: StepParams, pos, types):
    pos = _arr(pos, np.float64)
    types = _arr(types, np.int8)
    n = len(types)
    key = np.empty(n, np.uint32)
    cell = np.empty((n, 3), np.int32)
    P = prm.c_struct(n)
    _check(lib().orc_cell_keys(C.byref(P), n, _p(pos, C.c_double), _p(types, C.c_int8),
                               _p(key, C.c_uint32), _p(cell, C.c_int32)), "cell_keys")
    return key, cell


def neighbors(dim, pos, types, re, mode=1):
    """Neighbour sets as CSR (offsets[n+1], ids ascending per row)."""
    pos = _arr(pos, np.float64)
    types = _arr(types, np.int8)
    n = len(types)
    off = np.empty(n + 1, np.int64)
    L = lib()
    _check(L.orc_neighbors(dim, n, _p(pos, C.c_double), _p(types, C.c_int8), re, mode,
                           _p(off, C.c_int64), None, 0), "neighbors")
    ids = np.empty(max(int(off[-1]), 1), np.int32)
    _check(L.orc_neighbors(dim, n, _p(pos, C.c_double), _p(types, C.c_int8), re, mode,
                           _p(off, C.c_int64), _p(ids, C.c_int32), len(ids)), "neighbors")
    return off, ids[: off[-1]]


def pnd(dim, pos, types, re, mode=1, kernel=0):
    pos = _arr(pos, np.float64)
    types = _arr(types, np.int8)
    out = np.empty(len(types), np.float64)
    _check(lib().orc_pnd(dim, len(types), _p(pos, C.c_double), _p(types, C.c_int8), re, mode,
                         _p(out, C.c_double), kernel), "pnd")
    return out


def laplacian(dim, pos, types, re, n0, lam, phi, kernel=0):
    pos = _arr(pos, np.float64)
    types = _arr(types, np.int8)
    phi = _arr(phi, np.float64)
    ncomp = 1 if phi.ndim == 1 else phi.shape[1]
    out = np.empty_like(phi)
    _check(lib().orc_laplacian(dim, len(types), _p(pos, C.c_double), _p(types, C.c_int8), re,
                               n0, lam, _p(phi, C.c_double), ncomp, _p(out, C.c_double),
                               kernel), "laplacian")
    return out


def gradient(dim, pos, types, re, n0, p, phat, kernel=0, form=0):
    pos = _arr(pos, np.float64)
    types = _arr(types, np.int8)
    p = _arr(p, np.float64)
    phat = _arr(phat, np.float64)
    out = np.zeros((len(types), dim), np.float64)
    _check(lib().orc_gradient(dim, len(types), _p(pos, C.c_double), _p(types, C.c_int8), re,
                              n0, _p(p, C.c_double), _p(phat, C.c_double), _p(out, C.c_double),
                              kernel, form), "gradient")
    return out


@dataclass
class State:
    pos: np.ndarray
    vel: np.ndarray
    types: np.ndarray
    p: np.ndarray
    nstar: np.ndarray
    flags: np.ndarray

    @staticmethod
    def from_scene(scene) -> "State":
        n = scene.n
        return State(scene.pos.copy(), scene.vel.copy(), scene.types.copy(), np.zeros(n),
                     np.zeros(n), np.zeros(n, np.uint8))

    def copy(self) -> "State":
        return State(self.pos.copy(), self.vel.copy(), self.types.copy(), self.p.copy(),
                     self.nstar.copy(), self.flags.copy())


def step(prm: StepParams, st: State, solve_only: bool = False, nb_mode: int = 1,
         check: bool = True):
    """One oracle step in place on `st`; returns (rc, report dict)."""
    n = len(st.types)
    for name in ("pos", "vel"):
        setattr(st, name, _arr(getattr(st, name), np.float64))
    st.types = _arr(st.types, np.int8)
    st.p = _arr(st.p, np.float64)
    st.nstar = _arr(st.nstar, np.float64)
    st.flags = _arr(st.flags, np.uint8)
    P = prm.c_struct(n)
    R = Report()
    rc = lib().orc_step(C.byref(P), n, _p(st.pos, C.c_double), _p(st.vel, C.c_double),
                        _p(st.types, C.c_int8), _p(st.p, C.c_double), _p(st.nstar, C.c_double),
                        _p(st.flags, C.c_uint8), C.byref(R), int(solve_only), nb_mode)
    rep = {k: getattr(R, k) for k, _ in Report._fields_}
    rep["lambda"] = rep.pop("lambda_")
    if check:
        _check(rc, "step")
    return rc, rep


def ppe_system(prm: StepParams, scene_or_state):
    """(off, col, val, b, pstar, nstar, flags) of the PPE a step would solve."""
    s = scene_or_state
    pos = _arr(s.pos, np.float64)
    vel = _arr(s.vel, np.float64)
    types = _arr(s.types, np.int8)
    n = len(types)
    P = prm.c_struct(n)
    off = np.empty(n + 1, np.int64)
    L = lib()
    d = C.c_double
    _check(L.orc_ppe_system(C.byref(P), n, _p(pos, d), _p(vel, d), _p(types, C.c_int8),
                            _p(off, C.c_int64), None, None, None, None, None, None), "ppe_system")
    nnz = int(off[-1])
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    b = np.empty(n, np.float64)
    pstar = np.empty_like(pos)
    nstar = np.empty(n, np.float64)
    flags = np.empty(n, np.uint8)
    _check(L.orc_ppe_system(C.byref(P), n, _p(pos, d), _p(vel, d), _p(types, C.c_int8),
                            _p(off, C.c_int64), _p(col, C.c_int32), _p(val, d), _p(b, d),
                            _p(pstar, d), _p(nstar, d), _p(flags, C.c_uint8)), "ppe_system")
    return off, col, val, b, pstar, nstar, flags


def cg(off, col, val, b, tol=1e-8, max_iter=None):
    n = len(b)
    off = _arr(off, np.int64)
    col = _arr(col, np.int32)
    val = _arr(val, np.float64)
    b = _arr(b, np.float64)
    x = np.zeros(n)
    it = C.c_int32()
    res = C.c_double()
    rc = lib().orc_cg(n, _p(off, C.c_int64), _p(col, C.c_int32), _p(val, C.c_double),
                      _p(b, C.c_double), _p(x, C.c_double), tol,
                      max_iter if max_iter else 10 * n, C.byref(it), C.byref(res))
    _check(rc, "cg")
    return x, it.value, res.value


def dense_spd_solve(A, b):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    b = _arr(b, np.float64)
    x = np.zeros(len(b))
    rc = lib().orc_dense_spd_solve(len(b), _p(A, C.c_double), _p(b, C.c_double),
                                   _p(x, C.c_double))
    if rc != 0:
        raise OracleError(-1, "dense_spd_solve: matrix not positive definite")
    return x


def step_vjp(prm: StepParams, st, g_pos, g_vel, nb_mode: int = 1, with_nu: bool = False):
    """Vector-Jacobian product of one oracle step at the state `st` (not modified):
    given dL/dr^{k+1}, dL/du^{k+1} (n x dim), returns (dL/dr^k, dL/du^k, dL/dg[3]), and
    with `with_nu` also dL/dnu_i (n values: the viscosity of every particle; with one
    viscosity for all, dL/dnu is their sum)."""
    pos = _arr(st.pos, np.float64)
    vel = _arr(st.vel, np.float64)
    types = _arr(st.types, np.int8)
    g_pos = _arr(g_pos, np.float64)
    g_vel = _arr(g_vel, np.float64)
    n = len(types)
    assert g_pos.shape == pos.shape and g_vel.shape == vel.shape
    out_r = np.empty_like(pos)
    out_u = np.empty_like(vel)
    out_g = np.zeros(3)
    out_nu = np.zeros(n) if with_nu else None
    P = prm.c_struct(n)
    R = Report()
    d = C.c_double
    _check(lib().orc_step_vjp(C.byref(P), n, _p(pos, d), _p(vel, d), _p(types, C.c_int8),
                              _p(g_pos, d), _p(g_vel, d), _p(out_r, d), _p(out_u, d),
                              _p(out_g, d), None if out_nu is None else _p(out_nu, d),
                              C.byref(R), nb_mode), "step_vjp")
    if with_nu:
        return out_r, out_u, out_g, out_nu
    return out_r, out_u, out_g
