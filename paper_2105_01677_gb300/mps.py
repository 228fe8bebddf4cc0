"""ctypes binding of the GB300 MPS library (C ABI in include/mps.h).

Argument marshalling only: every stage of the time step runs in the library's CUDA kernels.
Functions keep the C names (mps_create, mps_step, mps_solve_ppe, mps_read_state, ...).
Device memory for a context comes from PyTorch's caching allocator when `torch_alloc=True`
(through the library's allocation hooks) and the context runs on the current PyTorch stream.

There is no CPU fallback: if the shared library is missing or cannot be loaded, `lib()`
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

FLUID, WALL, DUMMY, GHOST = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECG_NOCONV, ENONFINITE, ESKIN, ECOINCIDENT, ECAP, EDEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class mps_params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("pressure_mode", C.c_int32), ("l0", C.c_double),
                ("re_n", C.c_double), ("re_lap", C.c_double), ("rho", C.c_double),
                ("nu", C.c_double), ("dt", C.c_double), ("beta", C.c_double),
                ("g", C.c_double * 3), ("c0", C.c_double), ("gamma", C.c_double),
                ("alpha_c", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("precision", C.c_int32), ("clamp_negative_p", C.c_int32),
                ("nbr_cap", C.c_int32), ("cell_skin", C.c_double),
                ("box_min", C.c_double * 3), ("box_max", C.c_double * 3),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32),
                ("ppe_operator", C.c_int32), ("device", C.c_int32), ("gather_block", C.c_int32),
                ("list_every", C.c_int32), ("kernel", C.c_int32), ("gradient_form", C.c_int32),
                ("source_term", C.c_int32), ("ppe_host_loop", C.c_int32),
                ("cg_x0", C.c_int32), ("step_graph", C.c_int32), ("inner_cg", C.c_int32),
                ("spmv_block", C.c_int32), ("build_block", C.c_int32), ("bucket_sort", C.c_int32), ("cg_unroll", C.c_int32), ("predict_tpr", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("release", RELEASE_FN),
                ("alloc_user", C.c_void_p)]


class mps_scene(C.Structure):
    _fields_ = [("l0", C.c_double), ("box_min", C.c_double * 3), ("box_max", C.c_double * 3)]


class mps_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("cg_iters", C.c_int32), ("cg_outer", C.c_int32),
                ("list_gathered", C.c_int32), ("cg_resid", C.c_double), ("n_surface", C.c_int64),
                ("n_ghost", C.c_int64), ("n_ppe_rows", C.c_int64), ("max_disp", C.c_double),
                ("n0_pnd", C.c_double), ("n0_lap", C.c_double), ("lambda_", C.c_double),
                ("steps_done", C.c_int64), ("cand_tests", C.c_int64), ("pairs_ppe", C.c_int64),
                ("pairs_pnd", C.c_int64), ("list_tests", C.c_int64), ("step_graph", C.c_int32),
                ("n_fast", C.c_int32), ("bucket_merged", C.c_int32), ("n_moved", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


class mps_tuning(C.Structure):
    _fields_ = [("gather_block", C.c_int32), ("spmv_block", C.c_int32), ("cg_fused", C.c_int32),
                ("build_block", C.c_int32), ("cg_unroll", C.c_int32), ("predict_tpr", C.c_int32),
                ("gather_ms", C.c_double), ("spmv_ms", C.c_double),
                ("solve_ms", C.c_double), ("build_ms", C.c_double), ("cell_skin", C.c_double),
                ("cell_ms", C.c_double), ("predict_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class mps_vjp_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("cg_iters", C.c_int32), ("cg_outer", C.c_int32),
                ("pad", C.c_int32), ("cg_resid", C.c_double), ("forward", mps_report)]

    def as_dict(self) -> dict:
        return dict(status=self.status, cg_iters=self.cg_iters, cg_outer=self.cg_outer,
                    cg_resid=self.cg_resid, forward=self.forward.as_dict())


EXPORTS = ("mps_params_default", "mps_create", "mps_step", "mps_solve_ppe", "mps_read_state",
           "mps_write_state", "mps_debug_cells", "mps_debug_neighbors", "mps_get_constants",
           "mps_set_profiling", "mps_get_profile", "mps_ppe_cg_noalloc", "mps_destroy",
           "mps_strerror", "mps_set_fluid_properties", "mps_create_ensemble",
           "mps_scene_residuals", "mps_autotune", "mps_set_gravity", "mps_step_vjp",
           "mps_time_kernel", "mps_read_state_device", "mps_write_state_device",
           "mps_step_vjp_device", "mps_measure_peak", "mps_clear_history")
NOALLOC_MAX_ROWS = 262144
STAGES = ("bucket", "gather", "predict", "build", "ppe", "update")

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def lib(build_if_missing: bool = False):
    """Load the shared library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"GB300 MPS library not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    d, i8, u8 = C.POINTER(C.c_double), C.POINTER(C.c_int8), C.POINTER(C.c_uint8)
    vpp = C.POINTER(C.c_void_p)
    L.mps_params_default.argtypes = [C.POINTER(mps_params)]
    L.mps_params_default.restype = None
    L.mps_create.argtypes = [d, d, i8, C.c_int64, C.POINTER(mps_params), vpp]
    L.mps_step.argtypes = [C.c_void_p, C.c_int32, C.POINTER(mps_report)]
    L.mps_solve_ppe.argtypes = [C.c_void_p, C.POINTER(mps_report)]
    L.mps_read_state.argtypes = [C.c_void_p, d, d, d, d, u8, i8]
    L.mps_write_state.argtypes = [C.c_void_p, d, d, i8]
    L.mps_set_fluid_properties.argtypes = [C.c_void_p, d, d]
    L.mps_set_gravity.argtypes = [C.c_void_p, d]
    L.mps_time_kernel.argtypes = [C.c_void_p, C.c_int32, C.c_int32, d, d]
    L.mps_step_vjp.argtypes = [C.c_void_p, d, d, d, d, d, d, C.POINTER(mps_vjp_report)]
    vp = C.c_void_p
    L.mps_read_state_device.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.mps_write_state_device.argtypes = [vp, vp, vp, vp]
    L.mps_step_vjp_device.argtypes = [vp, vp, vp, vp, vp, d, vp, C.POINTER(mps_vjp_report)]
    L.mps_create_ensemble.argtypes = [d, d, i8, C.POINTER(C.c_int32), C.c_int64,
                                      C.POINTER(mps_params), C.POINTER(mps_scene), C.c_int32,
                                      C.POINTER(C.c_void_p)]
    L.mps_scene_residuals.argtypes = [C.c_void_p, d]
    L.mps_autotune.argtypes = [C.c_void_p, C.c_int32, C.POINTER(mps_tuning)]
    L.mps_debug_cells.argtypes = [C.c_void_p, C.POINTER(C.c_uint32)]
    L.mps_debug_neighbors.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int32), C.c_int64]
    L.mps_get_constants.argtypes = [C.c_void_p, d]
    L.mps_set_profiling.argtypes = [C.c_void_p, C.c_int32]
    L.mps_get_profile.argtypes = [C.c_void_p, d, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.mps_ppe_cg_noalloc.argtypes = [C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                     C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    L.mps_measure_peak.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, d, d]
    L.mps_clear_history.argtypes = [C.c_void_p]
    L.mps_destroy.argtypes = [C.c_void_p]
    L.mps_destroy.restype = None
    L.mps_strerror.argtypes = [C.c_int]
    L.mps_strerror.restype = C.c_char_p
    for f in ("mps_create", "mps_step", "mps_solve_ppe", "mps_read_state", "mps_write_state",
              "mps_debug_cells", "mps_debug_neighbors", "mps_get_constants", "mps_set_profiling",
              "mps_get_profile", "mps_ppe_cg_noalloc", "mps_set_fluid_properties",
              "mps_create_ensemble", "mps_scene_residuals", "mps_autotune", "mps_set_gravity",
              "mps_step_vjp", "mps_time_kernel", "mps_read_state_device",
              "mps_write_state_device", "mps_step_vjp_device", "mps_measure_peak",
              "mps_clear_history"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


class MPSError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().mps_strerror(code).decode()
        super().__init__(f"{where}: {msg}")
        self.code = code


def _check(rc: int, where: str):
    if rc != OK:
        raise MPSError(rc, where)


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def mps_strerror(code: int) -> str:
    return lib().mps_strerror(code).decode()


def mps_params_default(**kw) -> mps_params:
    """Defaults of the C library, then keyword overrides (g / box as sequences)."""
    P = mps_params()
    lib().mps_params_default(C.byref(P))
    for k, v in kw.items():
        if k in ("g", "box_min", "box_max"):
            arr = getattr(P, k)
            for a in range(3):
                arr[a] = float(v[a]) if a < len(v) else 0.0
        else:
            setattr(P, k, v)
    return P


class _TorchAllocator:
    """Device memory hooks backed by torch.cuda's caching allocator."""

    def __init__(self, device: int, stream_ptr, limit: int | None = None):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream_ptr
        self._live = {}
        # optional byte budget: beyond it an allocation fails (returns NULL) as a full
        # device would, so that callers can exercise the library's MPS_ENOMEM path
        self.limit = limit

        def _alloc(nbytes, user):
            if self.limit is not None and self.live_bytes() + int(nbytes) > self.limit:
                return None
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device)
            except Exception:
                return None
            self._live[ptr] = nbytes
            return ptr

        def _release(ptr, user):
            if ptr in self._live:
                del self._live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.release = RELEASE_FN(_release)

    def live_bytes(self) -> int:
        return int(sum(self._live.values()))


def mps_create(pos, vel, types, params: mps_params, torch_alloc: bool = False,
               use_torch_stream: bool = False, alloc_limit: int | None = None):
    """Create a context; returns an opaque handle (c_void_p).  pos/vel: (n, dim) float64."""
    L = lib()
    pos = np.ascontiguousarray(pos, np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64)
    types = np.ascontiguousarray(types, np.int8)
    n = len(types)
    keep = None
    if torch_alloc or use_torch_stream:
        import torch
        dev = int(params.device)
        if use_torch_stream:
            params.stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        if torch_alloc:
            keep = _TorchAllocator(dev, params.stream, alloc_limit)
            params.alloc = keep.alloc
            params.release = keep.release
    h = C.c_void_p()
    rc = L.mps_create(_ptr(pos, C.c_double), _ptr(vel, C.c_double), _ptr(types, C.c_int8), n,
                      C.byref(params), C.byref(h))
    _check(rc, "mps_create")
    _keepalive[h.value] = (keep, params)
    return h


_keepalive = {}


def mps_create_ensemble(pos, vel, types, scene, params: mps_params, scenes,
                        torch_alloc: bool = False, use_torch_stream: bool = False):
    """Create an ensemble context: scene[i] in [0, len(scenes)); scenes: sequence of
    (l0, box_min, box_max).  Returns the handle."""
    L = lib()
    pos = np.ascontiguousarray(pos, np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64)
    types = np.ascontiguousarray(types, np.int8)
    scene = np.ascontiguousarray(scene, np.int32)
    n = len(types)
    S = len(scenes)
    tab = (mps_scene * S)()
    for s, (l0, bmin, bmax) in enumerate(scenes):
        tab[s].l0 = float(l0)
        for a in range(3):
            tab[s].box_min[a] = float(bmin[a]) if a < len(bmin) else 0.0
            tab[s].box_max[a] = float(bmax[a]) if a < len(bmax) else 0.0
    keep = None
    if torch_alloc or use_torch_stream:
        import torch
        dev = int(params.device)
        if use_torch_stream:
            params.stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        if torch_alloc:
            keep = _TorchAllocator(dev, params.stream)
            params.alloc = keep.alloc
            params.release = keep.release
    h = C.c_void_p()
    rc = L.mps_create_ensemble(_ptr(pos, C.c_double), _ptr(vel, C.c_double), _ptr(types, C.c_int8),
                               _ptr(scene, C.c_int32), n, C.byref(params), tab, S, C.byref(h))
    _check(rc, "mps_create_ensemble")
    _keepalive[h.value] = (keep, params)
    return h


def mps_autotune(h, repeats: int = 3) -> dict:
    """Pick the fastest gather block shape, FP32 SpMV block and inner-CG form for the current
    state; returns the choice and its times (mps_tuning as a dict)."""
    t = mps_tuning()
    _check(lib().mps_autotune(h, int(repeats), C.byref(t)), "mps_autotune")
    return t.as_dict()


def mps_scene_residuals(h, n_scenes: int):
    out = np.zeros(n_scenes, np.float64)
    _check(lib().mps_scene_residuals(h, _ptr(out, C.c_double)), "mps_scene_residuals")
    return out


def mps_step(h, nsteps: int = 1, check: bool = True):
    rep = mps_report()
    rc = lib().mps_step(h, int(nsteps), C.byref(rep))
    if check:
        _check(rc, "mps_step")
    return rc, rep.as_dict()


def mps_solve_ppe(h, check: bool = True):
    rep = mps_report()
    rc = lib().mps_solve_ppe(h, C.byref(rep))
    if check:
        _check(rc, "mps_solve_ppe")
    return rc, rep.as_dict()


def mps_read_state(h, n: int, dim: int, pos=None, vel=None, p=None, n_star=None, flags=None,
                   types=None, want=("pos", "vel", "p", "n_star", "flags", "types")):
    """Read the state in original particle order into (optional, preallocated) arrays."""
    out = {}
    if "pos" in want:
        out["pos"] = pos if pos is not None else np.empty((n, dim), np.float64)
    if "vel" in want:
        out["vel"] = vel if vel is not None else np.empty((n, dim), np.float64)
    if "p" in want:
        out["p"] = p if p is not None else np.empty(n, np.float64)
    if "n_star" in want:
        out["n_star"] = n_star if n_star is not None else np.empty(n, np.float64)
    if "flags" in want:
        out["flags"] = flags if flags is not None else np.empty(n, np.uint8)
    if "types" in want:
        out["types"] = types if types is not None else np.empty(n, np.int8)
    rc = lib().mps_read_state(h, _ptr(out.get("pos"), C.c_double), _ptr(out.get("vel"), C.c_double),
                              _ptr(out.get("p"), C.c_double), _ptr(out.get("n_star"), C.c_double),
                              _ptr(out.get("flags"), C.c_uint8), _ptr(out.get("types"), C.c_int8))
    _check(rc, "mps_read_state")
    return out


def mps_write_state(h, pos, vel=None, types=None):
    pos = np.ascontiguousarray(pos, np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64)
    types = None if types is None else np.ascontiguousarray(types, np.int8)
    _check(lib().mps_write_state(h, _ptr(pos, C.c_double), _ptr(vel, C.c_double),
                                 _ptr(types, C.c_int8)), "mps_write_state")


def mps_set_fluid_properties(h, rho=None, nu=None, check: bool = True):
    """Per-particle density / viscosity (original order) of a two-phase flow; None keeps that
    property uniform.  Returns the status."""
    rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
    nu = None if nu is None else np.ascontiguousarray(nu, np.float64)
    rc = lib().mps_set_fluid_properties(h, _ptr(rho, C.c_double), _ptr(nu, C.c_double))
    if check:
        _check(rc, "mps_set_fluid_properties")
    return rc


def mps_set_gravity(h, g):
    """External acceleration g (3 values; the unused axis of 2D is ignored) for the next steps."""
    ga = np.zeros(3, np.float64)
    ga[: len(g)] = np.asarray(g, np.float64)
    _check(lib().mps_set_gravity(h, _ptr(ga, C.c_double)), "mps_set_gravity")


def mps_step_vjp(h, g_pos, g_vel, check: bool = True, want_nu: bool = False):
    """Reverse of the step from the current state: given dL/dr^{k+1}, dL/du^{k+1} ((n, dim)
    float64, original order) returns (rc, dL/dr^k, dL/du^k, dL/dg[3], report dict); with
    `want_nu` (rc, dL/dr^k, dL/du^k, dL/dg[3], dL/dnu_i[n], report dict)."""
    g_pos = np.ascontiguousarray(g_pos, np.float64)
    g_vel = np.ascontiguousarray(g_vel, np.float64)
    if g_pos.shape != g_vel.shape:
        raise ValueError("g_pos and g_vel must have the same shape (n, dim)")
    out_r = np.empty_like(g_pos)
    out_u = np.empty_like(g_vel)
    out_g = np.zeros(3, np.float64)
    out_nu = np.zeros(g_pos.shape[0], np.float64) if want_nu else None
    rep = mps_vjp_report()
    rc = lib().mps_step_vjp(h, _ptr(g_pos, C.c_double), _ptr(g_vel, C.c_double),
                            _ptr(out_r, C.c_double), _ptr(out_u, C.c_double),
                            _ptr(out_g, C.c_double), _ptr(out_nu, C.c_double), C.byref(rep))
    if check:
        _check(rc, "mps_step_vjp")
    if want_nu:
        return rc, out_r, out_u, out_g, out_nu, rep.as_dict()
    return rc, out_r, out_u, out_g, rep.as_dict()


def _dptr(t, dtype_name, shape=None):
    """Device address of a contiguous CUDA tensor (None passes through)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"expected a contiguous CUDA tensor of {dtype_name}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def mps_read_state_device(h, n: int, dim: int, pos=None, vel=None, p=None, n_star=None,
                          flags=None, types=None):
    """Read the state into preallocated CUDA tensors (float64 (n, dim) / (n,), uint8 flags,
    int8 types); any may be None."""
    _check(lib().mps_read_state_device(h, _dptr(pos, "float64", (n, dim)),
                                       _dptr(vel, "float64", (n, dim)), _dptr(p, "float64", (n,)),
                                       _dptr(n_star, "float64", (n,)), _dptr(flags, "uint8", (n,)),
                                       _dptr(types, "int8", (n,))), "mps_read_state_device")


def mps_write_state_device(h, pos, vel=None, types=None):
    _check(lib().mps_write_state_device(h, _dptr(pos, "float64"), _dptr(vel, "float64"),
                                        _dptr(types, "int8")), "mps_write_state_device")


def mps_step_vjp_device(h, g_pos, g_vel, out_pos, out_vel, check: bool = True, out_nu=None):
    """Reverse of the step with CUDA tensors: g_pos, g_vel in; out_pos, out_vel (same shape)
    and optionally out_nu (float64 (n,): dL/dnu_i) out; returns (rc, dL/dg[3] as numpy,
    report dict)."""
    out_g = np.zeros(3, np.float64)
    rep = mps_vjp_report()
    rc = lib().mps_step_vjp_device(h, _dptr(g_pos, "float64"), _dptr(g_vel, "float64"),
                                   _dptr(out_pos, "float64", tuple(g_pos.shape)),
                                   _dptr(out_vel, "float64", tuple(g_vel.shape)),
                                   _ptr(out_g, C.c_double),
                                   _dptr(out_nu, "float64", (g_pos.shape[0],)), C.byref(rep))
    if check:
        _check(rc, "mps_step_vjp_device")
    return rc, out_g, rep.as_dict()


KERNEL_SPMV32, KERNEL_RESID_FF, KERNEL_SPMV64 = 0, 1, 2


def mps_time_kernel(h, which: int, repeats: int = 10):
    """(mean ms per launch, algorithmic bytes per launch) of one PPE kernel on the system
    of the last step."""
    ms = C.c_double()
    by = C.c_double()
    _check(lib().mps_time_kernel(h, int(which), int(repeats), C.byref(ms), C.byref(by)),
           "mps_time_kernel")
    return ms.value, by.value


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA = 0, 1, 2


def mps_measure_peak(which: int, device: int = 0, repeats: int = 5, stream: int = 0):
    """(TFLOP/s, ms per launch) of the device's fused multiply-add rate: PEAK_FFMA (FP32),
    PEAK_FFMA2 (packed two-lane FP32) or PEAK_DFMA (FP64)."""
    tf = C.c_double()
    ms = C.c_double()
    _check(lib().mps_measure_peak(int(device), int(which), int(repeats), stream or None,
                                  C.byref(tf), C.byref(ms)), "mps_measure_peak")
    return tf.value, ms.value


def mps_debug_cells(h, n: int):
    out = np.empty(n, np.uint32)
    _check(lib().mps_debug_cells(h, _ptr(out, C.c_uint32)), "mps_debug_cells")
    return out


def mps_debug_neighbors(h, n: int, which: int):
    off = np.empty(n + 1, np.int64)
    _check(lib().mps_debug_neighbors(h, which, _ptr(off, C.c_int64), None, 0), "mps_debug_neighbors")
    ids = np.empty(max(int(off[-1]), 1), np.int32)
    _check(lib().mps_debug_neighbors(h, which, _ptr(off, C.c_int64), _ptr(ids, C.c_int32), len(ids)),
           "mps_debug_neighbors")
    return off, ids[: off[-1]]


def mps_get_constants(h):
    out = np.zeros(8, np.float64)
    _check(lib().mps_get_constants(h, _ptr(out, C.c_double)), "mps_get_constants")
    return dict(n0_pnd=out[0], n0_lap=out[1], lambda_=out[2], h=out[3],
                ncell=(int(out[4]), int(out[5]), int(out[6])), cap=int(out[7]))


def mps_set_profiling(h, on: bool = True):
    _check(lib().mps_set_profiling(h, 1 if on else 0), "mps_set_profiling")


def mps_get_profile(h):
    ms = np.zeros(len(STAGES), np.float64)
    calls = np.zeros(len(STAGES), np.int64)
    launches = np.zeros(1, np.int64)
    _check(lib().mps_get_profile(h, _ptr(ms, C.c_double), _ptr(calls, C.c_int64),
                                 _ptr(launches, C.c_int64)), "mps_get_profile")
    return dict(stage_ms=dict(zip(STAGES, ms.tolist())),
                stage_calls=dict(zip(STAGES, calls.tolist())), launches=int(launches[0]))


def mps_ppe_cg_noalloc(n: int, cap: int, col: int, cnt: int, val: int, diag: int, b: int, x: int,
                       tol: float, max_iter: int = 0, stream: int = 0, check: bool = True):
    """FP64 CG on a caller-owned system without any allocation (device pointers as ints).

    Returns (rc, iterations, relative residual)."""
    it = C.c_int32()
    res = C.c_double()
    rc = lib().mps_ppe_cg_noalloc(int(n), int(cap), col, cnt, val, diag, b, x, float(tol),
                                  int(max_iter), stream or None, C.byref(it), C.byref(res))
    if check:
        _check(rc, "mps_ppe_cg_noalloc")
    return rc, it.value, res.value


def mps_destroy(h):
    if h is not None and h.value:
        lib().mps_destroy(h)
        _keepalive.pop(h.value, None)


class Ensemble:
    """Convenience owner of an ensemble context built from a list of scene-like objects
    (all of one dimension), concatenated in order; read() returns per-scene states."""

    def __init__(self, scene_list, torch_alloc: bool = False, use_torch_stream: bool = False,
                 **params):
        self.scenes = list(scene_list)
        self.dim = self.scenes[0].dim
        self.sizes = [sc.n for sc in self.scenes]
        self.n = int(sum(self.sizes))
        pos = np.concatenate([sc.pos for sc in self.scenes])
        vel = np.concatenate([sc.vel for sc in self.scenes])
        types = np.concatenate([sc.types for sc in self.scenes])
        scene = np.concatenate([np.full(sc.n, s, np.int32) for s, sc in enumerate(self.scenes)])
        sc0 = self.scenes[0]
        g = (0.0, -9.81, 0.0) if self.dim == 2 else (0.0, 0.0, -9.81)
        base = dict(dim=self.dim, l0=sc0.l0, re_n=2.1 * sc0.l0, re_lap=4.0 * sc0.l0, g=g,
                    box_min=tuple(sc0.box_min), box_max=tuple(sc0.box_max))
        base.update(params)
        self.params = mps_params_default(**base)
        tab = [(sc.l0, tuple(sc.box_min), tuple(sc.box_max)) for sc in self.scenes]
        self.h = mps_create_ensemble(pos, vel, types, scene, self.params, tab, torch_alloc,
                                     use_torch_stream)

    def step(self, nsteps: int = 1, check: bool = True):
        return mps_step(self.h, nsteps, check)

    def read(self, **kw):
        st = mps_read_state(self.h, self.n, self.dim, **kw)
        out, o = [], 0
        for m in self.sizes:
            out.append({k: v[o:o + m] for k, v in st.items()})
            o += m
        return out

    def residuals(self):
        return mps_scene_residuals(self.h, len(self.scenes))

    def autotune(self, repeats: int = 3) -> dict:
        return mps_autotune(self.h, repeats)

    def close(self):
        mps_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h is not None:
                self.close()
        except Exception:
            pass


class Simulation:
    """Convenience owner of one context built from a scene-like object."""

    def __init__(self, scene, torch_alloc: bool = False, use_torch_stream: bool = False,
                 rho_i=None, nu_i=None, alloc_limit: int | None = None, **params):
        self.n, self.dim = scene.n, scene.dim
        g = (0.0, -9.81, 0.0) if scene.dim == 2 else (0.0, 0.0, -9.81)
        base = dict(dim=scene.dim, l0=scene.l0, re_n=2.1 * scene.l0, re_lap=4.0 * scene.l0, g=g,
                    box_min=tuple(scene.box_min), box_max=tuple(scene.box_max))
        base.update(params)
        self.params = mps_params_default(**base)
        self.h = mps_create(scene.pos, scene.vel, scene.types, self.params, torch_alloc,
                            use_torch_stream, alloc_limit)
        self.rho_i = self.nu_i = None
        if rho_i is not None or nu_i is not None:
            self.set_fluid_properties(rho_i, nu_i)

    def set_fluid_properties(self, rho=None, nu=None, check: bool = True):
        rc = mps_set_fluid_properties(self.h, rho, nu, check)
        if rc == OK:
            self.rho_i = None if rho is None else np.array(rho, np.float64)
            self.nu_i = None if nu is None else np.array(nu, np.float64)
        return rc

    def step(self, nsteps: int = 1, check: bool = True):
        return mps_step(self.h, nsteps, check)

    def solve_ppe(self, check: bool = True):
        return mps_solve_ppe(self.h, check)

    def set_gravity(self, g):
        mps_set_gravity(self.h, g)

    def step_vjp(self, g_pos, g_vel, check: bool = True, want_nu: bool = False):
        """(rc, dL/dr, dL/du, dL/dg, report) of the step from the current state; with
        `want_nu` (rc, dL/dr, dL/du, dL/dg, dL/dnu_i, report)."""
        return mps_step_vjp(self.h, g_pos, g_vel, check, want_nu)

    # device-memory variants (CUDA tensors in original order)
    def read_device(self, pos=None, vel=None, p=None, n_star=None, flags=None, types=None):
        mps_read_state_device(self.h, self.n, self.dim, pos, vel, p, n_star, flags, types)

    def write_device(self, pos, vel=None, types=None):
        mps_write_state_device(self.h, pos, vel, types)

    def step_vjp_device(self, g_pos, g_vel, out_pos, out_vel, check: bool = True, out_nu=None):
        return mps_step_vjp_device(self.h, g_pos, g_vel, out_pos, out_vel, check, out_nu)

    def read(self, **kw):
        return mps_read_state(self.h, self.n, self.dim, **kw)

    def write(self, pos, vel=None, types=None):
        mps_write_state(self.h, pos, vel, types)

    def clear_history(self):
        """The next PPE solve starts from zero (cg_x0's history cleared)."""
        _check(lib().mps_clear_history(self.h), "mps_clear_history")

    def constants(self):
        return mps_get_constants(self.h)

    def autotune(self, repeats: int = 3) -> dict:
        return mps_autotune(self.h, repeats)

    def close(self):
        mps_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if self.h is not None:
                self.close()
        except Exception:
            pass
