"""Shared helpers of the GPU parity tests: run one step on both sides from the same scene
bytes and compare.  The oracle side never sees a value produced by the CUDA path."""
import numpy as np

import oracle
import scenes

# FP64 state: relative to the largest magnitude of the oracle's field
FP64_TOL = 1e-10
# free-surface flags are compared outside the band |n* - beta n0| <= 1e-12 n0, where the
# two summation orders may legitimately disagree; the band is asserted empty on the scenes
FLAG_BAND = 1e-12
PARITY_CG_TOL = 1e-13


def small_3d(seed=1, l0=0.025):
    return scenes.dam_break_3d(seed=seed, l0=l0)


def gpu_params(scene, **kw):
    g = (0.0, -9.81, 0.0) if scene.dim == 2 else (0.0, 0.0, -9.81)
    base = dict(dim=scene.dim, l0=scene.l0, re_n=2.1 * scene.l0, re_lap=4.0 * scene.l0, g=g,
                box_min=tuple(scene.box_min), box_max=tuple(scene.box_max))
    base.update(kw)
    return base


def oracle_params(scene, **kw):
    kw = dict(kw)
    for k in ("precision", "ppe_operator", "inner_tol", "max_outer", "nbr_cap"):
        kw.pop(k, None)
    return oracle.params_for(scene, **kw)


def run_gpu(scene, nsteps=1, solve_only=False, torch_alloc=True, check=True, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(scene, torch_alloc=torch_alloc, use_torch_stream=True, **kw)
    try:
        if solve_only:
            rc, rep = sim.solve_ppe(check=check)
        else:
            rc, rep = sim.step(nsteps, check=check)
        st = sim.read()
        consts = sim.constants()
    finally:
        sim.close()
    return rc, rep, st, consts


def run_oracle(scene, nsteps=1, solve_only=False, **kw):
    prm = oracle_params(scene, **kw)
    st = oracle.State.from_scene(scene)
    rep = None
    for _ in range(nsteps):
        _, rep = oracle.step(prm, st, solve_only=solve_only)
    return rep, st, prm


def rel_err(val, ref):
    scale = np.abs(ref).max()
    if scale == 0.0:
        return float(np.abs(val).max())
    return float(np.abs(val - ref).max() / scale)


def flags_agree(gpu_flags, ref_flags, ref_nstar, beta, n0):
    band = np.abs(ref_nstar - beta * n0) <= FLAG_BAND * n0
    outside = ~band
    ok = np.array_equal(gpu_flags[outside], ref_flags[outside])
    return ok, int(band.sum())


def disp_err(scene, gpu_pos, ref_pos):
    """Displacement error over one step, relative to the largest displacement, after
    removing the rounding of the absolute positions themselves (a few ulps of |r|): the
    stored positions cannot resolve a displacement more finely than that."""
    d_ref = ref_pos - scene.pos
    ulp_floor = 8.0 * np.finfo(np.float64).eps * np.abs(ref_pos).max()
    dev = np.abs((gpu_pos - scene.pos) - d_ref).max()
    return max(0.0, dev - ulp_floor) / max(np.abs(d_ref).max(), 1e-300)


def compare_step(scene, gpu_st, ora_st, prm, tol=FP64_TOL, fields=("p", "n_star", "vel", "disp")):
    """Return dict of relative errors and asserts flag agreement."""
    errs = {}
    errs["pos"] = rel_err(gpu_st["pos"], ora_st.pos)
    if "p" in fields:
        errs["p"] = rel_err(gpu_st["p"], ora_st.p)
    if "n_star" in fields:
        # the library evaluates n* where the method uses it: FLUID and WALL particles
        rows = ora_st.types <= oracle.WALL
        errs["n_star"] = rel_err(gpu_st["n_star"][rows], ora_st.nstar[rows])
        assert np.all(gpu_st["n_star"][~rows] == 0.0)
    if "vel" in fields:
        errs["vel"] = rel_err(gpu_st["vel"], ora_st.vel)
    if "disp" in fields:
        errs["disp"] = disp_err(scene, gpu_st["pos"], ora_st.pos)
    n0, _ = oracle.lattice(scene.dim, prm.l0, prm.re_n)
    ok, nband = flags_agree(gpu_st["flags"], ora_st.flags, ora_st.nstar, prm.beta, n0)
    assert ok, "free-surface flags differ outside the rounding band"
    assert nband == 0, f"{nband} particles inside the flag rounding band"
    assert np.array_equal(gpu_st["types"], ora_st.types)
    for k, v in errs.items():
        assert v <= tol, f"{k}: relative error {v:.3e} > {tol:.1e}"
    return errs


def ulp_sensitivity(scene, nsteps, seed=0, **kw):
    """Conditioning of the oracle's own trajectory: relative change of each field after
    `nsteps` oracle steps when every FLUID coordinate is moved by one ulp (random sign).
    The PPE right-hand side (n* - n0)/(n0 dt^2) amplifies position rounding by ~1/dt^2,
    so over several steps p differs at ~1e-10 between two runs that differ only in the
    rounding of one operation; multi-step comparisons take a bound from this."""
    prm = oracle_params(scene, **kw)
    a = oracle.State.from_scene(scene)
    b = oracle.State.from_scene(scene)
    f = scene.types == scenes.FLUID
    rng = np.random.default_rng(seed)
    pert = b.pos.copy()
    pert[f] = np.nextafter(pert[f], pert[f] + rng.choice([-1.0, 1.0], size=pert[f].shape))
    b.pos = pert
    for _ in range(nsteps):
        oracle.step(prm, a)
        oracle.step(prm, b)
    return {k: rel_err(getattr(b, k), getattr(a, k)) for k in ("p", "vel", "pos")}

