"""The reverse step on the GPU (mps_step_vjp) against the oracle's reverse step on the same
seeded inputs and cotangents, against central differences of the GPU's own forward step,
and through the checkpointed differentiable rollout.

Scenes jitter walls and dummies too (see tests/test_oracle_adjoint.py: on the exact lattice
some wall pairs sit at r = re, where the step has no derivative).  Parity bound: both sides
solve the forward and the adjoint PPE to a relative residual of 1e-13 (FP64), so the
cotangents agree to ~1e-10 of their largest entry; 1e-8 is asserted."""
import numpy as np
import pytest

import __graft_entry__
import oracle
import scenes
from _parity import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

VJP_TOL = 1e-8
CG = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _scene(dim=2, seed=3, interior=None, fluid=None, l0=0.01):
    if dim == 2:
        sc = scenes.tank_scene(2, l0, interior or (20, 14), fluid or (8, 10), jitter=0.05,
                               wall_jitter=0.02, seed=seed)
    else:
        sc = scenes.tank_scene(3, l0, interior or (9, 6, 8), fluid or (4, 6, 5), jitter=0.05,
                               wall_jitter=0.02, seed=seed)
    f = sc.types == scenes.FLUID
    u = scenes.splitmix_uniform(seed + 17, np.arange(sc.pos.size, dtype=np.uint64))
    sc.vel[f] = 0.2 * (u.reshape(sc.pos.shape)[f] - 0.5)
    return sc


def _cotangents(sc, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(sc.pos.shape), rng.standard_normal(sc.vel.shape)


def _gpu_vjp(sc, gpos, gvel, rho_i=None, nu_i=None, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, rho_i=rho_i, nu_i=nu_i,
                         **gpu_params(sc, **kw))
    try:
        rc, gr, gu, gg, rep = sim.step_vjp(gpos, gvel)
        st = sim.read()
    finally:
        sim.close()
    return gr, gu, gg, rep, st


def _close(a, b, tol=VJP_TOL, what=""):
    scale = np.abs(b).max()
    err = np.abs(a - b).max() / scale
    assert err <= tol, (what, err)


CASES = [
    ("ppe", dict(pressure_mode=0)),
    ("ppe-no-clamp", dict(pressure_mode=0, clamp_negative_p=0)),
    ("eos", dict(pressure_mode=1, c0=20.0)),
    ("viscous", dict(pressure_mode=1, c0=1e-6, nu=0.5)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_vjp_fp64_matches_oracle_2d(name, kw):
    sc = _scene(2)
    gpos, gvel = _cotangents(sc)
    gr, gu, gg, rep, st = _gpu_vjp(sc, gpos, gvel, cg_tol=CG, **kw)
    prm = oracle_params(sc, cg_tol=CG, **kw)
    ogr, ogu, ogg = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel)
    _close(gr, ogr, what="dL/dr")
    _close(gu, ogu, what="dL/du")
    _close(gg, ogg, what="dL/dg")
    if kw["pressure_mode"] == 0:
        assert rep["cg_resid"] <= CG and rep["cg_iters"] > 0
    # the state is not advanced
    assert np.array_equal(st["pos"], sc.pos) and np.array_equal(st["vel"], sc.vel)


@pytest.mark.parametrize("mode", [0, 1])
def test_vjp_fp64_matches_oracle_3d(mode):
    sc = _scene(3, seed=4)
    gpos, gvel = _cotangents(sc, seed=1)
    kw = dict(pressure_mode=mode, c0=20.0, nu=0.05, cg_tol=CG)
    gr, gu, gg, _, _ = _gpu_vjp(sc, gpos, gvel, **kw)
    ogr, ogu, ogg = oracle.step_vjp(oracle_params(sc, **kw), oracle.State.from_scene(sc),
                                    gpos, gvel)
    _close(gr, ogr, what="dL/dr")
    _close(gu, ogu, what="dL/du")
    _close(gg, ogg, what="dL/dg")


def test_vjp_two_phase_matches_oracle():
    sc = _scene(2, seed=6)
    rho, nu = scenes.two_phase(sc, rho=(1000.0, 600.0), nu=(0.05, 0.3))
    gpos, gvel = _cotangents(sc, seed=3)
    gr, gu, gg, _, _ = _gpu_vjp(sc, gpos, gvel, rho_i=rho, nu_i=nu, cg_tol=CG)
    prm = oracle_params(sc, cg_tol=CG, rho_i=rho, nu_i=nu)
    ogr, ogu, ogg = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel)
    _close(gr, ogr, what="dL/dr")
    _close(gu, ogu, what="dL/du")


def test_vjp_ghosts_match_oracle():
    sc = _scene(2, seed=7)
    f = np.flatnonzero(sc.types == scenes.FLUID)
    sc.pos[f[0]] = [sc.box_max[0] + 0.05, 0.05]
    sc.types[f[1]] = scenes.GHOST
    gpos, gvel = _cotangents(sc, seed=4)
    gr, gu, gg, _, _ = _gpu_vjp(sc, gpos, gvel, cg_tol=CG)
    ogr, ogu, _ = oracle.step_vjp(oracle_params(sc, cg_tol=CG), oracle.State.from_scene(sc),
                                  gpos, gvel)
    _close(gr, ogr, what="dL/dr")
    _close(gu, ogu, what="dL/du")
    assert np.all(gu[f[0]] == 0.0) and np.array_equal(gu[f[1]], gvel[f[1]])


@pytest.mark.parametrize("dim", [2, 3])
def test_vjp_fluid_block_without_walls_matches_oracle(dim):
    """Degenerate scene for the reverse step: FLUID only (no walls, no dummies), a block
    compressed to 0.98 l0 with seeded jitter and velocities, so that every PPE row is a
    FLUID row and the surface rows are the only Dirichlet conditions."""
    l0 = 0.01
    m = (14, 10) if dim == 2 else (7, 6, 6)
    g = np.meshgrid(*[np.arange(k) for k in m], indexing="ij")
    pos = np.stack([a.reshape(-1) for a in g], axis=1).astype(np.float64) * (0.98 * l0) + 0.2
    u = scenes.splitmix_uniform(5, np.arange(2 * pos.size, dtype=np.uint64))
    pos = pos + 0.05 * l0 * (u[: pos.size].reshape(pos.shape) - 0.5)
    vel = 0.2 * (u[pos.size:].reshape(pos.shape) - 0.5)
    box = np.array([1.0, 1.0, 1.0 if dim == 3 else 0.0])
    sc = scenes.Scene(dim, l0, pos, vel, np.zeros(len(pos), np.int8), np.zeros(3), box)
    gpos, gvel = _cotangents(sc, seed=2)
    gr, gu, gg, rep, st = _gpu_vjp(sc, gpos, gvel, cg_tol=CG)
    prm = oracle_params(sc, cg_tol=CG)
    ogr, ogu, ogg = oracle.step_vjp(prm, oracle.State.from_scene(sc), gpos, gvel)
    _close(gr, ogr, what="pos")
    _close(gu, ogu, what="vel")
    _close(gg, ogg, what="g")


def test_vjp_mixed_precision_bound():
    """Mixed precision repeats the forward step in its own arithmetic and solves the adjoint
    PPE with the mixed solver to the same FP64 residual; the cotangents stay within the
    mixed path's single-step bound of the FP64 oracle's."""
    sc = _scene(3, seed=5)
    gpos, gvel = _cotangents(sc, seed=2)
    gr, gu, gg, rep, _ = _gpu_vjp(sc, gpos, gvel, precision=1, cg_tol=1e-10)
    ogr, ogu, ogg = oracle.step_vjp(oracle_params(sc, cg_tol=CG), oracle.State.from_scene(sc),
                                    gpos, gvel)
    _close(gr, ogr, tol=1e-5, what="dL/dr")
    _close(gu, ogu, tol=1e-5, what="dL/du")
    assert rep["cg_resid"] <= 1e-10


def _fd_dot(sc, gpos, gvel, v, which, h, **kw):
    from paper_2105_01677_gb300 import mps
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, **kw))
    try:
        outs = []
        for sgn in (1.0, -1.0):
            x = sc.pos + sgn * h * v if which == "pos" else sc.pos
            u = sc.vel + sgn * h * v if which == "vel" else sc.vel
            sim.write(x, u, sc.types)
            sim.step(1)
            st = sim.read(want=("pos", "vel"))
            outs.append((st["pos"], st["vel"]))
        sim.write(sc.pos, sc.vel, sc.types)
        _, gr, gu, _, _ = sim.step_vjp(gpos, gvel)
    finally:
        sim.close()
    (xp, up), (xm, um) = outs
    fd = float(((xp - xm) * gpos + (up - um) * gvel).sum()) / (2.0 * h)
    adj = float(((gr if which == "pos" else gu) * v).sum())
    return fd, adj


@pytest.mark.parametrize("which,h", [("pos", 1e-8), ("vel", 1e-6)])
def test_vjp_matches_central_differences_of_gpu_step(which, h):
    """3D, 2,500+ particles: <gbar, J v> from the GPU's own forward step."""
    sc = _scene(3, seed=8, interior=(14, 9, 12), fluid=(10, 9, 7), l0=0.01)
    gpos, gvel = _cotangents(sc, seed=5)
    v = np.random.default_rng(6).standard_normal(sc.pos.shape)
    fd, adj = _fd_dot(sc, gpos, gvel, v, which, h, cg_tol=1e-14)
    assert abs(fd - adj) <= 1e-6 * abs(adj), (fd, adj)


def test_vjp_rejects_options_without_a_reverse():
    from paper_2105_01677_gb300 import mps
    sc = _scene(2)
    z = np.zeros_like(sc.pos)
    for kw in (dict(kernel=1, pressure_mode=1), dict(gradient_form=1),
               dict(source_term=1)):
        sim = mps.Simulation(sc, torch_alloc=True, **gpu_params(sc, **kw))
        try:
            rc, *_ = sim.step_vjp(z, z, check=False)
            assert rc == mps.EINVAL
        finally:
            sim.close()


def _oracle_rollout_grad(sc, forcing, gT_pos, gT_vel, **kw):
    """Chained oracle reverse steps along the oracle's trajectory."""
    states = []
    st = oracle.State.from_scene(sc)
    for t in range(len(forcing)):
        prm = oracle_params(sc, g=tuple(forcing[t]), **kw)
        states.append((st.copy(), prm))
        oracle.step(prm, st)
    gr, gu = gT_pos.copy(), gT_vel.copy()
    gf = np.zeros_like(forcing)
    for t in reversed(range(len(forcing))):
        s, prm = states[t]
        gr, gu, gf[t] = oracle.step_vjp(prm, s, gr, gu)
    return st, gr, gu, gf


def test_rollout_gradients_match_chained_oracle_reverse():
    """Six steps with a checkpoint every four (two segments, the second recomputed from its
    checkpoint) under a time-varying horizontal forcing; torch.autograd gradients of
    <a, r_T> + <b, u_T> against the oracle's reverse steps chained along its trajectory."""
    import torch
    from paper_2105_01677_gb300 import autograd, mps
    sc = _scene(2, seed=9)
    T = 6
    forcing = np.zeros((T, 3))
    forcing[:, 0] = scenes.sloshing_forcing(np.arange(T) * 1e-4, amplitude=0.5, freq=20.0)
    forcing[:, 1] = -9.81
    a, b = _cotangents(sc, seed=8)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, cg_tol=CG))
    try:
        x = torch.tensor(sc.pos, dtype=torch.float64, requires_grad=True)
        u = torch.tensor(sc.vel, dtype=torch.float64, requires_grad=True)
        f = torch.tensor(forcing, dtype=torch.float64, requires_grad=True)
        xT, uT = autograd.rollout(sim, x, u, f, checkpoint_every=4)
        loss = (xT * torch.from_numpy(a)).sum() + (uT * torch.from_numpy(b)).sum()
        loss.backward()
    finally:
        sim.close()
    ost, ogr, ogu, ogf = _oracle_rollout_grad(sc, forcing, a, b, cg_tol=CG)
    assert np.abs(xT.detach().numpy() - ost.pos).max() / sc.l0 <= 1e-8
    _close(x.grad.numpy(), ogr, tol=1e-7, what="dL/dr0")
    _close(u.grad.numpy(), ogu, tol=1e-7, what="dL/du0")
    _close(f.grad.numpy()[:, :2], ogf[:, :2], tol=1e-7, what="dL/dg")


def test_rollout_forcing_gradient_matches_central_differences():
    """dL/d(forcing) of a 10-step rollout (checkpoint every 3) against central differences
    of the GPU rollout in a random direction of the forcing sequence."""
    import torch
    from paper_2105_01677_gb300 import autograd, mps
    sc = _scene(2, seed=10)
    T = 10
    f0 = np.zeros((T, 3))
    f0[:, 1] = -9.81
    a, b = _cotangents(sc, seed=11)
    v = np.random.default_rng(12).standard_normal((T, 3))
    v[:, 2] = 0.0
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, cg_tol=1e-14))
    try:
        def loss_of(fv, grad=False):
            x = torch.tensor(sc.pos, dtype=torch.float64)
            u = torch.tensor(sc.vel, dtype=torch.float64)
            f = torch.tensor(fv, dtype=torch.float64, requires_grad=grad)
            xT, uT = autograd.rollout(sim, x, u, f, checkpoint_every=3)
            loss = (xT * torch.from_numpy(a)).sum() + (uT * torch.from_numpy(b)).sum()
            if grad:
                loss.backward()
                return float(loss.detach()), f.grad.numpy()
            return float(loss)
        _, gf = loss_of(f0, grad=True)
        h = 1e-3
        fd = (loss_of(f0 + h * v) - loss_of(f0 - h * v)) / (2.0 * h)
    finally:
        sim.close()
    adj = float((gf * v).sum())
    assert abs(fd - adj) <= 1e-6 * abs(adj), (fd, adj)


def test_device_memory_calls_equal_host_calls():
    """read / write / reverse step with CUDA tensors give the host calls' results bit for bit."""
    import torch
    from paper_2105_01677_gb300 import mps
    sc = _scene(3, seed=11)
    a, b = _cotangents(sc, seed=12)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, **gpu_params(sc, cg_tol=CG))
    try:
        sim.step(2)
        host = sim.read()
        dev = torch.device("cuda", 0)
        x = torch.empty((sc.n, 3), dtype=torch.float64, device=dev)
        u = torch.empty_like(x)
        p = torch.empty(sc.n, dtype=torch.float64, device=dev)
        t = torch.empty(sc.n, dtype=torch.int8, device=dev)
        sim.read_device(pos=x, vel=u, p=p, types=t)
        assert np.array_equal(x.cpu().numpy(), host["pos"])
        assert np.array_equal(u.cpu().numpy(), host["vel"])
        assert np.array_equal(p.cpu().numpy(), host["p"])
        assert np.array_equal(t.cpu().numpy(), host["types"])
        _, gr_h, gu_h, gg_h, _ = sim.step_vjp(a, b)
        ga, gb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        ro, uo = torch.empty_like(ga), torch.empty_like(gb)
        _, gg_d, rep = sim.step_vjp_device(ga, gb, ro, uo)
        assert np.array_equal(ro.cpu().numpy(), gr_h) and np.array_equal(uo.cpu().numpy(), gu_h)
        assert np.array_equal(gg_d, gg_h)
        # write from device memory, then a step equals a step after the host write
        sim.write_device(x, u, t)
        sim.step(1)
        s1 = sim.read()
        sim.write(host["pos"], host["vel"], host["types"])
        sim.step(1)
        s2 = sim.read()
        for k in ("pos", "vel", "p"):
            assert np.array_equal(s1[k], s2[k]), k
    finally:
        sim.close()


def test_rollout_on_cuda_tensors_equals_host_rollout():
    import torch
    from paper_2105_01677_gb300 import autograd, mps
    sc = _scene(2, seed=13)
    T = 5
    forcing = np.zeros((T, 3))
    forcing[:, 0] = 0.3
    forcing[:, 1] = -9.81
    a, b = _cotangents(sc, seed=14)
    grads = []
    for device in ("cpu", "cuda"):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, cg_tol=CG))
        try:
            x = torch.tensor(sc.pos, dtype=torch.float64, device=device, requires_grad=True)
            u = torch.tensor(sc.vel, dtype=torch.float64, device=device, requires_grad=True)
            f = torch.tensor(forcing, dtype=torch.float64, device=device, requires_grad=True)
            xT, uT = autograd.rollout(sim, x, u, f, checkpoint_every=2)
            assert xT.device.type == device
            loss = (xT * torch.from_numpy(a).to(device)).sum() + (uT * torch.from_numpy(b).to(device)).sum()
            loss.backward()
            grads.append((xT.detach().cpu().numpy(), x.grad.cpu().numpy(), u.grad.cpu().numpy(),
                          f.grad.cpu().numpy()))
        finally:
            sim.close()
    for h, d in zip(*grads):
        assert np.array_equal(h, d)


# ------------------------------------------------------------------ the viscosity
@pytest.mark.parametrize("case", ["2d-ppe", "2d-eos-viscous", "3d-ppe", "two-phase"])
def test_vjp_viscosity_cotangent_matches_oracle(case):
    """dL/dnu_i of one step (the prediction's viscosity, Eq. 7) against the oracle's."""
    from paper_2105_01677_gb300 import mps
    nu_i = rho_i = None
    if case == "2d-ppe":
        sc, kw = _scene(2, seed=21), dict(cg_tol=CG, nu=0.05)
    elif case == "2d-eos-viscous":
        sc, kw = _scene(2, seed=22), dict(pressure_mode=1, c0=20.0, nu=0.5)
    elif case == "3d-ppe":
        sc, kw = _scene(3, seed=23), dict(cg_tol=CG, nu=0.05)
    else:
        sc, kw = _scene(2, seed=24), dict(cg_tol=CG)
        rho_i, nu_i = scenes.two_phase(sc, rho=(1000.0, 600.0), nu=(0.05, 0.3))
    gpos, gvel = _cotangents(sc, seed=25)
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True, rho_i=rho_i, nu_i=nu_i,
                         **gpu_params(sc, **kw))
    try:
        _, gr, gu, gg, gnu, _ = sim.step_vjp(gpos, gvel, want_nu=True)
    finally:
        sim.close()
    okw = dict(kw)
    if rho_i is not None:
        okw.update(rho_i=rho_i, nu_i=nu_i)
    ogr, ogu, ogg, ognu = oracle.step_vjp(oracle_params(sc, **okw), oracle.State.from_scene(sc),
                                          gpos, gvel, with_nu=True)
    _close(gnu, ognu, what="dL/dnu")
    _close(gu, ogu, what="dL/du")
    assert np.all(gnu[sc.types != scenes.FLUID] == 0.0)


def test_rollout_viscosity_gradient_matches_chained_oracle_and_differences():
    """A 6-step rollout (checkpoint every 4) with the viscosity as a differentiable 0-d
    tensor: d(kinetic energy)/dnu against the oracle's per-step dL/dnu summed along its
    trajectory, and against central differences of the GPU rollout in nu."""
    import torch
    from paper_2105_01677_gb300 import autograd, mps
    sc = _scene(2, seed=26)
    T, nu0 = 6, 0.05
    forcing = np.zeros((T, 3))
    forcing[:, 1] = -9.81
    sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                         **gpu_params(sc, cg_tol=1e-14, nu=nu0))
    try:
        def loss_of(nu_value, grad=False):
            x = torch.tensor(sc.pos, dtype=torch.float64)
            u = torch.tensor(sc.vel, dtype=torch.float64, requires_grad=grad)
            f = torch.tensor(forcing, dtype=torch.float64)
            nu = torch.tensor(nu_value, dtype=torch.float64, requires_grad=grad)
            xT, uT = autograd.rollout(sim, x, u, f, checkpoint_every=4, nu=nu)
            loss = autograd.kinetic_energy(uT, sc.types)
            if grad:
                loss.backward()
                return float(loss.detach()), float(nu.grad), u.grad.numpy(), uT.detach().numpy()
            return float(loss)
        L0, g_nu, g_u0, uT = loss_of(nu0, grad=True)
        h = 1e-6 * nu0
        fd = (loss_of(nu0 + h) - loss_of(nu0 - h)) / (2.0 * h)
    finally:
        sim.close()
    assert abs(fd - g_nu) <= 1e-6 * abs(g_nu), (fd, g_nu)
    # the chained oracle reverse: KE's cotangent at the final state is u_T on FLUID rows
    st = oracle.State.from_scene(sc)
    states = []
    for t in range(T):
        prm = oracle_params(sc, cg_tol=CG, nu=nu0, g=tuple(forcing[t]))
        states.append((st.copy(), prm))
        oracle.step(prm, st)
    f = (sc.types == scenes.FLUID)[:, None]
    gr, gu = np.zeros_like(sc.pos), st.vel * f
    onu = 0.0
    for t in reversed(range(T)):
        s, prm = states[t]
        gr, gu, _, gn = oracle.step_vjp(prm, s, gr, gu, with_nu=True)
        onu += gn.sum()
    assert abs(g_nu - onu) <= 1e-7 * abs(onu), (g_nu, onu)
    _close(g_u0, gu, tol=1e-7, what="dKE/du0")
