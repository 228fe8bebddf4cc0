"""Differentiable rollouts: a ``torch.autograd.Function`` over ``mps_step`` whose backward
runs the library's reverse step (``mps_step_vjp``) once per step, with the forward
trajectory checkpointed every ``checkpoint_every`` steps and recomputed segment by segment
(memory: one state per checkpoint plus one segment's states, instead of every step's).

The inputs are the initial positions and velocities (n x dim), the external acceleration
of every step (T x 3): a time-dependent body force such as the inertial acceleration of a
shaken tank in its own frame, and optionally the kinematic viscosity (one value, or one per
particle).  Gradients flow to all of them.  Particle kinds are those of the simulation's
state when the rollout starts.

Two losses of the final state are provided: the kinetic energy of the fluid and the mean
height of its free-surface particles (the free-surface set of the last step, Eq. 15, held
fixed as the reverse step holds every discrete choice fixed).

With CUDA tensors the states, checkpoints and cotangents stay in device memory (the
library's device-memory calls); with CPU tensors they pass through host memory.  Argument
marshalling only: the steps and their reverse run in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch
    return torch


class _HostIO:
    """State and cotangents as numpy arrays through the host calls."""

    def __init__(self, sim):
        self.sim = sim

    def types(self):
        return self.sim.read(want=("types",))["types"].copy()

    def from_tensor(self, t):
        return t.detach().to("cpu", _torch().float64).numpy().copy()

    def read(self):
        st = self.sim.read(want=("pos", "vel", "types"))
        return st["pos"].copy(), st["vel"].copy(), st["types"].copy()

    def write(self, x, u, types):
        self.sim.write(x, u, types)

    def vjp(self, gr, gu):
        _, r, u, g, nu, _ = self.sim.step_vjp(gr, gu, want_nu=True)
        return r, u, g, nu

    def zeros_like(self, x):
        return np.zeros_like(x)

    def to_tensor(self, a, device):
        return _torch().from_numpy(a).to(device)


class _DeviceIO:
    """State and cotangents as CUDA tensors through the device-memory calls."""

    def __init__(self, sim, device):
        self.sim = sim
        self.device = device
        torch = _torch()
        self.shape = (sim.n, sim.dim)
        self._f64 = dict(dtype=torch.float64, device=device)

    def types(self):
        torch = _torch()
        t = torch.empty(self.sim.n, dtype=torch.int8, device=self.device)
        self.sim.read_device(types=t)
        return t

    def from_tensor(self, t):
        return t.detach().to(self.device, _torch().float64).contiguous().clone()

    def read(self):
        torch = _torch()
        x = torch.empty(self.shape, **self._f64)
        u = torch.empty(self.shape, **self._f64)
        t = torch.empty(self.sim.n, dtype=torch.int8, device=self.device)
        self.sim.read_device(pos=x, vel=u, types=t)
        return x, u, t

    def write(self, x, u, types):
        self.sim.write_device(x, u, types)

    def vjp(self, gr, gu):
        torch = _torch()
        r = torch.empty_like(gr)
        u = torch.empty_like(gu)
        nu = torch.empty(self.sim.n, **self._f64)
        _, g, _ = self.sim.step_vjp_device(gr, gu, r, u, out_nu=nu)
        return r, u, g, nu

    def zeros_like(self, x):
        return _torch().zeros_like(x)

    def to_tensor(self, a, device):
        return a if a.device == device else a.to(device)


def _make_function():
    torch = _torch()

    class Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pos, vel, forcing, nu, sim, checkpoint_every):
            K = max(1, int(checkpoint_every))
            io = _DeviceIO(sim, pos.device) if pos.is_cuda else _HostIO(sim)
            if nu is not None:
                # the viscosity of every particle for the whole rollout (densities kept)
                nu_np = nu.detach().to("cpu", torch.float64).numpy()
                nu_i = np.broadcast_to(nu_np, (sim.n,)).copy()
                sim.set_fluid_properties(sim.rho_i, nu_i)
            ctx.nu_shape = None if nu is None else tuple(nu.shape)
            f = forcing.detach().to("cpu", torch.float64).numpy().copy()
            types = io.types()
            x, u = io.from_tensor(pos), io.from_tensor(vel)
            ckpts = []
            for t in range(f.shape[0]):
                if t % K == 0:
                    # every segment starts from a state written afresh with the solver's
                    # guess history cleared, so that its recomputation in backward repeats it
                    # bit for bit
                    if t > 0:
                        x, u, types = io.read()
                    ckpts.append((x, u, types))
                    io.write(x, u, types)
                    sim.clear_history()
                sim.set_gravity(f[t])
                sim.step(1)
            xT, uT, _ = io.read()
            ctx.sim, ctx.K, ctx.ckpts, ctx.f, ctx.io = sim, K, ckpts, f, io
            ctx.dev = pos.device
            return io.to_tensor(xT, pos.device), io.to_tensor(uT, pos.device)

        @staticmethod
        def backward(ctx, g_pos, g_vel):
            sim, K, f, io = ctx.sim, ctx.K, ctx.f, ctx.io
            n_steps = f.shape[0]
            x0 = ctx.ckpts[0][0]
            gr = io.zeros_like(x0) if g_pos is None else io.from_tensor(g_pos)
            gu = io.zeros_like(x0) if g_vel is None else io.from_tensor(g_vel)
            gf = np.zeros_like(f)
            gnu = None
            for s in reversed(range(len(ctx.ckpts))):
                t0, t1 = s * K, min(n_steps, (s + 1) * K)
                x, u, types = ctx.ckpts[s]
                io.write(x, u, types)
                sim.clear_history()
                states = [(x, u, types)]
                for t in range(t0, t1 - 1):
                    sim.set_gravity(f[t])
                    sim.step(1)
                    states.append(io.read())
                for t in reversed(range(t0, t1)):
                    xs, us, ts = states[t - t0]
                    io.write(xs, us, ts)
                    sim.clear_history()
                    sim.set_gravity(f[t])
                    gr, gu, gf[t], gn = io.vjp(gr, gu)
                    gnu = gn if gnu is None else gnu + gn
            dev = ctx.dev
            g_nu = None
            if ctx.nu_shape is not None:
                g_nu = io.to_tensor(gnu, dev)
                if ctx.nu_shape == ():
                    g_nu = g_nu.sum()
            return (io.to_tensor(gr, dev), io.to_tensor(gu, dev),
                    torch.from_numpy(gf).to(dev), g_nu, None, None)

    return Rollout


_FN = None


def rollout(sim, pos, vel, forcing, checkpoint_every: int = 20, nu=None):
    """Run len(forcing) steps of `sim` (an ``mps.Simulation``) from (pos, vel) with the
    external acceleration forcing[t] (3 values) at step t; returns (pos_T, vel_T) as
    float64 tensors on pos's device, differentiable with respect to pos, vel, forcing and,
    when given, nu: the kinematic viscosity [m^2/s] of the rollout, a 0-d tensor (one value
    for every particle) or an (n,) tensor (one per particle, original order), which is set
    on the simulation for the rollout (mps_set_fluid_properties; densities are kept).
    The simulation is left at the final state of the last call (forward or backward)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(pos, vel, forcing, nu, sim, checkpoint_every)


def kinetic_energy(vel, types, mass: float = 1.0):
    """Kinetic energy of the FLUID particles, (mass/2) sum |u_i|^2 (mass: of one particle,
    e.g. rho l0^dim), as a differentiable function of vel (n x dim tensor)."""
    torch = _torch()
    f = torch.as_tensor(np.asarray(types) == 0, device=vel.device)
    return 0.5 * mass * (vel[f] ** 2).sum()


def mean_surface_height(pos, flags, types, axis: int = -1):
    """Mean coordinate along `axis` (default the last one: z in 3D, y in 2D, the vertical of
    the scenes) of the FLUID particles flagged as free surface (bit 0 of flags, Eq. 15).  The
    set is held fixed: only the heights are differentiated."""
    torch = _torch()
    s = (np.asarray(types) == 0) & ((np.asarray(flags) & 1) != 0)
    if not s.any():
        raise ValueError("no free-surface FLUID particle in the state")
    m = torch.as_tensor(s, device=pos.device)
    return pos[m][:, axis].mean()
