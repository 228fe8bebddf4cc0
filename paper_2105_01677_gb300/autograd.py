"""Differentiable rollouts: a ``torch.autograd.Function`` over ``mps_step`` whose backward
runs the library's reverse step (``mps_step_vjp``) once per step, with the forward
trajectory checkpointed every ``checkpoint_every`` steps and recomputed segment by segment
(memory: one state per checkpoint plus one segment's states, instead of every step's).

The inputs are the initial positions and velocities (n x dim) and the external
acceleration of every step (T x 3): a time-dependent body force such as the inertial
acceleration of a shaken tank in its own frame.  Gradients flow to all three.  Particle
kinds are those of the simulation's state when the rollout starts.  Argument marshalling
only: the steps and their reverse run in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch
    return torch


def _state(sim):
    st = sim.read(want=("pos", "vel", "types"))
    return st["pos"].copy(), st["vel"].copy(), st["types"].copy()


def _make_function():
    torch = _torch()

    class Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pos, vel, forcing, sim, checkpoint_every):
            K = max(1, int(checkpoint_every))
            f = forcing.detach().to("cpu", torch.float64).numpy().copy()
            types = sim.read(want=("types",))["types"].copy()
            x = pos.detach().to("cpu", torch.float64).numpy()
            u = vel.detach().to("cpu", torch.float64).numpy()
            ckpts = []
            for t in range(f.shape[0]):
                if t % K == 0:
                    # every segment starts from a state written afresh, so that its
                    # recomputation in backward repeats it bit for bit
                    if t > 0:
                        x, u, types = _state(sim)
                    ckpts.append((x.copy(), u.copy(), types.copy()))
                    sim.write(x, u, types)
                sim.set_gravity(f[t])
                sim.step(1)
            xT, uT, _ = _state(sim)
            ctx.sim, ctx.K, ctx.ckpts, ctx.f = sim, K, ckpts, f
            ctx.dev = pos.device
            return (torch.from_numpy(xT).to(pos.device), torch.from_numpy(uT).to(pos.device))

        @staticmethod
        def backward(ctx, g_pos, g_vel):
            sim, K, f = ctx.sim, ctx.K, ctx.f
            n_steps = f.shape[0]
            x0 = ctx.ckpts[0][0]
            gr = np.zeros_like(x0) if g_pos is None else g_pos.detach().to("cpu", torch.float64).numpy().copy()
            gu = np.zeros_like(x0) if g_vel is None else g_vel.detach().to("cpu", torch.float64).numpy().copy()
            gf = np.zeros_like(f)
            for s in reversed(range(len(ctx.ckpts))):
                t0, t1 = s * K, min(n_steps, (s + 1) * K)
                x, u, types = ctx.ckpts[s]
                sim.write(x, u, types)
                states = [(x, u, types)]
                for t in range(t0, t1 - 1):
                    sim.set_gravity(f[t])
                    sim.step(1)
                    states.append(_state(sim))
                for t in reversed(range(t0, t1)):
                    xs, us, ts = states[t - t0]
                    sim.write(xs, us, ts)
                    sim.set_gravity(f[t])
                    _, gr, gu, gg, _ = sim.step_vjp(gr, gu)
                    gf[t] = gg
            dev = ctx.dev
            return (torch.from_numpy(gr).to(dev), torch.from_numpy(gu).to(dev),
                    torch.from_numpy(gf).to(dev), None, None)

    return Rollout


_FN = None


def rollout(sim, pos, vel, forcing, checkpoint_every: int = 20):
    """Run len(forcing) steps of `sim` (an ``mps.Simulation``) from (pos, vel) with the
    external acceleration forcing[t] (3 values) at step t; returns (pos_T, vel_T) as
    float64 tensors on pos's device, differentiable with respect to pos, vel and forcing.
    The simulation is left at the final state of the last call (forward or backward)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(pos, vel, forcing, sim, checkpoint_every)
