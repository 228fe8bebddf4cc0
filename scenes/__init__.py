"""Seeded synthetic particle scenes shared by the CUDA path's tests, the bench and the oracle.

This module only places particles on lattices and draws seeded jitter; it holds none of the
MPS arithmetic (no kernel weight, no number density, no pressure).  Both the CPU oracle and
the GB300 library consume the exact bytes produced here.

Scenes follow the shapes of the paper's dam-break workloads (Sec. 5.2 "Dam break": a water
column of height 2L on a floor of 4L, average particle distance l0) in 2D and 3D, with
2 wall layers and 2 dummy layers on the tank walls (the wall / dummy particle kinds are the
boundary flags of the PPE assembly listing (Listing 2, Sec. 4.3)).

Particle kinds (int8): FLUID=0, WALL=1, DUMMY=2, GHOST=3.

Jitter: fluid particles only, uniform in [-a*l0, +a*l0) per axis, drawn from the
counter-based SplitMix64 generator (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): value = mix(mix(seed + G) + (4*id + axis) + G), where
G = 0x9E3779B97F4A7C15 and mix is the published SplitMix64 finaliser; the top 53 bits
give a double in [0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FLUID, WALL, DUMMY, GHOST = 0, 1, 2, 3

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_uniform(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based uniform doubles in [0, 1): one value per uint64 counter."""
    with np.errstate(over="ignore"):
        s = _mix64(np.uint64(seed) + _G)
        v = _mix64(s + np.asarray(counters, dtype=np.uint64) + _G)
    return (v >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Scene:
    """A particle set: positions / velocities (n, dim) float64, kinds (n,) int8."""

    dim: int
    l0: float
    pos: np.ndarray
    vel: np.ndarray
    types: np.ndarray
    box_min: np.ndarray
    box_max: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.types.shape[0])

    @property
    def n_fluid(self) -> int:
        return int(np.count_nonzero(self.types == FLUID))

    def copy(self) -> "Scene":
        return Scene(self.dim, self.l0, self.pos.copy(), self.vel.copy(), self.types.copy(),
                     self.box_min.copy(), self.box_max.copy(), dict(self.meta))


def _jitter(seed: int, ids: np.ndarray, dim: int, amp: float) -> np.ndarray:
    ids = np.asarray(ids, dtype=np.uint64)
    ctr = ids[:, None] * np.uint64(4) + np.arange(dim, dtype=np.uint64)[None, :]
    u = splitmix_uniform(seed, ctr.reshape(-1)).reshape(len(ids), dim)
    return (2.0 * u - 1.0) * amp


def tank_scene(dim: int, l0: float, interior: tuple, fluid: tuple, *, layers_wall: int = 2,
               layers_dummy: int = 2, wall_height: int | None = None, seed: int = 1,
               jitter: float = 1e-4, headroom: float = 1.0, wall_jitter: float = 0.0) -> Scene:
    """Fluid block in the corner of an open-top tank.

    interior: interior lattice counts per axis (last axis is vertical).
    fluid:    fluid lattice counts per axis, placed at the origin corner.
    Lattice sites sit at (i + 0.5) * l0; boundary sites form `layers_wall` wall layers and
    `layers_dummy` dummy layers (Chebyshev layer index) on every side except the top.
    wall_height: number of lattice rows the side walls reach (default: full interior height).
    jitter, wall_jitter: uniform offsets of up to that many l0 per axis for the fluid and
    for the wall and dummy sites (default: walls on the exact lattice).
    """
    assert dim in (2, 3) and len(interior) == dim and len(fluid) == dim
    L = layers_wall + layers_dummy
    nint = [int(v) for v in interior]
    nfl = [int(v) for v in fluid]
    hw = nint[-1] if wall_height is None else int(wall_height)

    # fluid block, ids 0..nf-1, x fastest
    grids = np.meshgrid(*[np.arange(c) for c in nfl], indexing="ij")
    fidx = np.stack([g.reshape(-1, order="F") for g in grids], axis=1)
    # boundary sites
    ranges = [np.arange(-L, nint[a] + L) for a in range(dim - 1)] + [np.arange(-L, hw)]
    bgrids = np.meshgrid(*ranges, indexing="ij")
    bidx = np.stack([g.reshape(-1, order="F") for g in bgrids], axis=1)
    layer = np.zeros(len(bidx), dtype=np.int64)
    for a in range(dim):
        below = np.where(bidx[:, a] < 0, -bidx[:, a], 0)
        above = np.where(bidx[:, a] >= nint[a], bidx[:, a] - nint[a] + 1, 0) if a < dim - 1 else 0
        layer = np.maximum(layer, np.maximum(below, above))
    keep = layer > 0
    bidx, layer = bidx[keep], layer[keep]
    btypes = np.where(layer <= layers_wall, WALL, DUMMY).astype(np.int8)

    idx = np.concatenate([fidx, bidx], axis=0)
    types = np.concatenate([np.full(len(fidx), FLUID, np.int8), btypes])
    pos = (idx.astype(np.float64) + 0.5) * l0
    nf = len(fidx)
    if jitter > 0.0:
        pos[:nf] += _jitter(seed, np.arange(nf), dim, jitter * l0)
    if wall_jitter > 0.0:
        pos[nf:] += _jitter(seed + 7919, np.arange(nf, len(pos)), dim, wall_jitter * l0)
    vel = np.zeros_like(pos)

    box_min = np.zeros(3)
    box_max = np.zeros(3)
    for a in range(dim):
        box_min[a] = -(L + 1) * l0
        top = (nint[a] + L + 1) * l0 if a < dim - 1 else (hw + 1) * l0 * (1.0 + headroom)
        box_max[a] = top
    meta = dict(kind="tank", interior=tuple(nint), fluid=tuple(nfl), seed=seed, jitter=jitter,
                wall_jitter=wall_jitter,
                layers_wall=layers_wall, layers_dummy=layers_dummy, wall_height=hw)
    return Scene(dim, l0, pos, vel, types, box_min, box_max, meta)


def dam_break_2d(seed: int = 1, l0: float = 0.01, jitter: float = 1e-4) -> Scene:
    """2D dam break: 0.2 x 0.4 m column in a 0.8 x 0.5 m tank (800 fluid, 752 wall+dummy)."""
    n = lambda L: int(np.floor(L / l0 + 1e-9))
    return tank_scene(2, l0, (n(0.8), n(0.5)), (n(0.2), n(0.4)), seed=seed, jitter=jitter)


def dam_break_3d(seed: int = 1, l0: float = 0.0075, jitter: float = 1e-4,
                 tank=(1.6, 0.6, 0.6), column=(0.40, 0.60, 0.30)) -> Scene:
    """3D dam break: 0.40 x 0.60 x 0.30 m column in a 1.6 x 0.6 x 0.6 m open-top tank.

    At l0 = 0.0075 m: 53 x 80 x 40 = 169,600 fluid and 270,432 wall+dummy particles
    (2 + 2 layers, walls to full height), N = 440,032.
    """
    n = lambda L: int(np.floor(L / l0 + 1e-9))
    return tank_scene(3, l0, tuple(n(v) for v in tank), tuple(n(v) for v in column),
                      seed=seed, jitter=jitter)


def two_phase(scene: Scene, rho=(1000.0, 800.0), nu=(1e-6, 5e-6)):
    """Per-particle density and kinematic viscosity of a two-layer fluid (material inputs of
    the multi-density model, Sec. 3.2.1): fluid lattice layers whose centres lie in the lower
    half of the column are phase 0 (rho[0], nu[0]), the others phase 1; walls and dummies
    take phase 0's values.  Returns (rho, nu) arrays in particle order."""
    up = scene.dim - 1
    f = scene.types == FLUID
    h = scene.pos[f, up]
    base = h.min() - 0.5 * scene.l0          # bottom of the column (lattice sites at +l0/2)
    layers = int(round((h.max() - h.min()) / scene.l0)) + 1
    split = base + 0.5 * layers * scene.l0 + 0.25 * scene.l0   # between two layer centres
    upper = f & (scene.pos[:, up] > split)
    rho_i = np.where(upper, rho[1], rho[0]).astype(np.float64)
    nu_i = np.where(upper, nu[1], nu[0]).astype(np.float64)
    return rho_i, nu_i


def ensemble_2d(count: int = 256, seed: int = 1, fluid=(500, 20000), aspect=(0.5, 2.0),
                l0=(0.005, 0.01)) -> list:
    """Independent 2D dam breaks of seeded sizes: per scene a fluid count, a column aspect
    (height / width) and a particle spacing drawn uniformly from the given ranges (counter-
    based SplitMix64 draws of (seed, scene)); the column of nx x ny lattice sites
    (nx ny ~ fluid count, ny / nx ~ aspect) stands in the corner of a tank 4 nx wide and
    1.25 ny high (the proportions of the 2D dam break), 2 wall + 2 dummy layers."""
    out = []
    for s in range(count):
        u = splitmix_uniform(seed, np.arange(4 * s, 4 * s + 4, dtype=np.uint64))
        nf = fluid[0] + u[0] * (fluid[1] - fluid[0])
        a = aspect[0] + u[1] * (aspect[1] - aspect[0])
        h = l0[0] + u[2] * (l0[1] - l0[0])
        nx = max(2, int(round(np.sqrt(nf / a))))
        ny = max(2, int(round(a * nx)))
        out.append(tank_scene(2, h, (4 * nx, int(np.ceil(1.25 * ny))), (nx, ny),
                              seed=seed * 100003 + s, jitter=1e-4))
    return out


def sloshing_3d(seed: int = 1, l0: float = 0.008, tank=(0.5, 0.3, 0.3), fill: float = 0.5,
                jitter: float = 1e-4) -> Scene:
    """3D sloshing tank: a 0.5 x 0.3 x 0.3 m open-top tank filled over its whole floor to
    `fill` of its height (l0 = 0.008: 62 x 37 x 18 = 41,292 fluid, 85,564 particles with the
    2 wall + 2 dummy layers), fluid at rest."""
    n = lambda L: int(np.floor(L / l0 + 1e-9))
    interior = tuple(n(v) for v in tank)
    column = (interior[0], interior[1], n(fill * tank[2]))
    return tank_scene(3, l0, interior, column, seed=seed, jitter=jitter)


def sloshing_forcing(t, amplitude: float = 0.02, freq: float = 1.2):
    """Horizontal (x) body acceleration [m/s^2] in the frame of a tank displaced by
    X(t) = amplitude sin(2 pi freq t): the inertial acceleration -X''(t) =
    amplitude (2 pi freq)^2 sin(2 pi freq t).  t may be an array."""
    w = 2.0 * np.pi * freq
    return amplitude * w * w * np.sin(w * np.asarray(t, dtype=np.float64))


def still_tank_2d(l0: float = 0.01, width: float = 0.2, depth: float = 0.2, seed: int = 1,
                  jitter: float = 0.0) -> Scene:
    """Fluid at rest filling the full width of a 2D tank (hydrostatic check)."""
    n = lambda L: int(np.floor(L / l0 + 1e-9))
    return tank_scene(2, l0, (n(width), n(depth) + 10), (n(width), n(depth)), seed=seed,
                      jitter=jitter)


def random_cloud(n: int, dim: int, seed: int, extent: float = 1.0, clustered: bool = False,
                 kinds: bool = True) -> Scene:
    """Random particles (uniform, or in a few Gaussian clusters) with random kinds.

    Used for neighbour-set and cell-key checks; values come from SplitMix64 counters.
    """
    u = splitmix_uniform(seed, np.arange(n * dim, dtype=np.uint64)).reshape(n, dim)
    if clustered:
        k = 4
        centres = splitmix_uniform(seed + 7, np.arange(k * dim, dtype=np.uint64)).reshape(k, dim)
        which = (splitmix_uniform(seed + 11, np.arange(n, dtype=np.uint64)) * k).astype(np.int64)
        # Box-Muller-free spread: sum of three uniforms, centred
        s = sum(splitmix_uniform(seed + 13 + t, np.arange(n * dim, dtype=np.uint64))
                for t in range(3)).reshape(n, dim) / 3.0 - 0.5
        u = np.clip(centres[which] + 0.15 * s, 0.0, 1.0 - 1e-12)
    pos = u * extent
    if kinds:
        t = (splitmix_uniform(seed + 3, np.arange(n, dtype=np.uint64)) * 3).astype(np.int8)
    else:
        t = np.zeros(n, np.int8)
    box_min = np.full(3, -0.05 * extent)
    box_max = np.full(3, 1.05 * extent)
    if dim == 2:
        box_min[2] = 0.0
        box_max[2] = 0.0
    return Scene(dim, extent / 20.0, pos, np.zeros_like(pos), t, box_min, box_max,
                 dict(kind="random", seed=seed, clustered=clustered))
