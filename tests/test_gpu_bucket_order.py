"""The bucket build from the previous order against the radix sort.

A graph-run bucket build sorts only the particles whose cell key changed and merges them into
the previous order (bucket_sort = 0, the default); bucket_sort = 1 radix-sorts every build.
Both must give the stable order by cell key, so whole trajectories are bit-identical.  The
scenes start with a seeded random velocity field, so that particles cross cell faces in
every step (counted on the host from the positions), and cover radix sorts of an even pass
count (the small scenes: the merged order is copied back into the key buffer) and an odd one
(the 3D dam break at l0 = 0.01 m, 19 key bits)."""
import numpy as np
import pytest

import __graft_entry__
import scenes
from _parity import gpu_params, small_3d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    __graft_entry__.build()


def _stirred(sc, speed, seed, jitter=0.15):
    """FLUID particles shifted off the lattice (uniform within +-jitter l0, so that their
    distances to the cell faces spread out) and given a random velocity field."""
    sc = sc.copy()
    rng = np.random.default_rng(seed)
    f = sc.types == scenes.FLUID
    m = int(f.sum())
    sc.pos[f] += rng.uniform(-jitter, jitter, size=(m, sc.dim)) * sc.l0
    sc.vel[f] = rng.normal(0.0, speed, size=(m, sc.dim))
    return sc


def _cells(pos, bmin, h):
    return np.floor((pos - np.asarray(bmin)[: pos.shape[1]]) / h).astype(np.int64)


def _run(make, nsteps, reports=None, **kw):
    sim = make(**kw)
    try:
        states, crossed = [], 0
        prev = sim.read()
        h = sim.constants()["h"] if hasattr(sim, "constants") else None
        for _ in range(nsteps):
            rc, rep = sim.step(1)
            assert rc == 0
            if reports is not None:
                reports.append(rep)
            st = sim.read()
            states.append(st)
            if h is not None:
                a = _cells(prev["pos"], sim.scene.box_min, h)
                b = _cells(st["pos"], sim.scene.box_min, h)
                crossed += int(np.any(a != b, axis=1).sum())
            prev = st
    finally:
        sim.close()
    return states, crossed


def _same(sa, sb):
    for a, b in zip(sa, sb):
        for key in ("p", "n_star", "pos", "vel", "flags"):
            assert np.array_equal(a[key], b[key]), key


@pytest.mark.parametrize("case", ["2d-mixed", "2d-fp64", "3d-small-mixed", "3d-227k-mixed",
                                  "2d-eos"])
def test_merged_order_equals_radix_order(case):
    from paper_2105_01677_gb300 import mps
    if case.startswith("2d"):
        sc, kw = _stirred(scenes.dam_break_2d(seed=1), 1.0, 11), dict(dt=1e-4)
    elif case == "3d-small-mixed":
        sc, kw = _stirred(small_3d(seed=2), 1.0, 12), dict(dt=5e-5)
    else:
        sc, kw = _stirred(scenes.dam_break_3d(seed=3, l0=0.01), 1.0, 13), dict(dt=5e-5)
    kw["precision"] = 0 if case == "2d-fp64" else 1
    if case == "2d-eos":
        kw["pressure_mode"] = 1

    def make(bucket_sort):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, cg_x0=3, bucket_sort=bucket_sort, **kw))
        sim.scene = sc
        return sim

    rm, rr = [], []
    merged, crossed = _run(make, 8, rm, bucket_sort=0)
    radix, _ = _run(make, 8, rr, bucket_sort=1)
    assert crossed > 0, "no particle changed its cell: the merge was not exercised"
    # the first build sorts from scratch; the (graph-run) builds after it merge
    assert rm[0]["bucket_merged"] == 0
    assert all(r["bucket_merged"] == 1 for r in rm[1:])
    assert all(r["bucket_merged"] == 0 for r in rr)
    assert sum(r["n_moved"] for r in rm[1:]) > 0
    _same(merged, radix)


def test_merged_order_ensemble():
    from paper_2105_01677_gb300 import mps
    # gentler than the single scenes: an ensemble has no direct search for particles that
    # outrun the cell skin (its smallest spacing is 0.005 m)
    E = [_stirred(s, 0.3, 20 + k, jitter=0.05)
         for k, s in enumerate(scenes.ensemble_2d(count=6, seed=4, fluid=(500, 2000)))]

    def make(bucket_sort):
        return mps.Ensemble(E, torch_alloc=True, use_torch_stream=True, precision=1, dt=1e-4,
                            cg_tol=1e-8, cg_x0=3, bucket_sort=bucket_sort)

    merged, _ = _run(make, 8, bucket_sort=0)
    radix, _ = _run(make, 8, bucket_sort=1)
    for a, b in zip(merged, radix):
        _same(a, b)


def test_write_state_starts_from_the_radix_sort():
    """A written state (slot = particle id again) is sorted from scratch, and the next
    steps merge again: the trajectory matches the radix sort's through the write."""
    from paper_2105_01677_gb300 import mps
    sc = _stirred(scenes.dam_break_2d(seed=5), 0.5, 14)
    out = []
    for bs in (0, 1):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, dt=1e-4, cg_x0=0, bucket_sort=bs))
        try:
            sim.step(3)
            st = sim.read()
            st["pos"][0] += 1e-6   # a different state: written, not skipped
            sim.write(st["pos"], st["vel"])
            sim.step(3)
            out.append(sim.read())
        finally:
            sim.close()
    _same([out[0]], [out[1]])


@pytest.mark.parametrize("speed, skin, merged", [(100.0, 1.0, 1), (300.0, 1.2, 0)])
def test_many_movers(speed, skin, merged):
    """The full 3D dam break, off its lattice, in a shear flow along x (0 at the bottom of
    the column in y to 100 or 300 m/s at its top; dt 5e-5, equation of state, cell skin 1 or
    1.2): 5,000-8,000 particles change cells per step (merged), or more than the 16,384
    movers the merge records (the radix sort takes over); either way the trajectory equals
    the radix sort's bit for bit."""
    from paper_2105_01677_gb300 import mps
    sc = _stirred(scenes.dam_break_3d(seed=9), 0.0, 15)   # off the lattice, at rest
    f = sc.types == scenes.FLUID
    y = sc.pos[f, 1]
    sc.vel[f, 0] = speed * (y - y.min()) / (y.max() - y.min())
    outs, reps = [], []
    for bs in (0, 1):
        sim = mps.Simulation(sc, torch_alloc=True, use_torch_stream=True,
                             **gpu_params(sc, precision=1, pressure_mode=1, dt=5e-5,
                                          cell_skin=skin, bucket_sort=bs))
        try:
            rr = [sim.step(1)[1] for _ in range(3)]
            outs.append(sim.read())
            reps.append(rr)
        finally:
            sim.close()
    assert all(r["bucket_merged"] == merged for r in reps[0][1:])
    if merged:
        assert all(1000 < r["n_moved"] <= 16384 for r in reps[0][1:])
    else:
        assert all(r["n_moved"] > 16384 for r in reps[0][1:])
    _same([outs[0]], [outs[1]])
