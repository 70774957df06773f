"""Pins for the oracle's navigator: hand-built scenes with known answers, the
tie rules, and invariants on seeded random scenes checked against an
independent world-frame predicate (explicit rotation matrices, atan2 phi)."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.scenes import Scene, Solid, Placement, VoxelSpec, BOX, TUBE, ORB
from synth.materials import vacuum, toy_materials
from geomref import inside_strict, rot_matrix, random_unit

INF = math.inf


def handmade():
    m = toy_materials()
    mats = [m["water"], m["lead"], m["scint"]]
    solids = [Solid(BOX, (100.0, 100.0, 100.0)), Solid(BOX, (10.0, 10.0, 10.0)), Solid(ORB, (5.0,)),
              Solid(ORB, (3.0,)), Solid(BOX, (5.0, 5.0, 5.0))]
    places = [Placement(-1, 0, 0, (0, 0, 0)),
              Placement(0, 1, 1, (30.0, 0.0, 0.0)),          # 1: box A
              Placement(0, 2, 2, (-30.0, 0.0, 0.0)),         # 2: orb B
              Placement(1, 3, 2, (5.0, 0.0, 0.0)),           # 3: orb C inside A (world x in [32, 38])
              Placement(0, 4, 1, (0.0, 50.0, 0.0)),          # 4: box D
              Placement(0, 4, 2, (0.0, 50.0, 0.0))]          # 5: box E, same place as D (deliberate overlap)
    return Scene("handmade", mats, solids, places, VoxelSpec(mode="none"))


def test_locate_known_points(oracle_lib):
    g = oracle.Geometry(handmade())
    z = [1.0, 0.0, 0.0]
    assert g.locate([0, 0, 0], z)[0] == 1
    d, p = g.locate([30, 0, 0], z)
    assert d == 2 and list(p[:2]) == [0, 1]
    d, p = g.locate([35, 0, 0], z)
    assert d == 3 and list(p[:3]) == [0, 1, 3]
    d, p = g.locate([-30, 2, 0], z)
    assert d == 2 and p[1] == 2
    assert g.locate([150, 0, 0], z)[0] == 0
    d, p = g.locate([0, 50, 0], z)           # overlap: the lower placement index wins
    assert d == 2 and p[1] == 4


def test_compute_step_known(oracle_lib):
    g = oracle.Geometry(handmade())
    path = [0] + [-1] * 7
    assert g.compute_step(1, path, [0, 0, 0], [1, 0, 0]) == (20.0, 1, 20.0)
    s, lim, saf = g.compute_step(1, path, [0, 0, 0], [-1, 0, 0])
    assert (s, lim) == (25.0, 2)
    s, lim, _ = g.compute_step(1, path, [0, 0, 0], [0, 0, 1])
    assert (s, lim) == (100.0, -1)
    # two identical overlapping daughters: equal distances, the lower index wins
    s, lim, _ = g.compute_step(1, path, [0, 0, 0], [0, 1, 0])
    assert (s, lim) == (45.0, 4)
    # inside A: orb C ahead, A's face behind
    pa = [0, 1] + [-1] * 6
    assert g.compute_step(2, pa, [30, 0, 0], [1, 0, 0])[:2] == (2.0, 3)
    assert g.compute_step(2, pa, [30, 0, 0], [-1, 0, 0])[:2] == (10.0, -1)
    # physics wins only when strictly shorter; a tie goes to geometry
    assert g.compute_step(2, pa, [30, 0, 0], [1, 0, 0], proposed=1.5)[:2] == (1.5, -2)
    assert g.compute_step(2, pa, [30, 0, 0], [1, 0, 0], proposed=2.0)[:2] == (2.0, 3)


def test_relocate_after_steps(oracle_lib):
    g = oracle.Geometry(handmade())
    path = np.array([0] + [-1] * 7, dtype=np.int32)
    d, p = g.relocate(path, 1, [20.0, 0, 0], [1, 0, 0])      # on A's face moving in
    assert d == 2 and p[1] == 1
    d, p = g.relocate(np.array([0, 1, 3] + [-1] * 5, dtype=np.int32), 3, [38.0, 0, 0], [1, 0, 0])
    assert d == 2 and list(p[:2]) == [0, 1]                   # left C, still in A
    d, p = g.relocate(np.array([0, 1] + [-1] * 6, dtype=np.int32), 2, [40.0, 0, 0], [1, 0, 0])
    assert d == 1                                             # left A into the world
    d, p = g.relocate(np.array([0] + [-1] * 7, dtype=np.int32), 1, [100.0, 0, 0], [1, 0, 0])
    assert d == 0                                             # left the world


class WorldPredicate:
    """Which daughter of the world strictly contains a point (independent of the oracle)."""

    def __init__(self, scene):
        self.items = []
        for i, pl in enumerate(scene.placements):
            if pl.mother != 0:
                continue
            s = scene.solids[pl.solid]
            R = rot_matrix(*pl.rot)
            self.items.append((i, s.kind, s.params, R, np.array(pl.t)))

    def region(self, q):
        q = np.atleast_2d(q)
        out = np.full(q.shape[0], 0)
        for i, kind, par, R, t in self.items:
            loc = (q - t) @ R            # R^T (q - t) row-wise
            out = np.where((out == 0) & inside_strict(kind, par, loc), i, out)
        return out


def mixed_scene(seed=5, n=60):
    rng = np.random.default_rng(seed)
    m = toy_materials()
    dsol, dpl = synth.scenes.random_world(rng, n, world_half=200.0, fill=0.15)
    solids = [Solid(BOX, (200.0, 200.0, 200.0))] + dsol
    places = [Placement(-1, 0, 0, (0, 0, 0))] + [Placement(0, i + 1, 1 + i % 2, t, rot) for i, (t, rot) in enumerate(dpl)]
    return Scene("mixed", [m["water"], m["lead"], m["scint"]], solids, places, VoxelSpec(mode="smart"))


def test_step_matches_world_march(oracle_lib):
    """compute_step from random points equals the first region change found by marching the
    independent world-frame predicate (pins transforms, rotations and all solid types)."""
    sc = mixed_scene()
    g = oracle.Geometry(sc)
    pred = WorldPredicate(sc)
    rng = np.random.default_rng(6)
    checked = 0
    for _ in range(300):
        p = rng.uniform(-180, 180, 3)
        v = random_unit(rng, 1)[0]
        depth, path = g.locate(p, v)
        reg = pred.region(p)[0]
        assert (path[depth - 1] if depth > 1 else 0) == reg
        s, lim, saf = g.compute_step(depth, path, p, v)
        # march the predicate: the region must not change before s and must change right after
        ts = np.linspace(0.0, s, 400)[1:-1]
        assert np.all(pred.region(p[None, :] + ts[:, None] * v[None, :]) == reg)
        after = p + (s + 1e-6) * v
        if np.all(np.abs(after) < 200.0):
            nreg = pred.region(after)[0]
            if lim >= 0:
                assert nreg == lim
            else:
                assert nreg != reg
        # isotropic safety: a ball of that radius stays in the region
        q = p[None, :] + 0.999999 * saf * random_unit(rng, 32)
        assert np.all(pred.region(q) == reg)
        checked += 1
    assert checked == 300


def test_locate_relocate_invariants(oracle_lib):
    """After any step: relocate-with-hint == locate-from-root; a daughter limiter is entered;
    locate of a strictly interior point is stable under +-tol jitter."""
    for sc in (mixed_scene(), synth.scenes.tiny_scene()):
        g = oracle.Geometry(sc)
        rng = np.random.default_rng(7)
        entered = 0
        half = sc.solids[0].params[0] * 0.9
        for _ in range(400):
            p = rng.uniform(-half, half, 3)
            v = random_unit(rng, 1)[0]
            if rng.uniform() < 0.5:   # aim at a daughter
                t = np.array(sc.placements[int(rng.integers(1, sc.n_volumes))].t) + rng.uniform(-3, 3, 3)
                if np.linalg.norm(t - p) > 0:
                    v = (t - p) / np.linalg.norm(t - p)
            depth, path = g.locate(p, v)
            s, lim, saf = g.compute_step(depth, path, p, v)
            x = p + s * v
            nd, npath = g.relocate(path, depth, x, v)
            rd, rpath = g.locate(x, v)
            assert nd == rd and np.array_equal(npath, rpath)
            if lim >= 0:
                assert lim in list(npath[:nd])
                entered += 1
            if saf > 1e-6:
                for _ in range(3):
                    jd, jp = g.locate(p + rng.uniform(-1e-9, 1e-9, 3), random_unit(rng, 1)[0])
                    assert jd == depth and np.array_equal(jp, path)
        assert entered > 50


def test_free_path_algorithm1_closed_form(oracle_lib):
    """Algorithm 1 / Eq. 7 on a stack of slabs: T = t_M + (Y - S_M) / mu_{M+1}, exactly."""
    mats = [synth.materials.constant_material(f"m{k}", 1.0, mu) for k, mu in enumerate([0.01, 0.5, 0.0, 0.2])]
    th = [30.0, 4.0, 10.0, 25.0]
    sc = synth.scenes.layered_scene(th, mats)
    g = oracle.Geometry(sc)
    mus = [0.01, 0.5, 0.0, 0.2]
    bounds = np.cumsum([0.0] + th)
    def G_inv(Y):
        S = 0.0
        for k in range(4):
            seg = th[k] * mus[k]
            if mus[k] > 0 and S + seg >= Y:
                return bounds[k] + (Y - S) / mus[k]
            S += seg
        return INF
    for Y in [0.0, 1e-3, 0.1, 0.3, 0.29999, 2.29, 2.3, 2.31, 7.0, 7.3, 7.31, 50.0]:
        T, _ = g.free_path([1.0, 2.0, -5.0], [0.0, 0.0, 1.0], 1.0, Y)
        ref = G_inv(Y) + 5.0 if G_inv(Y) < INF else INF
        if Y == 0.0:
            ref = 0.0
        assert (T == ref) or abs(T - ref) < 1e-12 * max(1.0, ref), (Y, T, ref)
