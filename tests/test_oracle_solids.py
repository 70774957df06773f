"""Pins for the oracle's solids (local frame): closed forms, interval arithmetic,
march + bisection on an independent strict-inside predicate, safety bounds and
the direction-aware surface rule."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.scenes import Scene, Solid, Placement, VoxelSpec
from synth.materials import vacuum
from geomref import (BOX, TUBE, ORB, CONE, inside_strict, first_entry_closed_form, first_exit_closed_form,
                     march_entry, march_exit, random_unit)

TOL = 1e-9
INF = math.inf


def lab(solids):
    """Oracle geometry whose solid k+1 is solids[k] (solid 0 is an unused world box)."""
    sc = Scene("lab", [vacuum()], [Solid(BOX, (1e4, 1e4, 1e4))] + list(solids), [Placement(-1, 0, 0, (0, 0, 0))],
               VoxelSpec(mode="none"))
    return oracle.Geometry(sc)


def test_box_closed_forms(oracle_lib):
    g = lab([Solid(BOX, (1.0, 2.0, 3.0))])
    assert g.solid_dist_in(1, [-10, 0, 0], [1, 0, 0]) == 9.0
    assert g.solid_dist_in(1, [0, 10, 0], [0, -1, 0]) == 8.0
    assert g.solid_dist_in(1, [-10, 5, 0], [1, 0, 0]) == INF          # misses in y
    assert g.solid_dist_in(1, [-10, 0, 0], [-1, 0, 0]) == INF         # moving away
    d = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    assert abs(g.solid_dist_in(1, [-3, -3, 0], d) - 2 * math.sqrt(2)) < 1e-15 * 10
    assert g.solid_dist_out(1, [0, 0, 0], [1, 0, 0]) == 1.0
    assert g.solid_dist_out(1, [0, 0, 0], [0, 0, -1]) == 3.0
    assert abs(g.solid_dist_out(1, [0.5, 0, 0], d) - 0.5 * math.sqrt(2)) < 1e-15 * 10
    assert g.solid_safety_in(1, [5, 0, 0]) == 4.0
    assert g.solid_safety_out(1, [0.25, 0, 0]) == 0.75


def test_box_surface_rule(oracle_lib):
    g = lab([Solid(BOX, (1.0, 1.0, 1.0))])
    on = [1.0, 0.2, 0.3]
    assert g.solid_inside(1, on, [-1, 0, 0])          # entering through +x face
    assert not g.solid_inside(1, on, [1, 0, 0])       # leaving
    assert not g.solid_inside(1, on, [0, 1, 0])       # tangent
    assert g.solid_inside(1, [1 + 0.4 * TOL, 0, 0], [-1, 0, 0])
    assert not g.solid_inside(1, [1 + 0.6 * TOL, 0, 0], [-1, 0, 0])
    edge = [1.0, 1.0, 0.0]
    assert g.solid_inside(1, edge, [-0.6, -0.8, 0])
    assert not g.solid_inside(1, edge, [-0.6, 0.8, 0])
    # from a surface point that is not inside, DistanceToIn ignores the surface itself
    assert g.solid_dist_in(1, on, [1, 0, 0]) == INF
    assert g.solid_dist_in(1, on, [0, 1, 0]) == INF


def test_orb_closed_forms(oracle_lib):
    g = lab([Solid(ORB, (2.0,))])
    assert g.solid_dist_in(1, [-10, 0, 0], [1, 0, 0]) == 8.0
    b = 1.2
    assert abs(g.solid_dist_in(1, [-10, b, 0], [1, 0, 0]) - (10 - math.sqrt(4 - b * b))) < 1e-14
    assert g.solid_dist_in(1, [-10, 2.5, 0], [1, 0, 0]) == INF
    assert g.solid_dist_out(1, [0, 0, 0], [0, 1, 0]) == 2.0
    assert abs(g.solid_dist_out(1, [1, 0, 0], [0, 1, 0]) - math.sqrt(3)) < 1e-15 * 10
    assert g.solid_safety_in(1, [0, 5, 0]) == 3.0
    assert g.solid_safety_out(1, [0, 0.5, 0]) == 1.5
    assert g.solid_inside(1, [2, 0, 0], [-1, 0.1, 0])
    assert not g.solid_inside(1, [2, 0, 0], [0, 1, 0])


FULL_TUBES = [(0.0, 3.0, 4.0, 0.0, 2 * math.pi), (1.5, 3.0, 4.0, 0.0, 2 * math.pi)]


@pytest.mark.parametrize("par", FULL_TUBES + [(0.0, 2.0, 2.0, 0, 0), (0.0, 1.0, 1.0, 0, 0)])
def test_closed_form_distances_random(oracle_lib, par):
    """Random rays: box/orb/full tube (hollow or solid) against interval arithmetic."""
    if par[3:] == (0, 0):
        kind, p_ = (BOX, (2.0, 1.5, 2.5)) if par[0] == 0.0 and par[1] == 2.0 else (ORB, (2.2,))
    else:
        kind, p_ = TUBE, par
    g = lab([Solid(kind, p_)])
    rng = np.random.default_rng(1)
    n_hit = 0
    for _ in range(3000):
        p = rng.uniform(-8, 8, 3)
        if inside_strict(kind, p_, p):
            v = random_unit(rng, 1)[0]
            ref = first_exit_closed_form(kind, p_, p, v)
            assert abs(g.solid_dist_out(1, p, v) - ref) < 1e-11
            continue
        aim = rng.uniform(-3, 3, 3)
        v = (aim - p) / np.linalg.norm(aim - p)
        ref, chord = first_entry_closed_form(kind, p_, p, v)
        got = g.solid_dist_in(1, p, v)
        if ref == INF:
            assert got == INF
        elif chord > 1e-6:
            n_hit += 1
            assert abs(got - ref) < 1e-11, (p, v, got, ref)
    assert n_hit > 500


SEGMENTS = [(0.0, 3.0, 2.0, 0.3, 1.1), (1.0, 3.0, 2.0, -0.5, 2.5), (1.2, 2.5, 1.5, 2.0, 4.5),
            (0.0, 2.0, 1.0, 1.0, math.pi)]


@pytest.mark.parametrize("par", SEGMENTS)
def test_tube_segment_vs_march(oracle_lib, par):
    """Tube segments (narrow, wide, pi): DistanceToIn/Out against a march + bisection on atan2 phi."""
    g = lab([Solid(TUBE, par)])
    pred = lambda q: inside_strict(TUBE, par, q)
    rng = np.random.default_rng(2)
    n_in = n_out = 0
    while n_out < 60:
        p = rng.uniform(-3.2, 3.2, 3)
        if not pred(p):
            continue
        v = random_unit(rng, 1)[0]
        ref = march_exit(pred, p, v, 20.0, 0.01)
        got = g.solid_dist_out(1, p, v)
        assert abs(got - ref) < 1e-9, (p, v, got, ref)
        n_out += 1
    for _ in range(400):
        p = rng.uniform(-5, 5, 3)
        if pred(p):
            continue
        aim = rng.uniform(-2.5, 2.5, 3)
        v = (aim - p) / np.linalg.norm(aim - p)
        ref, chord = march_entry(pred, p, v, 20.0, 0.01)
        got = g.solid_dist_in(1, p, v)
        if ref == INF:
            # only grazes thinner than the march step may be seen by the oracle
            if got != INF:
                assert g.solid_dist_out(1, p + got * v, v) < 0.02
        elif chord > 1e-3:
            assert abs(got - ref) < 1e-9, (p, v, got, ref)
            n_in += 1
    assert n_in > 50 and n_out > 20


CONES = [(0.0, 1.0, 0.0, 3.0, 2.0), (0.5, 3.0, 0.3, 1.0, 1.5), (1.0, 2.0, 1.2, 2.5, 3.0), (0.0, 3.0, 0.0, 0.3, 0.5)]


@pytest.mark.parametrize("kind,par", [(BOX, (2.0, 1.0, 0.5)), (ORB, (1.5,)), (TUBE, (0.5, 2.0, 1.0, 0.0, 2 * math.pi))]
                         + [(TUBE, s) for s in SEGMENTS] + [(CONE, c) for c in CONES])
def test_safety_is_lower_bound(oracle_lib, kind, par):
    g = lab([Solid(kind, par)])
    pred = lambda q: inside_strict(kind, par, q)
    rng = np.random.default_rng(3)
    dirs = random_unit(rng, 64)
    for _ in range(150):
        p = rng.uniform(-4, 4, 3)
        if pred(p):
            s = g.solid_safety_out(1, p)
            assert s >= 0.0
            # the ball of radius s stays inside
            q = p + 0.999999 * s * dirs
            assert np.all(pred(q))
            for v in dirs[:16]:
                assert s <= g.solid_dist_out(1, p, v) + 1e-12
        else:
            s = g.solid_safety_in(1, p)
            q = p + 0.999999 * s * dirs
            assert not np.any(pred(q))
            for v in dirs[:16]:
                assert s <= g.solid_dist_in(1, p, v) + 1e-12


def test_tube_surface_rule(oracle_lib):
    g = lab([Solid(TUBE, (1.0, 2.0, 3.0, 0.0, math.pi / 2))])
    assert g.solid_inside(1, [2.0 * math.cos(0.5), 2.0 * math.sin(0.5), 0], [-1, 0, 0])   # rmax, inward
    assert not g.solid_inside(1, [2.0 * math.cos(0.5), 2.0 * math.sin(0.5), 0], [1, 0, 0])
    assert g.solid_inside(1, [math.cos(0.5), math.sin(0.5), 0], [1, 1, 0])                # rmin, outward radially
    assert not g.solid_inside(1, [math.cos(0.5), math.sin(0.5), 0], [-1, -1, 0])
    assert g.solid_inside(1, [1.5, 0.0, 0], [0, 1, 0])                                     # start plane, into wedge
    assert not g.solid_inside(1, [1.5, 0.0, 0], [0, -1, 0])
    assert g.solid_inside(1, [0.0, 1.5, 0], [1, 0, 0])                                     # end plane
    assert not g.solid_inside(1, [0.0, 1.5, 0], [-1, 0, 0])
    assert g.solid_inside(1, [1.0, 1.0, 3.0], [0, 0, -1])                                  # z plane
    assert not g.solid_inside(1, [1.0, 1.0, 3.0], [0, 0, 1])
    assert not g.solid_inside(1, [-1.5, 0.0, 0], [0, 1, 0])                                # outside phi range
    # exact plane crossing distances
    assert abs(g.solid_dist_in(1, [1.5, -1.0, 0], [0, 1, 0]) - 1.0) < 1e-15
    assert abs(g.solid_dist_out(1, [1.5, 0.5, 0], [-1, 0, 0]) - (1.5 - math.sqrt(0.75))) < 1e-15 * 10


def test_rejects_bad_solids(oracle_lib):
    L = oracle.lib()
    g = lab([])
    for kind, par in [(BOX, [0, 1, 1, 0, 0]), (ORB, [-1, 0, 0, 0, 0]), (TUBE, [2, 1, 1, 0, 1]),
                      (TUBE, [0, 1, 1, 0, 7.0]), (TUBE, [0, 1, 0, 0, 1])]:
        a = np.array(par, dtype=np.float64)
        assert L.o_add_solid(g.gid, kind, a.ctypes.data) < 0


@pytest.mark.parametrize("rmin,rmax,hz", [(0.0, 2.0, 1.5), (0.7, 2.0, 1.5)])
def test_cone_with_equal_ends_is_the_tube(oracle_lib, rmin, rmax, hz):
    """A cone whose end radii are equal is the (pinned) full tube: same answers on random points and rays."""
    g = lab([Solid(CONE, (rmin, rmax, rmin, rmax, hz)), Solid(TUBE, (rmin, rmax, hz, 0.0, 2 * math.pi))])
    rng = np.random.default_rng(8)
    for _ in range(3000):
        p = rng.uniform(-3, 3, 3)
        v = random_unit(rng, 1)[0]
        assert g.solid_inside(1, p, v) == g.solid_inside(2, p, v)
        if g.solid_inside(1, p, v):
            assert g.solid_dist_out(1, p, v) == pytest.approx(g.solid_dist_out(2, p, v), rel=1e-13, abs=1e-13)
            assert g.solid_safety_out(1, p) == pytest.approx(g.solid_safety_out(2, p), rel=1e-13, abs=1e-13)
        else:
            a, b = g.solid_dist_in(1, p, v), g.solid_dist_in(2, p, v)
            assert (a == INF and b == INF) or a == pytest.approx(b, rel=1e-13, abs=1e-13)
            assert g.solid_safety_in(1, p) == pytest.approx(g.solid_safety_in(2, p), rel=1e-13, abs=1e-13)


def test_cone_closed_forms(oracle_lib):
    g = lab([Solid(CONE, (0.0, 1.0, 0.0, 3.0, 2.0)), Solid(CONE, (1.0, 2.0, 0.5, 3.0, 1.0))])
    # along the axis: the end faces
    assert g.solid_dist_in(1, [0, 0, -10], [0, 0, 1]) == 8.0
    assert g.solid_dist_out(1, [0, 0, 0.5], [0, 0, 1]) == 1.5
    # in the plane z = 0 the outer radius is the mean of the end radii
    assert abs(g.solid_dist_out(1, [0, 0, 0], [1, 0, 0]) - 2.0) < 1e-15
    assert abs(g.solid_dist_in(1, [-10, 0, 0], [1, 0, 0]) - 8.0) < 1e-14
    # hollow cone at z = 0: inner radius 0.75, outer 2.5; from the axis the ray enters at the inner cone
    assert abs(g.solid_dist_in(2, [0, 0, 0], [0, 1, 0]) - 0.75) < 1e-15
    assert abs(g.solid_dist_out(2, [0, 1.0, 0], [0, 1, 0]) - 1.5) < 1e-15
    assert abs(g.solid_dist_out(2, [0, 1.0, 0], [0, -1, 0]) - 0.25) < 1e-15
    # the outer surface of solid 1 is r = z / 2 + 2; the ray r = z from the origin would meet it at z = 4,
    # beyond the +z face, so it leaves through that face
    v = np.array([1.0, 0.0, 1.0]) / math.sqrt(2)
    t = g.solid_dist_out(1, [0, 0, 0], v)
    q = np.array([0, 0, 0]) + t * v
    assert abs(q[2] - 2.0) < 1e-14
    # safety at the origin: the perpendicular distance to the line r = z / 2 + 2, 2 / sqrt(1.25)
    assert abs(g.solid_safety_out(1, [0, 0, 0]) - 2.0 / math.sqrt(1.25)) < 1e-15


@pytest.mark.parametrize("par", CONES)
def test_cone_vs_march(oracle_lib, par):
    """Cones (solid, hollow, widening, narrowing, flat): DistanceToIn/Out against a march + bisection on an
    independent strict-inside predicate."""
    g = lab([Solid(CONE, par)])
    pred = lambda q: inside_strict(CONE, par, q)
    rng = np.random.default_rng(4)
    ext = max(par[1], par[3], par[4]) * 1.1
    n_in = n_out = 0
    tries = 0
    while n_out < 60 and tries < 100000:
        tries += 1
        p = rng.uniform(-ext, ext, 3)
        if not pred(p):
            continue
        v = random_unit(rng, 1)[0]
        ref = march_exit(pred, p, v, 20.0, 0.01)
        got = g.solid_dist_out(1, p, v)
        assert abs(got - ref) < 1e-9, (p, v, got, ref)
        n_out += 1
    for _ in range(400):
        p = rng.uniform(-2 * ext, 2 * ext, 3)
        if pred(p):
            continue
        aim = rng.uniform(-0.8 * ext, 0.8 * ext, 3)
        v = (aim - p) / np.linalg.norm(aim - p)
        ref, chord = march_entry(pred, p, v, 30.0, 0.01)
        got = g.solid_dist_in(1, p, v)
        if ref == INF or got < ref - 1e-9:
            # the oracle found an entry the march stepped over: a chord thinner than the march step
            if got != INF:
                assert g.solid_dist_out(1, p + got * v, v) < 0.02
                assert pred(p + (got + 1e-7) * v) and not pred(p + (got - 1e-7) * v)
        elif chord > 1e-3:
            assert abs(got - ref) < 1e-9, (p, v, got, ref)
            n_in += 1
    assert n_in > 40 and n_out == 60


def test_cone_surface_rule(oracle_lib):
    g = lab([Solid(CONE, (0.5, 1.0, 1.5, 3.0, 2.0))])
    # outer surface r = 0.5 z + 2, inner r = 0.25 z + 1; outward normal of the outer one along (1, 0, -0.5)
    on_out = [2.0, 0.0, 0.0]
    assert g.solid_inside(1, on_out, [-1, 0, 0])
    assert not g.solid_inside(1, on_out, [1, 0, 0])
    assert g.solid_inside(1, on_out, [0, 0, 1])          # up the widening cone: v . n = -0.5 < 0
    assert not g.solid_inside(1, on_out, [0, 0, -1])
    assert not g.solid_inside(1, on_out, [0.5, 0, 1.0])  # along the surface's generator: tangent
    on_in = [1.0, 0.0, 0.0]
    assert g.solid_inside(1, on_in, [1, 0, 0])           # into the solid across the inner cone
    assert not g.solid_inside(1, on_in, [-1, 0, 0])
    assert g.solid_inside(1, [1.5, 0.0, 2.0], [0, 0, -1])  # end face
    assert not g.solid_inside(1, [1.5, 0.0, 2.0], [0, 0, 1])
    assert g.solid_inside(1, [2.0 + 0.4 * TOL, 0, 0], [-1, 0, 0])
    assert not g.solid_inside(1, [2.0 + 0.6 * TOL, 0, 0], [-1, 0, 0])


def test_rejects_bad_cones(oracle_lib):
    L = oracle.lib()
    g = lab([])
    for par in [(0, 1, 0, 1, 0), (1, 0.5, 0, 1, 1), (0, 1, 2, 1, 1), (0, 1, 0.5, 2, 1), (-1, 1, 0, 1, 1)]:
        a = np.array(par, dtype=np.float64)
        assert L.o_add_solid(g.gid, CONE, a.ctypes.data) < 0


@pytest.mark.parametrize("kind,par", [(BOX, (2.0, 1.0, 0.5)), (ORB, (1.5,)), (TUBE, (0.5, 2.0, 1.0, 0.0, 2 * math.pi))]
                         + [(TUBE, s) for s in SEGMENTS] + [(CONE, c) for c in CONES])
def test_reported_crossings_lie_on_the_surface(oracle_lib, kind, par):
    """At the exit DistanceToOut reports, the point belongs to the solid moving back and not moving on, and
    DistanceToOut from there is 0; at the entry DistanceToIn reports (chord > 1e-6), the reverse."""
    g = lab([Solid(kind, par)])
    pred = lambda q: inside_strict(kind, par, q)
    rng = np.random.default_rng(4)
    n_out = n_in = 0
    for _ in range(20000):
        if n_out >= 40:
            break
        p = rng.uniform(-3, 3, 3)
        if not pred(p):
            continue
        v = random_unit(rng, 1)[0]
        s = g.solid_dist_out(1, p, v)
        x = p + s * v
        assert g.solid_dist_out(1, x, v) <= 1e-9
        assert not g.solid_inside(1, x, v) and g.solid_inside(1, x, -v), (p, v, s)
        n_out += 1
    for _ in range(20000):
        if n_in >= 40:
            break
        p = rng.uniform(-5, 5, 3)
        if pred(p):
            continue
        aim = rng.uniform(-2, 2, 3)
        v = (aim - p) / np.linalg.norm(aim - p)
        t = g.solid_dist_in(1, p, v)
        if t == INF:
            continue
        y = p + t * v
        if g.solid_dist_out(1, y, v) < 1e-6:
            continue
        assert g.solid_inside(1, y, v) and not g.solid_inside(1, y, -v), (p, v, t)
        n_in += 1
    assert n_out == 40 and n_in == 40
