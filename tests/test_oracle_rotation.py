"""Pins for the oracle's Compton direction change and for its per-step trace.

The new direction after a scatter is fixed by the mathematics: a unit vector at
polar angle theta from the old one, cos theta = 1 - (E / E' - 1) m_e c^2 / E
(Compton's relation, which Kahn's method samples through eta = E / E'), at an
azimuth that is uniform about the old direction.  The rotation turns a frame
(e1, e2, u) into the new direction; here the azimuth is measured in a frame
built independently (cross products with a fixed axis), where a right-handed
rotation shows as a constant offset from the input azimuth and a mirrored one
as a sign flip.

The trace is the transport loop itself run with a recorder; its records,
hashed with the published FNV-1a (pinned by its test vectors), must give the
history hash and step count that the transport reports.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import synth
from synth.materials import ME_C2_MEV

EV_NONE, EV_PHOTO, EV_COMPTON, EV_CUTOFF, EV_ESCAPE, EV_PUSH = 0, 1, 2, 3, 4, 5


def frame(u):
    """An orthonormal right-handed frame (e1, e2, u) built from a fixed axis, independent of the oracle's."""
    u = np.asarray(u, dtype=float)
    a = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.6 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    return e1, e2


def azimuth_in(u, w):
    e1, e2 = frame(u)
    return math.atan2(float(np.dot(w, e2)), float(np.dot(w, e1)))


def wrap(x):
    return (x + math.pi) % (2.0 * math.pi) - math.pi


def random_units(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


@pytest.mark.parametrize("case", ["random", "plus_z", "minus_z", "near_z"])
def test_rotation_polar_angle_norm_and_handedness(oracle_lib, case):
    rng = np.random.default_rng(11)
    if case == "random":
        us = random_units(rng, 200)
    elif case == "plus_z":
        us = np.array([[0.0, 0.0, 1.0]])
    elif case == "minus_z":
        us = np.array([[0.0, 0.0, -1.0]])
    else:
        us = np.array([[1e-9, -2e-9, 1.0], [3e-12, 1e-12, -1.0], [0.0, 1e-300, 1.0]])
        us /= np.linalg.norm(us, axis=1)[:, None]
    for u in us:
        offsets = []
        for ct in (-1.0, -0.7, -0.2, 0.0, 0.35, 0.9, 0.999999, 1.0):
            for phi in np.linspace(-3.0, 3.0, 7):
                w = oracle.rotate(u, ct, math.cos(phi), math.sin(phi))
                assert abs(np.linalg.norm(w) - 1.0) < 1e-15 * 4
                assert abs(float(np.dot(u, w)) - ct) < 1e-14
                if abs(ct) < 0.999:
                    offsets.append(wrap(azimuth_in(u, w) - phi))
        # one constant offset for every input azimuth: the rotation is right-handed about u
        offsets = np.array(offsets)
        assert np.max(np.abs(np.array([wrap(o - offsets[0]) for o in offsets]))) < 1e-12


def test_rotation_mirror_would_fail(oracle_lib):
    """The handedness check separates a rotation from its mirror image (the test above is not vacuous)."""
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    phis = np.linspace(-3.0, 3.0, 9)
    w = [oracle.rotate(u, 0.2, math.cos(p), math.sin(p)) for p in phis]
    mirrored = [x - 2.0 * np.dot(x, frame(u)[1]) * frame(u)[1] for x in w]   # reflect across the (e1, u) plane
    off = [wrap(azimuth_in(u, m) - p) for m, p in zip(mirrored, phis)]
    assert np.max(np.abs([wrap(o - off[0]) for o in off])) > 0.1


def scatters(scene, source, seed, tids):
    """(u before, u after, E before, E after) of every Compton scatter followed by another step."""
    g = oracle.Geometry(scene)
    out = []
    for tid in tids:
        tr = g.trace(source, seed, int(tid))
        for k in np.nonzero(tr["event"][:-1] == EV_COMPTON)[0]:
            out.append((tr["dir"][k], tr["dir"][k + 1], tr["E"][k], tr["E"][k + 1]))
    return out


def test_transport_scatters_follow_compton_relation(oracle_lib):
    """Every scatter of the tiny scene's histories: |u'| = 1, u.u' = 1 - (E/E' - 1) m c^2 / E, and the azimuth of u'
    about u (in the independent frame) uniform on (-pi, pi] (KS)."""
    sc, src = synth.scenes.tiny_scene(), synth.scenes.tiny_source()
    seed = synth.scenes.CONFIG_SEEDS[0][1]
    sc_list = scatters(sc, src, seed, range(600))
    assert len(sc_list) > 1500
    az = []
    for u, w, E, E1 in sc_list:
        assert abs(np.linalg.norm(w) - 1.0) < 1e-14
        ct = 1.0 - (E / E1 - 1.0) * ME_C2_MEV / E
        assert abs(float(np.dot(u, w)) - ct) < 1e-11
        az.append(azimuth_in(u, w))
    assert stats.kstest(np.array(az), stats.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-3


def test_isotropic_source_directions_uniform_on_sphere(oracle_lib):
    """The source's isotropic direction (cos theta uniform, the disc azimuth) -- the same azimuth sampler the
    scatter uses: cos theta and the azimuth uniform (KS)."""
    src = synth.scenes.tiny_source()
    _, d, _ = oracle.source_sample(src, 123, 4000)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    assert stats.kstest(d[:, 2], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(phi, stats.uniform(loc=-math.pi, scale=2 * math.pi).cdf).pvalue > 1e-3


def fnv_records(records):
    return oracle.fnv1a(np.ascontiguousarray(records, dtype="<i4").tobytes())


@pytest.mark.parametrize("scene_name", ["tiny", "barrel", "calorimeter"])
def test_trace_reproduces_transport(oracle_lib, scene_name):
    """The trace's hashed records give the transport's history hash; its step count and path length are the
    transport's; its steps chain (position after a step = position before the next, up to the push of
    100 tol), and every step record with event 'none' names the leaf of the next state."""
    if scene_name == "tiny":
        sc, src, seed = synth.scenes.tiny_scene(), synth.scenes.tiny_source(), synth.scenes.CONFIG_SEEDS[0][1]
    elif scene_name == "barrel":
        sc, src, seed = synth.scenes.barrel_scene(), synth.scenes.barrel_source(), synth.scenes.CONFIG_SEEDS[3][1]
    else:
        sc, src, seed = (synth.scenes.calorimeter_scene(), synth.scenes.calorimeter_source(),
                         synth.scenes.CONFIG_SEEDS[1][1])
    g = oracle.Geometry(sc)
    tol = oracle.lib().o_tolerance()
    for tid in range(0, 400, 7):
        r = g.transport(src, seed, 1, tid0=tid)
        tr = g.trace(src, seed, tid)
        assert fnv_records(tr["records"]) == tr["hash"] == int(r["hashes"][0])
        assert tr["n_steps"] == len(tr["step"]) == int(r["counters"][1])
        assert tr["length"] == float(r["lengths"][0])
        n = len(tr["step"])
        for k in range(n - 1):
            moved = tr["pos"][k] + tr["step"][k] * tr["dir"][k]
            assert np.max(np.abs(tr["pos"][k + 1] - moved)) <= 100 * tol + 1e-9
        # one record per step besides the push records: its limiter and event are the step's, and after a
        # crossing its leaf is the volume of the next step
        rec = tr["records"][(tr["records"][:, 2] != EV_PUSH) & (tr["records"][:, 2] != 6)]
        assert len(rec) == n
        assert np.array_equal(rec[:, 1], tr["limiter"]) and np.array_equal(rec[:, 2], tr["event"])
        for k in range(n - 1):
            if tr["event"][k] == EV_NONE:
                assert rec[k, 0] == tr["path"][k + 1][tr["depth"][k + 1] - 1]
