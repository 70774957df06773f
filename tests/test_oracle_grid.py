"""The oracle's timing mode (uniform grids over the daughters of crowded mothers) gives the results of
its brute-force search: identical histories, counters and tallies on track subsets of every workload,
identical located paths and steps on random queries, identical free paths on the Spheres inputs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import mixed_scene, random_queries


def _pair(scene):
    brute, grid = oracle.Geometry(scene), oracle.Geometry(scene)
    grid.use_grids(True)
    return brute, grid


def _same_transport(scene, src, seed, n, tid0=0):
    brute, grid = _pair(scene)
    a = brute.transport(src, seed, n, tid0=tid0)
    b = grid.transport(src, seed, n, tid0=tid0)
    assert np.array_equal(a["hashes"], b["hashes"])
    assert np.array_equal(a["lengths"], b["lengths"])
    assert np.array_equal(a["counters"][:10], b["counters"][:10])
    assert np.allclose(a["tally"], b["tally"], rtol=1e-12, atol=0.0)
    # the grids pay: fewer DistanceToIn evaluations and Inside tests
    return int(a["counters"][10] + a["counters"][11]), int(b["counters"][10] + b["counters"][11])


@pytest.mark.parametrize("name", ["tiny", "calorimeter", "barrel", "nested_barrel", "mixed"])
def test_grid_transport_equals_brute_force(oracle_lib, name):
    if name == "tiny":
        sc, src, seed, n = synth.scenes.tiny_scene(), synth.scenes.tiny_source(), synth.scenes.CONFIG_SEEDS[0][1], 3000
    elif name == "calorimeter":
        sc, src, seed, n = (synth.scenes.calorimeter_scene(), synth.scenes.calorimeter_source(),
                            synth.scenes.CONFIG_SEEDS[1][1], 1500)
    elif name == "barrel":
        sc, src, seed, n = synth.scenes.barrel_scene(), synth.scenes.barrel_source(), synth.scenes.CONFIG_SEEDS[3][1], 3000
    elif name == "nested_barrel":
        sc, src, seed, n = (synth.scenes.nested_barrel_scene(), synth.scenes.barrel_source(),
                            synth.scenes.CONFIG_SEEDS[3][1], 2000)
    else:
        sc = mixed_scene(seed=3, n=400, half=300.0)
        src = synth.scenes.Source(pos=(1.0, 2.0, 3.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
        seed, n = 17, 3000
    e_brute, e_grid = _same_transport(sc, src, seed, n, tid0=123)
    if name in ("calorimeter", "mixed"):
        assert e_grid < 0.2 * e_brute, (e_grid, e_brute)


def test_grid_batched_worlds_equal_brute_force(oracle_lib):
    src, seed = synth.scenes.batched_source(), synth.scenes.CONFIG_SEEDS[2][1]
    for k, (sc, nt) in enumerate(synth.scenes.batched_scenes()):
        if k % 37:
            continue
        _same_transport(sc, src, seed, 300, tid0=1000 * k)


@pytest.mark.parametrize("name", ["calorimeter", "mixed"])
def test_grid_queries_equal_brute_force(oracle_lib, name):
    sc = synth.scenes.calorimeter_scene() if name == "calorimeter" else mixed_scene(seed=4, n=300, half=300.0)
    brute, grid = _pair(sc)
    box = (600.0, 600.0, 400.0) if name == "calorimeter" else None
    p, v = random_queries(brute, sc, 4000, seed=5, box_half=box)
    d1, p1 = brute.locate_many(p, v)
    d2, p2 = grid.locate_many(p, v)
    assert np.array_equal(d1, d2) and np.array_equal(p1, p2)
    ok = d1 > 0
    for k in np.nonzero(ok)[0][:1500]:
        a = brute.compute_step(d1[k], p1[k], p[k], v[k], safety=False)
        b_ = grid.compute_step(d1[k], p1[k], p[k], v[k], safety=False)
        assert a[0] == b_[0] and a[1] == b_[1]


def test_grid_free_path_equals_brute_force(oracle_lib):
    sc = synth.scenes.spheres_scene()
    brute, grid = _pair(sc)
    for kind in ("regular", "random"):
        p, v, Y = synth.scenes.spheres_rays(kind, seed=0x7A0C0005)
        idx = np.arange(0, len(Y), 50)
        T1, s1, _ = brute.free_path_many(p[idx], v[idx], synth.scenes.SPHERES_ENERGY, Y[idx])
        T2, s2, _ = grid.free_path_many(p[idx], v[idx], synth.scenes.SPHERES_ENERGY, Y[idx])
        assert np.array_equal(T1, T2) and np.array_equal(s1, s2)
