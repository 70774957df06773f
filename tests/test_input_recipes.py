"""The synthetic workloads have the shapes the documentation states (sizes, counts, seeds, sources),
so that a change of a generator cannot silently change what the tests and the bench run on."""
import math

import numpy as np
import pytest

from synth import scenes as S


def test_seeds_follow_the_config_index():
    for i in range(5):
        assert S.CONFIG_SEEDS[i] == (0x6E4A0000 + i, 0x7A0C0000 + i)


def test_tiny_world():
    sc = S.tiny_scene()
    assert sc.n_volumes == 11
    assert (sc.voxel.mode, tuple(sc.voxel.slices)) == ("fixed", (8, 8, 8))
    src = S.tiny_source()
    assert src.isotropic and src.e_kind == "mono" and src.e0 == 1.0 and tuple(src.pos) == (0.0, 0.0, 0.0)


def test_calorimeter():
    sc = S.calorimeter_scene()
    assert sc.n_volumes == 2 + 50 * 10 * 10
    cells = [p for p in sc.placements if p.mother == 1]
    assert len(cells) == 5000
    env = sc.solids[sc.placements[1].solid].params
    assert tuple(env) == (500.0, 500.0, 187.5)                 # 1000 x 1000 x 375 mm
    half_z = sorted({sc.solids[p.solid].params[2] for p in cells})
    assert half_z == [2.5, 5.0]                                 # 5 mm lead-like, 10 mm scintillator-like
    assert all(sc.solids[p.solid].params[:2] == (50.0, 50.0) for p in cells)
    src = S.calorimeter_source()
    assert (src.pos, src.spot_sigma, src.direction, src.e_kind, src.e0, src.e1) == \
        ((0.0, 0.0, -10.0), 10.0, (0.0, 0.0, 1.0), "uniform", 0.1, 10.0)


def test_batched_worlds():
    worlds = list(S.batched_scenes())
    assert len(worlds) == 256
    assert sum(sc.n_volumes for sc, _ in worlds) == 205_670
    n = [nt for _, nt in worlds]
    assert sum(n) == 5_649_656 and 1_000 <= min(n) and max(n) <= 100_000
    nd = [sc.n_volumes - 1 for sc, _ in worlds]
    assert 10 <= min(nd) and max(nd) <= 5000
    src = S.batched_source()
    assert src.isotropic and (src.e_kind, src.e0, src.e1) == ("loguniform", 0.05, 5.0)


@pytest.mark.parametrize("make", [S.barrel_scene, S.nested_barrel_scene])
def test_barrels(make):
    sc = make()
    assert sc.n_volumes == 1 + 30 + 30 * 64 + 2000            # world, shells, φ segments, orbs
    src = S.barrel_source()
    assert src.isotropic and tuple(src.z_range) == (-1500.0, 1500.0)
    assert (src.e_kind, src.e0, src.e1) == ("loguniform", 0.02, 20.0)


def test_spheres():
    sc = S.spheres_scene()
    assert sc.n_volumes == 8001
    c = np.array([p.t for p in sc.placements[1:]])
    assert c.min() == -2375.0 and c.max() == 2375.0
    assert sc.solids[1].params == (100.0,)
    pos, d, Y = S.spheres_rays("regular")
    assert pos.shape == (100_000, 3) and np.all(Y == 1.0)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    # ray i*250 + j aims at the centre of pixel (i, j) of the 400 x 250 grid on the +z face
    i, j = 123, 45
    t = 2500.0 / d[i * 250 + j, 2]
    assert math.isclose(t * d[i * 250 + j, 0], -2500.0 + (i + 0.5) * 5000.0 / 400, abs_tol=1e-9)
    assert math.isclose(t * d[i * 250 + j, 1], -2500.0 + (j + 0.5) * 5000.0 / 250, abs_tol=1e-9)
