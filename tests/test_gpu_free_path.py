"""GPU parity of the free path of Algorithm 1 (the Spheres benchmark of Sec. 3.4) against the
oracle's o_free_path: T within 1e-9 mm (+1e-12 relative), segment counts and escapes exact."""
import numpy as np
import pytest

import oracle
import synth
from synth.materials import toy_materials
from gpu_common import to_soa

pytestmark = pytest.mark.gpu

MODES = [0, 1, 2]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_5235_gb300 import build
    build.build()
    import paper_1209_5235_gb300 as g4
    from synth.mlp_init import mlp_init
    ctx = g4.g4n_create(0)
    g4.g4n_mlp_load(ctx, mlp_init(7))
    sc = synth.scenes.spheres_scene()
    og = oracle.Geometry(sc)
    gid = g4.build_scene(ctx, sc)
    yield g4, torch, ctx, og, gid
    g4.g4n_destroy(ctx)


def _gpu(env, p, v, Y, E, mode, gid=None, counters=None):
    g4, torch, ctx, og, gid0 = env
    T, st = g4.g4n_free_path(ctx, gid0 if gid is None else gid, to_soa(p, torch), to_soa(v, torch),
                             torch.tensor(Y, dtype=torch.float64, device="cuda"), E, mode=mode, counters=counters)
    g4.g4n_sync(ctx)
    return T.cpu().numpy(), st.cpu().numpy()


def _compare(T, st, T_ref, st_ref):
    inf = np.isinf(T_ref)
    assert np.array_equal(np.isinf(T), inf), f"{np.sum(np.isinf(T) != inf)} escape mismatches"
    assert np.array_equal(st, st_ref.astype(np.int32)), f"{np.sum(st != st_ref)} segment-count mismatches"
    f = ~inf
    err = np.abs(T[f] - T_ref[f])
    assert np.all(err <= 1e-9 + 1e-12 * np.abs(T_ref[f])), f"max |dT| {err.max()}"


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("kind", ["regular", "random"])
def test_spheres_free_path_parity(env, kind, mode):
    """All 10^5 rays of the paper's Regular and Random inputs (full size)."""
    g4, torch, ctx, og, gid = env
    p, v, Y = synth.scenes.spheres_rays(kind)
    T_ref, st_ref, _ = og.free_path_many(p, v, synth.scenes.SPHERES_ENERGY, Y)
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    T, st = _gpu(env, p, v, Y, synth.scenes.SPHERES_ENERGY, mode, counters=cnt)
    _compare(T, st, T_ref, st_ref)
    c = g4.counters_dict(cnt)
    assert c["tracks"] == len(Y)
    assert c["escaped"] == int(np.isinf(T_ref).sum())
    assert c["phys_steps"] == int((np.isfinite(T_ref) & (T_ref > 0)).sum())
    assert c["steps"] == int(st_ref.sum())
    assert c["geom_steps"] == c["steps"] - c["phys_steps"]
    # both outcomes occur: rays absorbed in a ball and rays escaping between the balls
    assert 0 < np.isinf(T_ref).sum() < len(Y)


def test_regular_image_structure(env):
    """The Regular output is the 400 x 250 image (column-major ray order): every finite T lies in a
    ball on the ray, i.e. between the entry and exit of some sphere of radius 100 on the 250 mm grid."""
    g4, torch, ctx, og, gid = env
    p, v, Y = synth.scenes.spheres_rays("regular")
    T, _ = _gpu(env, p, v, Y, synth.scenes.SPHERES_ENERGY, 0)
    img = T.reshape(synth.scenes.SPHERES_GRID)
    assert img.shape == (400, 250)
    f = np.isfinite(T)
    x = p[f] + T[f, None] * v[f]
    c = np.round((x + 2375.0) / 250.0) * 250.0 - 2375.0
    r = np.linalg.norm(x - c, axis=1)
    assert np.all(r <= 100.0 + 1e-6)


def test_layered_closed_form(env):
    """Rays along +z through touching slabs of two materials (Eq. 8: piecewise-constant mu): T from the
    closed form of Eqs. 6-7, and equal to the oracle."""
    g4, torch, ctx, og0, gid0 = env
    m = toy_materials()
    th = [30.0, 50.0, 20.0, 40.0]
    mats = [m["lead"], m["water"], m["al"], m["scint"]]
    sc = synth.scenes.layered_scene(th, mats)
    og = oracle.Geometry(sc)
    gid = g4.build_scene(ctx, sc)
    E = 1.0
    mus = np.array([og.mu(k + 1, E)[0] for k in range(len(th))])
    rng = np.random.default_rng(3)
    n = 4000
    Y = rng.exponential(1.0, n) * 0.5
    p = np.column_stack([rng.uniform(-50, 50, n), rng.uniform(-50, 50, n), np.full(n, -5.0)])
    v = np.tile([0.0, 0.0, 1.0], (n, 1))
    T, st = _gpu(env, p, v, Y, E, 0, gid=gid)
    T_ref, st_ref, _ = og.free_path_many(p, v, E, Y)
    _compare(T, st, T_ref, st_ref)
    # closed form: 5 mm of vacuum, then the slabs
    edges = np.concatenate([[0.0], np.cumsum(th)])
    S = np.concatenate([[0.0], np.cumsum(mus * np.array(th))])
    k = np.searchsorted(S, Y, side="right") - 1
    inside = k < len(th)
    T_cf = 5.0 + edges[k[inside]] + (Y[inside] - S[k[inside]]) / mus[k[inside]]
    assert np.allclose(T[inside], T_cf, rtol=1e-12, atol=1e-9)
    assert np.all(np.isinf(T[~inside]))


def test_free_path_edge_cases(env):
    g4, torch, ctx, og, gid = env
    p = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [9000.0, 0.0, 0.0], [0.0, 0.0, 0.0], [2375.0, 2375.0, 2375.0]])
    v = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.0, 1.0]])
    Y = np.array([0.0, -1.0, 1.0, 50.0, 1e-12])
    T, st = _gpu(env, p, v, Y, 1.0, 0)
    T_ref, st_ref, _ = og.free_path_many(p, v, 1.0, Y)
    _compare(T, st, T_ref, st_ref)
    assert T[0] == 0.0 and T[1] == 0.0       # Y <= 0: the interaction is at the start
    assert np.isinf(T[2])                     # starts outside the world
    # empty input
    T0, _ = g4.g4n_free_path(ctx, gid, torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                             torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                             torch.zeros(0, dtype=torch.float64, device="cuda"), 1.0)
    assert T0.numel() == 0
    # a non-unit direction: NaN and an argument error at sync
    pb = to_soa(np.zeros((2, 3)), torch)
    vb = to_soa(np.array([[0.0, 0.0, 2.0], [0.0, 0.0, 1.0]]), torch)
    T2, _ = g4.g4n_free_path(ctx, gid, pb, vb, torch.ones(2, dtype=torch.float64, device="cuda"), 1.0)
    with pytest.raises(g4.G4NError):
        g4.g4n_sync(ctx)
    T2 = T2.cpu().numpy()
    assert np.isnan(T2[0]) and not np.isnan(T2[1])
    with pytest.raises(g4.G4NError):
        g4.g4n_free_path(ctx, gid, pb, vb, torch.ones(2, dtype=torch.float64, device="cuda"), -1.0)
