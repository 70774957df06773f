"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Located volume ids and limiters bit-exact, steps within
1e-9 mm, per-track history hashes bit-exact, tallies within 3 sigma."""
import math

import numpy as np
import pytest

import oracle
import synth
from synth.scenes import VoxelSpec, Source
from gpu_common import cones_scene, mixed_scene, nested_scene, random_queries, segments_scene, to_soa

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9


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
    g4.g4n_mlp_load(ctx, mlp_init(7))   # learned mode: any weights give the same results
    yield g4, torch, ctx
    g4.g4n_destroy(ctx)


SCENES = {
    "tiny": lambda: synth.scenes.tiny_scene(),
    "calorimeter": lambda: synth.scenes.calorimeter_scene(),
    "mixed_smart": lambda: mixed_scene(),
    "mixed_fixed": lambda: mixed_scene(voxel=VoxelSpec(mode="fixed", axes=(1, 2, 0), slices=(7, 5, 3))),
    "mixed_none": lambda: mixed_scene(voxel=VoxelSpec(mode="none")),
    "barrel": lambda: synth.scenes.barrel_scene(),
    "nested": lambda: nested_scene(),
    "nested_core": lambda: nested_scene(),
    "spheres": lambda: synth.scenes.spheres_scene(),
    "segments": lambda: segments_scene(),
    "nested_barrel": lambda: synth.scenes.nested_barrel_scene(),
    "cones": lambda: cones_scene(),
}
BOX_HALF = {"barrel": (1600.0, 1600.0, 1600.0), "nested_barrel": (1600.0, 1600.0, 1600.0), "calorimeter": (600.0, 600.0, 400.0), "nested_core": (12.0, 12.0, 12.0),
            "segments": (360.0, 360.0, 90.0)}
AIM = {"segments": 0.8, "mixed_smart": 0.3, "mixed_fixed": 0.3, "mixed_none": 0.3, "cones": 0.6}
EXACT_SAFETY = ("tiny", "calorimeter", "spheres")   # boxes aligned with their mother, orbs


def _build(env, name):
    g4, torch, ctx = env
    sc = SCENES[name]()
    return sc, oracle.Geometry(sc), g4.build_scene(ctx, sc)


@pytest.mark.parametrize("name", list(SCENES))
def test_locate_parity(env, name):
    g4, torch, ctx = env
    sc, og, gid = _build(env, name)
    n = 4000 if name in ("calorimeter", "spheres") else 20000
    p, v = random_queries(og, sc, n, seed=11, box_half=BOX_HALF.get(name), aim_frac=AIM.get(name, 0.0))
    d_ref, path_ref = og.locate_many(p, v)
    d, path = g4.g4n_locate(ctx, gid, to_soa(p, torch), to_soa(v, torch))
    g4.g4n_sync(ctx)
    d = d.cpu().numpy()
    path = path.cpu().numpy().T
    bad = np.nonzero((d != d_ref) | np.any(path != path_ref, axis=1))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first: {p[bad[0]]} {v[bad[0]]} gpu {path[bad[0]]} ref {path_ref[bad[0]]}"
    assert (d_ref >= 2).sum() > 0  # the cases do reach daughters
    if name == "nested_barrel":
        assert d_ref.max() == g4.G4N_DMAX  # the deepest level is reached


def _band_edge_points(sc, n, seed, half=0.5e-9):
    """Points within a few ulps of the edges of the +-half surface band of world-level boxes
    (and of the box centre planes' neighbours inside), on one, two or three axes at once,
    with directions that are often axis-parallel or have zero components."""
    rng = np.random.default_rng(seed)
    boxes = [(np.array(pl.t, dtype=np.float64), np.array(sc.solids[pl.solid].params[:3], dtype=np.float64))
             for pl in sc.placements[1:] if pl.mother == 0]
    p = np.empty((n, 3))
    v = rng.normal(size=(n, 3))
    for q in range(n):
        c, h = boxes[rng.integers(len(boxes))]
        x = c + rng.uniform(-0.9, 0.9, 3) * h
        for a in range(3):
            if a == 0 or rng.uniform() < 0.3:
                side = 1.0 if rng.uniform() < 0.5 else -1.0
                delta = (half, -half, 0.0)[rng.integers(3)]
                xa = c[a] + side * (h[a] + delta)
                k = int(rng.integers(-3, 4))
                for _ in range(abs(k)):
                    xa = np.nextafter(xa, np.inf if k > 0 else -np.inf)
                x[a] = xa
        p[q] = x
        for a in range(3):
            if rng.uniform() < 0.3:
                v[q, a] = 0.0
        if not np.any(v[q]):
            v[q, rng.integers(3)] = 1.0
    v /= np.linalg.norm(v, axis=1)[:, None]
    return p, v


@pytest.mark.parametrize("voxel", ["smart", "fixed", "none"])
def test_locate_band_edges(env, voxel):
    """Inside decisions on the edges of the surface band (x = c +- (h +- half), +-3 ulps): the
    GPU's exact-threshold box tests and voxel lookups agree with the oracle's FP64 tests."""
    g4, torch, ctx = env
    spec = {"smart": VoxelSpec(mode="smart"), "fixed": VoxelSpec(mode="fixed", axes=(0, 1, 2), slices=(9, 7, 5)),
            "none": VoxelSpec(mode="none")}[voxel]
    sc = synth.scenes.tiny_scene(seed=123, n_boxes=40, voxel=spec)
    og = oracle.Geometry(sc)
    gid = g4.build_scene(ctx, sc)
    p, v = _band_edge_points(sc, 30000, seed=5)
    d_ref, path_ref = og.locate_many(p, v)
    d, path = g4.g4n_locate(ctx, gid, to_soa(p, torch), to_soa(v, torch))
    g4.g4n_sync(ctx)
    d = d.cpu().numpy()
    path = path.cpu().numpy().T
    bad = np.nonzero((d != d_ref) | np.any(path != path_ref, axis=1))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first: {p[bad[0]]!r} {v[bad[0]]!r} gpu {path[bad[0]]} ref {path_ref[bad[0]]}"
    # both outcomes of the band rule occur
    assert 0 < (d_ref == 2).sum() < len(d_ref)


def test_locate_cone_bands(env):
    """Points around the conical surfaces and end faces of cones (offsets along r or z of 0, +-0.3, +-0.7, +-2 and +-3
    half-tolerances, i.e. on both sides of both band edges) with random directions: located paths agree with the oracle."""
    g4, torch, ctx = env
    from synth.scenes import CONE
    from synth.materials import toy_materials
    m = toy_materials()
    cones = [(0.0, 40.0, 0.0, 90.0, 60.0), (20.0, 70.0, 35.0, 50.0, 45.0), (15.0, 60.0, 5.0, 25.0, 30.0)]
    centres = [(-200.0, 0.0, 0.0), (0.0, 150.0, 50.0), (200.0, -100.0, -80.0)]
    rot = (math.cos(0.7), math.sin(0.7))
    solids = [synth.scenes.Solid(synth.scenes.BOX, (400.0, 400.0, 400.0))] + [synth.scenes.Solid(CONE, c) for c in cones]
    places = [synth.scenes.Placement(-1, 0, 0, (0.0, 0.0, 0.0))] + [
        synth.scenes.Placement(0, k + 1, 1, centres[k], rot) for k in range(len(cones))]
    sc = synth.scenes.Scene("cone_bands", [m["water"], m["lead"]], solids, places, VoxelSpec(mode="smart"))
    og = oracle.Geometry(sc)
    gid = g4.build_scene(ctx, sc)
    half = 0.5e-9
    rng = np.random.default_rng(17)
    pts, dirs = [], []
    offs = np.array([0.0, 0.3, -0.3, 0.7, -0.7, 2.0, -2.0, 3.0, -3.0]) * half
    for _ in range(4000):
        k = int(rng.integers(len(cones)))
        rmin1, rmax1, rmin2, rmax2, hz = cones[k]
        surf = int(rng.integers(3))          # outer cone, inner cone, end face
        off = offs[int(rng.integers(len(offs)))]
        ph = rng.uniform(0, 2 * math.pi)
        if surf == 2:
            zsign = 1.0 if rng.uniform() < 0.5 else -1.0
            z = zsign * hz + zsign * off
            ro, ri = (rmax2, rmin2) if zsign > 0 else (rmax1, rmin1)
            r = ri + (ro - ri) * rng.uniform(0.05, 0.95)
        else:
            z = rng.uniform(-0.95, 0.95) * hz
            ko, co = (rmax2 - rmax1) / (2 * hz), 0.5 * (rmax1 + rmax2)
            ki, ci = (rmin2 - rmin1) / (2 * hz), 0.5 * (rmin1 + rmin2)
            if surf == 1 and rmin1 == 0.0:
                surf = 0
            r = (ko * z + co + off) if surf == 0 else (ki * z + ci + off)
        local = np.array([r * math.cos(ph), r * math.sin(ph), z])
        c, s_ = rot
        world = np.array([c * local[0] - s_ * local[1], s_ * local[0] + c * local[1], local[2]]) + np.array(centres[k])
        pts.append(world)
        w = rng.normal(size=3)
        dirs.append(w / np.linalg.norm(w))
    p, v = np.array(pts), np.array(dirs)
    d_ref, path_ref = og.locate_many(p, v)
    d, path = g4.g4n_locate(ctx, gid, to_soa(p, torch), to_soa(v, torch))
    g4.g4n_sync(ctx)
    d = d.cpu().numpy()
    path = path.cpu().numpy().T
    bad = np.nonzero((d != d_ref) | np.any(path != path_ref, axis=1))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first: {p[bad[0]]!r} {v[bad[0]]!r} gpu {path[bad[0]]} ref {path_ref[bad[0]]}"
    assert 0.2 < (d_ref == 2).mean() < 0.8   # both sides of the surfaces occur


MODES = [0, 1, 2]   # G4N_MODE_FP64, G4N_MODE_FP32_RECHECK, G4N_MODE_LEARNED


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", list(SCENES))
def test_compute_step_parity(env, name, mode):
    g4, torch, ctx = env
    sc, og, gid = _build(env, name)
    n = 3000 if name in ("calorimeter", "spheres") else 20000
    p, v = random_queries(og, sc, n, seed=12, box_half=BOX_HALF.get(name), aim_frac=AIM.get(name, 0.0))
    d_ref, path_ref = og.locate_many(p, v)
    ok = d_ref > 0
    p, v, d_ref, path_ref = p[ok], v[ok], d_ref[ok], path_ref[ok]
    rng = np.random.default_rng(13)
    prop = np.where(rng.uniform(size=p.shape[0]) < 0.5, np.inf, rng.exponential(60.0, size=p.shape[0]))
    s_ref, l_ref, _ = og.compute_step_many(p, v, d_ref, path_ref, prop)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    s, saf, lim = g4.g4n_compute_step(ctx, gid, to_soa(p, torch), to_soa(v, torch), T(d_ref.astype(np.int32)),
                                      T(np.ascontiguousarray(path_ref.T).astype(np.int32)), T(prop), mode=mode)
    g4.g4n_sync(ctx)
    s, saf, lim = s.cpu().numpy(), saf.cpu().numpy(), lim.cpu().numpy()
    badl = np.nonzero(lim != l_ref)[0]
    assert badl.size == 0, f"{badl.size} limiter mismatches; first {p[badl[0]]} {v[badl[0]]} gpu {lim[badl[0]]} {s[badl[0]]} ref {l_ref[badl[0]]} {s_ref[badl[0]]}"
    assert np.all(np.abs(s - s_ref) <= STEP_TOL), np.max(np.abs(s - s_ref))
    # isotropic safety: non-negative, never beyond the step, and the ball it defines stays in the volume
    assert np.all(saf >= 0.0)
    s_geo, _, s_ref_saf = og.compute_step_many(p, v, d_ref, path_ref, None)
    assert np.all(saf <= s_geo + STEP_TOL)
    if name in EXACT_SAFETY:
        # every solid here is an orb or a box aligned with its mother, whose brute-force safety the oracle
        # computes from all daughters: the device's (from the node's candidates and slab faces) is no larger
        bad = np.nonzero(saf > s_ref_saf + STEP_TOL)[0]
        assert bad.size == 0, (bad.size, p[bad[0]], saf[bad[0]], s_ref_saf[bad[0]])
    idx = np.nonzero(saf > 1e-6)[0][:300]
    dirs = rng.normal(size=(16, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    for i in idx:
        q = p[i] + 0.999 * saf[i] * dirs
        dq, pq = og.locate_many(q, np.repeat(v[i][None, :], 16, axis=0))
        assert np.all(dq == d_ref[i]) and np.all(pq == path_ref[i]), (i, p[i], saf[i])
    # geometry wins a tie with the proposed step
    s2, _, lim2 = g4.g4n_compute_step(ctx, gid, to_soa(p, torch), to_soa(v, torch), T(d_ref.astype(np.int32)),
                                      T(np.ascontiguousarray(path_ref.T).astype(np.int32)), T(s), mode=mode)
    lim2 = lim2.cpu().numpy()
    geo = lim != g4.G4N_LIM_PHYSICS
    assert np.array_equal(lim2[geo], lim[geo])


def _transport_gpu(env, gid, sc, src, seed, n, tid0=0, n_batches=100, max_steps=0, **kw):
    g4, torch, ctx = env
    stride = sc.n_volumes + 2
    items = g4.make_items([(gid, n, tid0, src, 0)])
    edep = torch.zeros((n_batches, stride), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    h = torch.zeros(n, dtype=torch.int64, device="cuda")
    ln = torch.zeros(n, dtype=torch.float64, device="cuda")
    g4.g4n_transport_batch(ctx, items, seed, edep, cnt, h, ln, n_batches=n_batches, max_steps=max_steps, **kw)
    return edep, cnt, h, ln


def _compare_transport(g4, r, edep, cnt, h, ln, nv, exact_tally_rel=1e-9):
    hashes = h.cpu().numpy().view(np.uint64)
    bad = np.nonzero(hashes != r["hashes"])[0]
    assert bad.size == 0, f"{bad.size} history mismatches (first track index {bad[:5]})"
    assert np.allclose(ln.cpu().numpy(), r["lengths"], rtol=1e-12, atol=1e-7)
    c = g4.counters_dict(cnt)
    for k, name in enumerate(oracle.COUNTER_NAMES[:10]):
        assert c[name] == int(r["counters"][k]), name
    tg = edep.cpu().numpy()
    to = r["tally"]
    nb = tg.shape[0]
    sg = tg.std(axis=0) * math.sqrt(nb)
    so = to.std(axis=0) * math.sqrt(nb)
    dg, do = tg.sum(axis=0), to.sum(axis=0)
    assert np.all(np.abs(dg - do) <= 3.0 * np.sqrt(sg ** 2 + so ** 2) + 1e-12)
    # identical histories: only the summation order differs
    assert np.all(np.abs(dg - do) <= exact_tally_rel * np.maximum(np.abs(do), 1.0))
    # energy conservation: deposits + escaped = source (a track stopped by the step cap keeps its energy)
    if c["step_limit"] == 0:
        assert abs(dg[:nv + 1].sum() - dg[nv + 1]) <= 1e-9 * dg[nv + 1]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,n", [("tiny", 10000), ("calorimeter", 20000), ("mixed_smart", 20000),
                                    ("barrel", 20000), ("nested", 20000), ("spheres", 5000), ("segments", 20000),
                                    ("nested_barrel", 20000), ("cones", 20000)])
def test_transport_parity(env, name, n, mode):
    g4, torch, ctx = env
    sc, og, gid = _build(env, name)
    src = {"tiny": synth.scenes.tiny_source(), "calorimeter": synth.scenes.calorimeter_source(),
           "barrel": synth.scenes.barrel_source(),
           "nested_barrel": synth.scenes.barrel_source()}.get(name, Source(pos=(1.0, 2.0, 3.0), isotropic=True,
                                                                   e_kind="loguniform", e0=0.05, e1=5.0))
    seed = 0x7A0C0000
    r = og.transport(src, seed, n, threads=0)
    edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, seed, n, mode=mode, diagnostics=(mode >= 1))
    g4.g4n_sync(ctx)
    _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)


@pytest.mark.parametrize("schedule", [0, 1, 2])   # 2: staged with the relocation kernel
@pytest.mark.parametrize("mode", MODES)
def test_transport_calorimeter_full_size_sampled(env, mode, schedule):
    """The benchmark workload (10^6 tracks, default launch shape): sampled histories replayed one by one
    by the oracle must match bit for bit; whole-run invariants hold at full size."""
    g4, torch, ctx = env
    sc, og, gid = _build(env, "calorimeter")
    src = synth.scenes.calorimeter_source()
    seed = synth.scenes.CONFIG_SEEDS[1][1]
    n = 1_000_000
    edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, seed, n, mode=mode, schedule=min(schedule, 1),
                                      staged_flags=1 if schedule == 2 else 0)
    g4.g4n_sync(ctx)
    hashes = h.cpu().numpy().view(np.uint64)
    lens = ln.cpu().numpy()
    rng = np.random.default_rng(3)
    ids = np.unique(np.concatenate([rng.integers(0, n, 400), [0, n - 1]]))
    for i in ids:
        r = og.transport(src, seed, 1, tid0=int(i), threads=1)
        assert hashes[i] == r["hashes"][0], i
        assert abs(lens[i] - r["lengths"][0]) <= 1e-7, i
    c = g4.counters_dict(cnt)
    assert c["tracks"] == n
    assert c["steps"] == c["geom_steps"] + c["phys_steps"]
    assert c["tracks"] == c["photo"] + c["escaped"] + c["cutoff"] + c["step_limit"]
    d = edep.cpu().numpy().sum(axis=0)
    nv = sc.n_volumes
    assert abs(d[:nv + 1].sum() - d[nv + 1]) <= 1e-9 * d[nv + 1]
    assert abs(d[nv + 1] / n - 5.05) < 0.05   # mean source energy of U(0.1, 10)


def test_transport_edge_cases(env):
    g4, torch, ctx = env
    sc, og, gid = _build(env, "tiny")
    # a track that starts outside the world escapes at once; a zero-track item is a no-op
    out = Source(pos=(900.0, 0.0, 0.0), isotropic=True, e_kind="mono", e0=1.0, e1=1.0)
    r = og.transport(out, 5, 64)
    edep, cnt, h, ln = _transport_gpu(env, gid, sc, out, 5, 64)
    g4.g4n_sync(ctx)
    _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)
    assert g4.counters_dict(cnt)["escaped"] == 64
    edep0, cnt0, _, _ = _transport_gpu(env, gid, sc, synth.scenes.tiny_source(), 5, 0)
    g4.g4n_sync(ctx)
    assert cnt0.abs().sum().item() == 0
    # a tiny step cap: the device reports it and histories still match the oracle under the same cap
    src = synth.scenes.tiny_source()
    r = og.transport(src, 6, 500, max_steps=3)
    edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, 6, 500, max_steps=3)
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_sync(ctx)
    assert e.value.code == g4.G4N_ERR_STEP_LIMIT
    _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)
    # odd launch shapes give identical histories
    r = og.transport(src, 7, 3001)
    for bs, per_sm, rm, im, mode in ((32, 1, 1, 1, 0), (96, 3, 32, 32, 1), (128, 0, 0, 0, 2), (64, 2, 5, 17, 2)):
        edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, 7, 3001, block_size=bs, blocks_per_sm=per_sm,
                                          refill_min=rm, interact_min=im, mode=mode)
        g4.g4n_sync(ctx)
        _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)


def test_query_edge_cases(env):
    g4, torch, ctx = env
    sc, og, gid = _build(env, "tiny")
    e = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    d, p = g4.g4n_locate(ctx, gid, e, e)
    g4.g4n_sync(ctx)
    assert d.numel() == 0
    # a point outside the world has depth 0
    pos = to_soa(np.array([[600.0, 0.0, 0.0], [0.0, 0.0, 0.0]]), torch)
    dirs = to_soa(np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]]), torch)
    d, p = g4.g4n_locate(ctx, gid, pos, dirs)
    g4.g4n_sync(ctx)
    assert d.cpu().tolist()[0] == 0
    # a non-unit direction is rejected by the device check
    bad = to_soa(np.array([[2.0, 0.0, 0.0]]), torch)
    g4.g4n_locate(ctx, gid, to_soa(np.zeros((1, 3)), torch), bad)
    with pytest.raises(g4.G4NError) as ex:
        g4.g4n_sync(ctx)
    assert ex.value.code == g4.G4N_ERR_ARG
    with pytest.raises(g4.G4NError):
        g4.g4n_locate(ctx, 999, pos, dirs)


def test_graph_replay_identical(env):
    """A batch recorded as a CUDA graph and replayed with new seeds gives the direct launches' histories."""
    g4, torch, ctx = env
    sc, og, gid = _build(env, "mixed_smart")
    src = Source(pos=(1.0, 2.0, 3.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
    n = 5000
    items = g4.make_items([(gid, n, 0, src, 0)])
    stride = sc.n_volumes + 2
    out = [torch.zeros((100, stride), dtype=torch.float64, device="cuda"),
           torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda"),
           torch.zeros(n, dtype=torch.int64, device="cuda")]
    graph = g4.g4n_graph_create(ctx, items, 0, out[0], out[1], out[2], mode=1)
    try:
        for seed in (17, 18, 17):
            for t in out:
                t.zero_()
            g4.g4n_graph_launch(graph, seed)
            g4.g4n_sync(ctx)
            r = og.transport(src, seed, n)
            assert np.array_equal(out[2].cpu().numpy().view(np.uint64), r["hashes"])
            assert g4.counters_dict(out[1])["steps"] == int(r["counters"][1])
    finally:
        g4.g4n_graph_destroy(graph)


def test_autotuned_shape_gives_identical_results(env):
    from paper_1209_5235_gb300.autotune import autotune
    g4, torch, ctx = env
    sc, og, gid = _build(env, "barrel")
    src = synth.scenes.barrel_source()
    n = 20000
    items = g4.make_items([(gid, n, 0, src, 0)])
    res = autotune(ctx, items, sc.n_volumes + 2, 5, modes=(0, 1), budget_s=5.0, reps=1)
    assert res["mode"] in (0, 1) and res["trials"] >= 2
    edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, 33, n, mode=res["mode"], **res["cfg"])
    g4.g4n_sync(ctx)
    r = og.transport(src, 33, n)
    _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)


@pytest.mark.parametrize("mode", [0, 1])
def test_walk_budget_gives_identical_results(env, mode):
    """A boundary search that yields after its voxel-node budget and resumes in a later round gives the
    same histories: budgets 1, 3 and 8 (yielding often) and 65536 (never) against the oracle, on a random
    world whose walks cross many voxel nodes."""
    g4, torch, ctx = env
    sc = mixed_scene(seed=11, n=400, half=500.0)
    og = oracle.Geometry(sc)
    gid = g4.build_scene(ctx, sc)
    src = Source(pos=(1.0, 2.0, 3.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
    n, seed = 6000, 0x7A0C0011
    r = og.transport(src, seed, n, threads=0)
    for budget in (1, 3, 8, 1 << 16):
        edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, seed, n, mode=mode, walk_budget=budget)
        g4.g4n_sync(ctx)
        _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)
    c = {}
    for budget in (1, 1 << 16):
        edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, seed, n, mode=mode, walk_budget=budget, diagnostics=True)
        g4.g4n_sync(ctx)
        c[budget] = g4.counters_dict(cnt)
    # budget 1 yields at every node step after the first; the continued searches visit the same nodes
    assert c[1]["walk_yields"] > 0 and c[1 << 16]["walk_yields"] == 0
    assert c[1]["vox_nodes"] == c[1 << 16]["vox_nodes"]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", ["barrel", "mixed_smart"])
def test_regroup_gives_identical_results(env, name, mode):
    """Block-wide regrouping of the tracks between rounds (periods 1 and 3, with and without yielding
    searches) moves histories between lanes and warps without changing them: compared with the oracle."""
    g4, torch, ctx = env
    sc, og, gid = _build(env, name)
    src = synth.scenes.barrel_source() if name == "barrel" else Source(pos=(1.0, 2.0, 3.0), isotropic=True,
                                                                      e_kind="loguniform", e0=0.05, e1=5.0)
    n, seed = 8000, 0x7A0C0012
    r = og.transport(src, seed, n, threads=0)
    for period, budget in ((1, 1 << 16), (3, 2), (1, 8)):
        edep, cnt, h, ln = _transport_gpu(env, gid, sc, src, seed, n, mode=mode, regroup_period=period,
                                          walk_budget=budget)
        g4.g4n_sync(ctx)
        _compare_transport(g4, r, edep, cnt, h, ln, sc.n_volumes)


@pytest.mark.parametrize("mode", [0, 1])
def test_logical_volume_scene_parity(env, mode):
    """The modular calorimeter built from reused logical volumes (expanded on the host into 1989 touchables):
    histories bit-exact against the oracle on the independently expanded scene, and the same as those of the
    scene built from explicit placements."""
    g4, torch, ctx = env
    base, lvs, pls = synth.scenes.modular_calorimeter()
    flat, _ = synth.scenes.expand_logical(base, lvs, pls)
    og = oracle.Geometry(flat)
    gid = g4.build_logical_scene(ctx, base, lvs, pls)
    gid_flat = g4.build_scene(ctx, flat)
    src = Source(pos=(3.0, -7.0, -5.0), spot_sigma=40.0, isotropic=False, direction=(0.0, 0.0, 1.0),
                 e_kind="uniform", e0=0.1, e1=5.0)
    n, seed = 20000, 0x7A0C0013
    r = og.transport(src, seed, n, threads=0)
    edep, cnt, h, ln = _transport_gpu(env, gid, flat, src, seed, n, mode=mode)
    g4.g4n_sync(ctx)
    _compare_transport(g4, r, edep, cnt, h, ln, flat.n_volumes)
    _, _, h2, _ = _transport_gpu(env, gid_flat, flat, src, seed, n, mode=mode)
    g4.g4n_sync(ctx)
    assert torch.equal(h, h2)
    assert g4.counters_dict(cnt)["geom_steps"] > 5 * n   # the tracks cross many cells


def _full_size_sampled(env, entries_fn, seed, n_sample=300, modes=(0, 1, 2), schedules=(0, 1, 2)):
    # schedules: 0 the persistent kernel, 1 staged, 2 staged with the relocation kernel
    """Every mode and schedule over a full-size launch: identical histories across them, and a random
    sample of the histories replayed one by one by the oracle."""
    g4, torch, ctx = env
    entries, stride, total, geoms = entries_fn(g4, ctx)
    items = g4.make_items(entries)
    hashes = {}
    for mode in modes:
        for sched in schedules:
            edep = torch.zeros((100, stride), dtype=torch.float64, device="cuda")
            cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
            h = torch.zeros(total, dtype=torch.int64, device="cuda")
            g4.g4n_transport_batch(ctx, items, seed, edep, cnt, h, mode=mode, schedule=min(sched, 1),
                                   staged_flags=1 if sched == 2 else 0)
            g4.g4n_sync(ctx)
            hashes[mode, sched] = h.cpu().numpy().view(np.uint64)
            c = g4.counters_dict(cnt)
            assert c["tracks"] == total and c["steps"] == c["geom_steps"] + c["phys_steps"]
    keys = list(hashes)
    for k in keys[1:]:
        bad = np.nonzero(hashes[keys[0]] != hashes[k])[0]
        assert bad.size == 0, f"{bad.size} histories differ between (mode, schedule) {keys[0]} and {k}, first {bad[:5]}"
    rng = np.random.default_rng(seed)
    starts = np.cumsum([0] + [e[1] for e in entries])
    for gidx in np.unique(rng.integers(0, total, n_sample)):
        k = int(np.searchsorted(starts, gidx, side="right") - 1)
        gid, nt, tid0, src, off = entries[k]
        r = geoms[k].transport(src, seed, 1, tid0=int(tid0 + gidx - starts[k]), threads=1)
        for key in keys:
            assert hashes[key][gidx] == r["hashes"][0], (key, gidx, k)


def test_batched_full_size_sampled(env):
    def entries_fn(g4, ctx):
        entries, geoms, off, tid = [], [], 0, 0
        for sc, nt in synth.scenes.batched_scenes():
            gid = g4.build_scene(ctx, sc)
            entries.append((gid, nt, tid, synth.scenes.batched_source(), off))
            geoms.append(oracle.Geometry(sc))
            off += sc.n_volumes + 2
            tid += nt
        return entries, off, tid, geoms
    _full_size_sampled(env, entries_fn, synth.scenes.CONFIG_SEEDS[2][1])


def test_barrel_full_size_sampled(env):
    def entries_fn(g4, ctx):
        sc = synth.scenes.barrel_scene()
        gid = g4.build_scene(ctx, sc)
        n = 10_000_000
        return [(gid, n, 0, synth.scenes.barrel_source(), 0)], sc.n_volumes + 2, n, [oracle.Geometry(sc)]
    _full_size_sampled(env, entries_fn, synth.scenes.CONFIG_SEEDS[3][1])
