"""GPU parity of the staged schedule (G4N_SCHEDULE_STAGED): the track-state queues, the step and
finish kernels and the drain kernel, through the C ABI, against the FP64 oracle on the same seeded
inputs (per-track history hashes bit-exact, lengths to 1e-7 mm, tallies within 3 sigma and 1e-9
relative), for every precision mode, with pools smaller than the batch (admissions spread over
many iterations), with and without the drain, and at the edges (empty items, tracks that escape at
once, a pool of one track, the step cap, several items and geometries in one batch)."""
import numpy as np
import pytest

import oracle
import synth
from synth.scenes import Source
from gpu_common import cones_scene, mixed_scene, nested_scene, segments_scene

pytestmark = pytest.mark.gpu

STAGED = 1


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
    "tiny": (synth.scenes.tiny_scene, synth.scenes.tiny_source, 10000),
    "calorimeter": (synth.scenes.calorimeter_scene, synth.scenes.calorimeter_source, 20000),
    "mixed_smart": (mixed_scene, None, 20000),
    "barrel": (synth.scenes.barrel_scene, synth.scenes.barrel_source, 20000),
    "nested": (nested_scene, None, 20000),
    "segments": (segments_scene, None, 20000),
    "cones": (cones_scene, None, 20000),
    "nested_barrel": (synth.scenes.nested_barrel_scene, synth.scenes.barrel_source, 20000),
}
OTHER_SOURCE = Source(pos=(1.0, 2.0, 3.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
SEED = 0x57A6E000
_cache = {}


def _scene(env, name):
    g4, torch, ctx = env
    if name not in _cache:
        make, src, n = SCENES[name]
        sc = make()
        src = src() if src else OTHER_SOURCE
        og = oracle.Geometry(sc)
        _cache[name] = (sc, src, n, og, g4.build_scene(ctx, sc), og.transport(src, SEED, n, threads=0))
    return _cache[name]


def _run(env, gid, sc, src, seed, n, tid0=0, want=True, **kw):
    g4, torch, ctx = env
    items = g4.make_items([(gid, n, tid0, src, 0)])
    edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    h = torch.zeros(n, dtype=torch.int64, device="cuda") if want else None
    ln = torch.zeros(n, dtype=torch.float64, device="cuda") if want else None
    g4.g4n_transport_batch(ctx, items, seed, edep, cnt, h, ln, schedule=STAGED, **kw)
    return edep, cnt, h, ln


def _compare(g4, r, edep, cnt, h, ln, nv):
    if h is not None:
        hashes = h.cpu().numpy().view(np.uint64)
        bad = np.nonzero(hashes != r["hashes"])[0]
        assert bad.size == 0, f"{bad.size} history mismatches (first track index {bad[:5]})"
        assert np.allclose(ln.cpu().numpy(), r["lengths"], rtol=1e-12, atol=1e-7)
    c = g4.counters_dict(cnt)
    for k, name in enumerate(oracle.COUNTER_NAMES[:10]):
        assert c[name] == int(r["counters"][k]), name
    tg, to = edep.cpu().numpy(), r["tally"]
    nb = tg.shape[0]
    dg, do = tg.sum(axis=0), to.sum(axis=0)
    sg, so = tg.std(axis=0) * np.sqrt(nb), to.std(axis=0) * np.sqrt(nb)
    assert np.all(np.abs(dg - do) <= 3.0 * np.sqrt(sg ** 2 + so ** 2) + 1e-12)
    assert np.all(np.abs(dg - do) <= 1e-9 * np.maximum(np.abs(do), 1.0))
    if c["step_limit"] == 0:
        assert abs(dg[:nv + 1].sum() - dg[nv + 1]) <= 1e-9 * dg[nv + 1]


@pytest.mark.parametrize("flags", [0, 1])   # 1: G4N_STAGED_RELOCATION_KERNEL
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("name", list(SCENES))
def test_staged_parity(env, name, mode, flags):
    """Default pool (the whole batch in flight) and default drain, relocation searches in the step kernel or in
    their own kernel."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, name)
    out = _run(env, gid, sc, src, SEED, n, mode=mode, staged_flags=flags)
    g4.g4n_sync(ctx)
    _compare(g4, r, *out, sc.n_volumes)


@pytest.mark.parametrize("pool,drain", [(1024, -1), (4096, -1), (4096, 1500), (3000, 100000), (7, -1)])
@pytest.mark.parametrize("name", ["calorimeter", "barrel", "mixed_smart"])
def test_staged_pool_and_drain(env, name, pool, drain):
    """Pools smaller than the batch admit new tracks over many iterations; the drain takes over at
    various points (never, late, at once); a pool of 7 tracks keeps only a few lanes busy."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, name)
    if pool < 100:   # a tiny pool takes one iteration per step of every track: fewer tracks
        n = 500
        r = og.transport(src, SEED, n, threads=0)
    for mode, flags in ((0, 0), (1, 0), (0, 1)):
        out = _run(env, gid, sc, src, SEED, n, mode=mode, pool_tracks=pool, drain_tracks=drain, staged_flags=flags)
        g4.g4n_sync(ctx)
        _compare(g4, r, *out, sc.n_volumes)


def test_staged_without_history_outputs(env):
    """The timed launches ask for no hash or length: tallies and counters are unchanged."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, "barrel")
    out = _run(env, gid, sc, src, SEED, n, want=False, mode=0, pool_tracks=5000)
    g4.g4n_sync(ctx)
    _compare(g4, r, *out, sc.n_volumes)


def test_staged_edge_cases(env):
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, "tiny")
    # tracks that start outside the world escape at once; an empty batch is a no-op
    outside = Source(pos=(900.0, 0.0, 0.0), isotropic=True, e_kind="mono", e0=1.0, e1=1.0)
    r0 = og.transport(outside, 5, 64)
    out = _run(env, gid, sc, outside, 5, 64)
    g4.g4n_sync(ctx)
    _compare(g4, r0, *out, sc.n_volumes)
    assert g4.counters_dict(out[1])["escaped"] == 64
    _, cnt0, _, _ = _run(env, gid, sc, src, 5, 0)
    g4.g4n_sync(ctx)
    assert cnt0.abs().sum().item() == 0
    # the step cap: reported by g4n_sync, histories still those of the oracle under the same cap
    r3 = og.transport(src, 6, 500, max_steps=3)
    out = _run(env, gid, sc, src, 6, 500, max_steps=3, pool_tracks=64, drain_tracks=-1)
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_sync(ctx)
    assert e.value.code == g4.G4N_ERR_STEP_LIMIT
    _compare(g4, r3, *out, sc.n_volumes)
    # a pool of one track, a track id offset, the blocks per SM set; the step cap with the relocation kernel
    r1 = og.transport(src, 8, 40, tid0=12345)
    for flags in (0, 1):
        out = _run(env, gid, sc, src, 8, 40, tid0=12345, pool_tracks=1, drain_tracks=-1, blocks_per_sm=1,
                   staged_flags=flags)
        g4.g4n_sync(ctx)
        _compare(g4, r1, *out, sc.n_volumes)
    out = _run(env, gid, sc, src, 6, 500, max_steps=3, pool_tracks=64, drain_tracks=-1, staged_flags=1)
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_sync(ctx)
    assert e.value.code == g4.G4N_ERR_STEP_LIMIT
    _compare(g4, r3, *out, sc.n_volumes)


def test_staged_several_geometries(env):
    """One staged batch over work items in different geometries (the batched workload's form): each
    track's geometry follows it through the queues."""
    g4, torch, ctx = env
    entries, geoms, off, tid = [], [], 0, 0
    for sc, _ in list(synth.scenes.batched_scenes())[:12]:
        gid = g4.build_scene(ctx, sc)
        entries.append((gid, 700, tid, synth.scenes.batched_source(), off))
        geoms.append((sc, oracle.Geometry(sc), off, tid))
        off += sc.n_volumes + 2
        tid += 700
    items = g4.make_items(entries)
    seed = 0x5A7E
    for mode, pool, flags in ((0, 0, 0), (1, 2000, 1), (2, 777, 0), (0, 999, 1)):
        edep = torch.zeros((100, off), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
        h = torch.zeros(tid, dtype=torch.int64, device="cuda")
        g4.g4n_transport_batch(ctx, items, seed, edep, cnt, h, mode=mode, schedule=STAGED, pool_tracks=pool,
                               staged_flags=flags)
        g4.g4n_sync(ctx)
        hashes = h.cpu().numpy().view(np.uint64)
        for sc, og, o, t0 in geoms:
            r = og.transport(synth.scenes.batched_source(), seed, 700, tid0=t0, threads=0)
            assert np.array_equal(hashes[t0:t0 + 700], r["hashes"]), (mode, t0)
        assert g4.counters_dict(cnt)["tracks"] == tid


def test_staged_matches_persistent_and_reuses_queues(env):
    """The two schedules give the same outputs; a second, larger batch grows the context's queues and
    a smaller one reuses them."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, "calorimeter")
    outs = []
    for sched, pool in ((0, 0), (STAGED, 2000), (STAGED, 30000), (STAGED, 500)):
        items = g4.make_items([(gid, n, 0, src, 0)])
        edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        g4.g4n_transport_batch(ctx, items, SEED, edep, cnt, h, schedule=sched, pool_tracks=pool)
        g4.g4n_sync(ctx)
        outs.append((h.cpu().numpy(), cnt.cpu().numpy()))
    for h, c in outs[1:]:
        assert np.array_equal(h, outs[0][0])
        assert np.array_equal(c[:10], outs[0][1][:10])


def test_staged_explicit_pool_out_of_memory(env):
    """An explicit pool whose queues cannot be allocated is refused with G4N_ERR_OOM before any kernel runs (a
    batch of 10^10 tracks asks for 8.4 TB of queues); the context then runs the next batch as usual."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, "tiny")
    items = g4.make_items([(gid, 10 ** 10, 0, src, 0)])
    edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_transport_batch(ctx, items, SEED, edep, cnt, schedule=STAGED, pool_tracks=10 ** 10)
    assert e.value.code == g4.G4N_ERR_OOM and "pool_tracks" in str(e.value)
    assert cnt.abs().sum().item() == 0
    out = _run(env, gid, sc, src, SEED, n, pool_tracks=2000)
    g4.g4n_sync(ctx)
    _compare(g4, r, *out, sc.n_volumes)


def test_allocation_free_entry_point_keeps_the_persistent_kernel(env):
    """The allocation-free entry point runs the persistent kernel whatever the batch's schedule (the staged
    queues are allocated memory): the same histories as the oracle, no queue memory taken."""
    g4, torch, ctx = env
    sc, src, n, og, gid, r = _scene(env, "calorimeter")
    items = g4.make_items([(gid, n, 0, src, 0)])
    edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    h = torch.zeros(n, dtype=torch.int64, device="cuda")
    ln = torch.zeros(n, dtype=torch.float64, device="cuda")
    launches = g4.g4n_kernel_launches(ctx)
    g4.g4n_transport_batch_noalloc(ctx, items, SEED, edep, cnt, h, ln, schedule=STAGED)
    torch.cuda.synchronize()
    assert int(cnt[g4.G4N_NOALLOC_STATUS_SLOT].item()) == 0
    assert g4.g4n_kernel_launches(ctx) - launches == 1    # one persistent launch
    cnt[g4.G4N_NOALLOC_STATUS_SLOT] = 0
    _compare(g4, r, edep, cnt, h, ln, sc.n_volumes)
