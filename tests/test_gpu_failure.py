"""Failure detection on the GPU without a GPU fault: every capped device loop gives up at its cap
and the context reports it (G4N_ERR_TIMEOUT / G4N_ERR_STEP_LIMIT) through g4n_sync; the context
stays usable afterwards.  Also: a CUDA graph's device errors reach g4n_sync after the context's
workspace has grown."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import to_soa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_5235_gb300 import build
    build.build()
    import paper_1209_5235_gb300 as g4
    ctx = g4.g4n_create(0)
    sc = synth.scenes.tiny_scene()
    gid = g4.build_scene(ctx, sc)
    yield g4, torch, ctx, sc, gid
    g4.g4n_destroy(ctx)


def _run(env, n=2000, seed=11, mode=0, **kw):
    g4, torch, ctx, sc, gid = env
    items = g4.make_items([(gid, n, 0, synth.scenes.tiny_source(), 0)])
    edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    h = torch.zeros(n, dtype=torch.int64, device="cuda")
    g4.g4n_transport_batch(ctx, items, seed, edep, cnt, h, mode=mode, **kw)
    return edep, cnt, h


def _expect(env, code, text):
    g4, torch, ctx, sc, gid = env
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_sync(ctx)
    assert e.value.code == code and text in str(e.value), str(e.value)


@pytest.mark.parametrize("schedule", [0, 1, 2])   # 2: staged with the relocation kernel
@pytest.mark.parametrize("mode", [0, 1])
def test_walk_cap_reports_timeout_and_context_recovers(env, mode, schedule):
    """A voxel walk capped at one node gives up on every search that crosses a node boundary; the device
    status reaches g4n_sync as G4N_ERR_TIMEOUT.  With the default cap restored the same context gives
    the oracle's histories again."""
    g4, torch, ctx, sc, gid = env
    g4.g4n_set_loop_caps(ctx, 1, 0)
    try:
        _run(env, mode=mode, schedule=min(schedule, 1), staged_flags=1 if schedule == 2 else 0)
        _expect(env, g4.G4N_ERR_TIMEOUT, "voxel walk")
    finally:
        g4.g4n_set_loop_caps(ctx, 0, 0)
    edep, cnt, h = _run(env, n=3000, seed=12, mode=mode, schedule=min(schedule, 1),
                        staged_flags=1 if schedule == 2 else 0)
    g4.g4n_sync(ctx)
    ref = oracle.Geometry(sc).transport(synth.scenes.tiny_source(), 12, 3000)
    assert np.array_equal(h.cpu().numpy().view(np.uint64), ref["hashes"])


@pytest.mark.parametrize("schedule", [0, 1])
def test_sampler_cap_reports_timeout(env, schedule):
    """Kahn's method and the disc azimuth capped at one trial reject some draws outright: reported as
    G4N_ERR_TIMEOUT (a rejection sampler reached its trial cap)."""
    g4, torch, ctx, sc, gid = env
    g4.g4n_set_loop_caps(ctx, 0, 1)
    try:
        _run(env, schedule=schedule)
        _expect(env, g4.G4N_ERR_TIMEOUT, "rejection sampler")
    finally:
        g4.g4n_set_loop_caps(ctx, 0, 0)
    _run(env, schedule=schedule)
    g4.g4n_sync(ctx)


def test_walk_cap_in_queries(env):
    """compute_step and the free path share the capped walk."""
    g4, torch, ctx, sc, gid = env
    rng = np.random.default_rng(5)
    n = 4000
    p = rng.uniform(-400.0, 400.0, size=(n, 3))
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    P, V = to_soa(p, torch), to_soa(v, torch)
    depth, path = g4.g4n_locate(ctx, gid, P, V)
    g4.g4n_sync(ctx)
    g4.g4n_set_loop_caps(ctx, 1, 0)
    try:
        g4.g4n_compute_step(ctx, gid, P, V, depth, path)
        _expect(env, g4.G4N_ERR_TIMEOUT, "voxel walk")
        Y = torch.full((n,), 50.0, dtype=torch.float64, device="cuda")
        g4.g4n_free_path(ctx, gid, P, V, Y, 1.0)
        _expect(env, g4.G4N_ERR_TIMEOUT, "voxel walk")
    finally:
        g4.g4n_set_loop_caps(ctx, 0, 0)
    g4.g4n_compute_step(ctx, gid, P, V, depth, path)
    g4.g4n_sync(ctx)


def test_loop_caps_reject_negative(env):
    g4, torch, ctx, sc, gid = env
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_set_loop_caps(ctx, -1, 0)
    assert e.value.code == g4.G4N_ERR_ARG


def test_graph_status_survives_workspace_growth(env):
    """A graph recorded before the context's item table grows (a 400-item batch) still reports its
    device errors (here the step cap) through g4n_sync."""
    g4, torch, ctx, sc, gid = env
    src = synth.scenes.tiny_source()
    stride = sc.n_volumes + 2
    edep = torch.zeros((100, stride), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    graph = g4.g4n_graph_create(ctx, g4.make_items([(gid, 500, 0, src, 0)]), 3, edep, cnt, max_steps=1)
    try:
        big = g4.make_items([(gid, 5, 5 * k, src, 0) for k in range(400)])
        e2 = torch.zeros_like(edep)
        c2 = torch.zeros_like(cnt)
        g4.g4n_transport_batch(ctx, big, 4, e2, c2)
        g4.g4n_sync(ctx)
        assert g4.counters_dict(c2)["tracks"] == 2000
        g4.g4n_graph_launch(graph, 5)
        _expect(env, g4.G4N_ERR_STEP_LIMIT, "step cap")
        assert g4.counters_dict(cnt)["step_limit"] > 0
    finally:
        g4.g4n_graph_destroy(graph)
