"""The learned candidate proposal on the GPU: inference and gradients against the
FP64 reference network, training on samples logged by the plain navigator, identical
transport results in learned mode, and what the trained network saves."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
import synth
from synth.mlp_init import mlp_init
from gpu_common import mixed_scene

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
    yield g4, torch, ctx
    g4.g4n_destroy(ctx)


def random_data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (n, 9)).astype(np.float32)
    nc = rng.integers(2, 33, n).astype(np.int32)
    X[:, 7] = nc / 32.0
    X[:, 8] = 1.0
    y = np.array([rng.integers(0, k) for k in nc], dtype=np.int32)
    return X, y, nc


def params(seed):
    return (mlp_init(seed) + np.random.default_rng(seed).normal(0, 0.05, omlp.N_PARAMS)).astype(np.float32)


def test_predict_matches_reference(env):
    g4, torch, ctx = env
    p = params(5)
    g4.g4n_mlp_load(ctx, p)
    assert np.array_equal(g4.g4n_mlp_get(ctx), p)
    X, _, nc = random_data(1001, 6)   # ragged: not a multiple of the 32-row warp tile
    logits = g4.g4n_mlp_predict(ctx, torch.tensor(X, device="cuda")).cpu().numpy()
    ref, _ = omlp.forward(p, X, emulate_bf16=True)
    assert np.all(np.abs(logits - ref) <= 0.03 + 0.02 * np.abs(ref)), np.max(np.abs(logits - ref))
    top2 = np.sort(ref, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 0.1
    assert np.all(np.argmax(logits, axis=1)[clear] == np.argmax(ref, axis=1)[clear])


@pytest.mark.parametrize("precision,rtol", [(1, 1e-5), (0, 2e-2)])
def test_gradients_match_reference(env, precision, rtol):
    g4, torch, ctx = env
    p = params(7)
    g4.g4n_mlp_load(ctx, p)
    X, y, nc = random_data(512, 8)
    T = lambda a: torch.tensor(a, device="cuda")
    loss, g = g4.g4n_mlp_grad(ctx, T(X), T(y), T(nc), precision=precision)
    ref_loss, ref_g = omlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y, nc)
    assert abs(loss - ref_loss) <= max(rtol, 1e-6) * abs(ref_loss)
    for got, want in zip(omlp.unpack(g), omlp.unpack(ref_g)):
        assert np.linalg.norm(got - want) <= rtol * np.linalg.norm(want) + 1e-12


def _items(g4, gid, n, src, tid0=0):
    return g4.make_items([(gid, n, tid0, src, 0)])


def test_logging_and_training(env):
    g4, torch, ctx = env
    sc = mixed_scene(seed=9, n=400, half=300.0)
    gid = g4.build_scene(ctx, sc)
    src = synth.scenes.Source(pos=(0.0, 0.0, 0.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
    feat, label, ncand = g4.g4n_mlp_log(ctx, _items(g4, gid, 200000, src), 11, 400000, sc.n_volumes + 2)
    n = feat.shape[0]
    assert n > 10000
    lab, nc, F = label.cpu().numpy(), ncand.cpu().numpy(), feat.cpu().numpy()
    assert np.all((nc >= 2) & (nc <= 32) & (lab >= 0) & (lab < nc))
    assert np.all(np.abs(F[:, :3]) <= 2.0) and np.allclose(np.linalg.norm(F[:, 3:6], axis=1), 1.0, atol=1e-6)
    assert np.allclose(F[:, 7], nc / 32.0) and np.all(F[:, 8] == 1.0)
    g4.g4n_mlp_load(ctx, mlp_init(12))
    losses = g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=4, batch=1024, lr=2e-3, seed=3)
    assert losses[-1] < losses[0] < math.log(32)
    pred = g4.g4n_mlp_predict(ctx, feat).cpu().numpy()
    pred = np.where(np.arange(32)[None, :] < nc[:, None], pred, -np.inf).argmax(axis=1)
    acc = (pred == lab).mean()
    base = max(np.mean(lab == 0), np.mean(lab == np.bincount(lab).argmax()))
    # better than always proposing the most common slot: the error rate drops by a fifth at least
    assert (1.0 - acc) < 0.8 * (1.0 - base), (acc, base)


@pytest.mark.parametrize("name", ["mixed", "barrel"])
def test_learned_transport_identical(env, name):
    g4, torch, ctx = env
    sc = mixed_scene(seed=10, n=300, half=300.0) if name == "mixed" else synth.scenes.barrel_scene()
    src = (synth.scenes.Source(pos=(5.0, -3.0, 2.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
           if name == "mixed" else synth.scenes.barrel_source())
    gid = g4.build_scene(ctx, sc)
    g4.g4n_mlp_load(ctx, mlp_init(21))
    n, seed = 20000, 4321
    og = oracle.Geometry(sc)
    r = og.transport(src, seed, n)
    out = {}
    for mode in (0, 1, 2):
        edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(32, dtype=torch.int64, device="cuda")
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        g4.g4n_transport_batch(ctx, _items(g4, gid, n, src), seed, edep, cnt, h, mode=mode, diagnostics=True)
        g4.g4n_sync(ctx)
        out[mode] = (h.cpu().numpy().view(np.uint64), g4.counters_dict(cnt), edep.cpu().numpy().sum(axis=0))
        assert np.array_equal(out[mode][0], r["hashes"]), mode
        for k, nm in enumerate(oracle.COUNTER_NAMES[:10]):
            assert out[mode][1][nm] == int(r["counters"][k]), (mode, nm)
    assert out[2][1]["proposals"] > 0


def test_trained_proposal_saves_exact_evaluations(env):
    """What the trained network gains, at identical histories, on random worlds (voxel lists in id order,
    the first-hit daughter already first in most nodes): the plain navigator evaluates every listed
    candidate in FP64; the learned mode evaluates the proposal first and prunes the rest by the rigorous
    FP32 bounds, as many evaluations as the FP32 bounds alone or fewer."""
    g4, torch, ctx = env
    sc = mixed_scene(seed=13, n=1500, half=400.0)
    gid = g4.build_scene(ctx, sc)
    src = synth.scenes.Source(pos=(0.0, 0.0, 0.0), isotropic=True, e_kind="loguniform", e0=0.05, e1=5.0)
    feat, label, ncand = g4.g4n_mlp_log(ctx, _items(g4, gid, 300000, src, tid0=10_000_000), 5, 1_000_000,
                                        sc.n_volumes + 2)
    g4.g4n_mlp_load(ctx, mlp_init(14))
    g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=6, batch=2048, lr=2e-3, seed=4)
    res = _evaluations(env, gid, sc, src, 200000, 99)
    plain_evals = sum(res[0][1][k] for k in ("cand_box", "cand_tube", "cand_orb"))
    fp32_evals = res[1][1]["rechecks"]
    learned_evals = res[2][1]["rechecks"]
    print(f"FP64 candidate evaluations: plain {plain_evals}, fp32 bounds {fp32_evals}, learned {learned_evals}, "
          f"proposals {res[2][1]['proposals']}, pruned {res[2][1]['pruned']}")
    assert learned_evals <= fp32_evals
    assert learned_evals < 0.25 * plain_evals


def _evaluations(env, gid, sc, src, n, seed):
    g4, torch, ctx = env
    res = {}
    for mode in (0, 1, 2):
        edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(32, dtype=torch.int64, device="cuda")
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        g4.g4n_transport_batch(ctx, _items(g4, gid, n, src), seed, edep, cnt, h, mode=mode, diagnostics=True)
        g4.g4n_sync(ctx)
        res[mode] = (h.cpu().numpy(), g4.counters_dict(cnt))
    assert np.array_equal(res[0][0], res[2][0]) and np.array_equal(res[1][0], res[2][0])
    return res


def test_trained_proposal_gains_where_list_order_misleads(env):
    """The gain of the trained network over the method without it (the FP32-bounded navigator), at
    identical histories and against the oracle: in a stack of plates numbered from the far end, the
    candidate list puts the plates an upward ray reaches last first, so the bounds alone evaluate every
    plate ahead of the ray in FP64, farthest first; the trained proposal names the next plate, whose
    exact distance then prunes the rest."""
    g4, torch, ctx = env
    sc = synth.scenes.reversed_stack_scene()
    src = synth.scenes.reversed_stack_source()
    gid = g4.build_scene(ctx, sc)
    feat, label, ncand = g4.g4n_mlp_log(ctx, _items(g4, gid, 100000, src, tid0=20_000_000), 7, 1_000_000,
                                        sc.n_volumes + 2)
    assert feat.shape[0] > 100000
    g4.g4n_mlp_load(ctx, mlp_init(15))
    losses = g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=4, batch=2048, lr=2e-3, seed=6)
    n, seed = 50000, 77
    res = _evaluations(env, gid, sc, src, n, seed)
    r = oracle.Geometry(sc).transport(src, seed, n)
    assert np.array_equal(res[2][0].view(np.uint64), r["hashes"])
    fp32_evals = res[1][1]["rechecks"]
    learned_evals = res[2][1]["rechecks"]
    print(f"losses {losses.tolist()}; FP64 candidate evaluations: fp32 bounds {fp32_evals}, learned {learned_evals}, "
          f"proposals {res[2][1]['proposals']}, pruned {res[2][1]['pruned']}, steps {res[2][1]['steps']}")
    assert learned_evals < 0.5 * fp32_evals


def test_trained_learned_barrel_full_size_sampled(env):
    """The learned mode with a trained network on the barrel at full size (10^7 tracks): identical
    histories to the plain FP64 navigator, and 300 sampled histories replayed one by one by the oracle."""
    g4, torch, ctx = env
    sc = synth.scenes.barrel_scene()
    src = synth.scenes.barrel_source()
    gid = g4.build_scene(ctx, sc)
    feat, label, ncand = g4.g4n_mlp_log(ctx, _items(g4, gid, 500000, src, tid0=50_000_000), 3, 2_000_000,
                                        sc.n_volumes + 2)
    g4.g4n_mlp_load(ctx, mlp_init(41))
    losses = g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=2, batch=4096, lr=2e-3, seed=5)
    assert losses[-1] < losses[0]
    del feat, label, ncand
    n, seed = 10_000_000, synth.scenes.CONFIG_SEEDS[4][1]
    hashes = {}
    # the plain navigator, the learned mode with its counters (persistent kernel), the learned mode staged
    for mode, diag, sched in ((0, False, 0), (2, True, 0), (2, False, 1)):
        edep = torch.zeros((100, sc.n_volumes + 2), dtype=torch.float64, device="cuda")
        cnt = torch.zeros(32, dtype=torch.int64, device="cuda")
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        g4.g4n_transport_batch(ctx, _items(g4, gid, n, src), seed, edep, cnt, h, mode=mode, diagnostics=diag,
                               schedule=sched)
        g4.g4n_sync(ctx)
        hashes[mode, sched] = h.cpu().numpy().view(np.uint64)
        c = g4.counters_dict(cnt)
        assert c["tracks"] == n and c["steps"] == c["geom_steps"] + c["phys_steps"]
        if diag:
            assert c["proposals"] > 0
        del edep, cnt, h
    for key in ((2, 0), (2, 1)):
        bad = np.nonzero(hashes[0, 0] != hashes[key])[0]
        assert bad.size == 0, f"{bad.size} histories differ between the plain navigator and {key}"
    og = oracle.Geometry(sc)
    for i in np.unique(np.random.default_rng(8).integers(0, n, 300)):
        r = og.transport(src, seed, 1, tid0=int(i), threads=1)
        assert hashes[2, 1][i] == r["hashes"][0], i
