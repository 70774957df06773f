"""The allocation-free transport entry point (g4n_transport_batch_noalloc).

It exists for callers that must not allocate device memory once running (a
process whose allocator reserved the GPU up front, a latency-critical loop that
forbids cudaMalloc/cudaFree): it runs the same transport kernel with its
scratch in a fixed device array of the library.  Here it is called through the
C ABI twice in a row and each result is compared with the allocating entry
point's on the same inputs, with the tolerances of the other transport tests;
the device's free memory must not move across the two calls.

This file is collected last on purpose, so a run that stops at its first
failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest

import synth

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


def _outputs(torch, g4, nb, stride, n):
    return (torch.zeros((nb, stride), dtype=torch.float64, device="cuda"),
            torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda"),
            torch.zeros(n, dtype=torch.int64, device="cuda"),
            torch.zeros(n, dtype=torch.float64, device="cuda"))


def test_noalloc_matches_allocating_entry_point_twice(env):
    g4, torch, ctx = env
    sc = synth.scenes.calorimeter_scene()
    src = synth.scenes.calorimeter_source()
    gid = g4.build_scene(ctx, sc)
    n, nb, stride, seed = 50000, 100, sc.n_volumes + 2, 4242
    items = g4.make_items([(gid, n, 0, src, 0)])
    ref = _outputs(torch, g4, nb, stride, n)
    g4.g4n_transport_batch(ctx, items, seed, *ref, n_batches=nb)
    g4.g4n_sync(ctx)
    # first call on this device: looks up the scratch array's address (set-up)
    warm = _outputs(torch, g4, nb, stride, n)
    g4.g4n_transport_batch_noalloc(ctx, items, seed, *warm, n_batches=nb)
    outs = [_outputs(torch, g4, nb, stride, n) for _ in range(2)]   # every output exists before the check
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        out = outs[call]
        g4.g4n_transport_batch_noalloc(ctx, items, seed, *out, n_batches=nb)
        torch.cuda.synchronize()
        e, c, h, ln = out
        cr = c.cpu().numpy()
        assert cr[g4.G4N_NOALLOC_STATUS_SLOT] == 0, "device-side status"
        assert np.array_equal(cr[:g4.G4N_NOALLOC_STATUS_SLOT], ref[1].cpu().numpy()[:g4.G4N_NOALLOC_STATUS_SLOT])
        assert np.array_equal(h.cpu().numpy(), ref[2].cpu().numpy()), f"call {call}: histories differ"
        assert np.allclose(ln.cpu().numpy(), ref[3].cpu().numpy(), rtol=1e-12, atol=1e-7)
        er, ee = ref[0].cpu().numpy().sum(axis=0), e.cpu().numpy().sum(axis=0)
        assert np.all(np.abs(ee - er) <= 1e-9 * np.maximum(np.abs(er), 1.0)), f"call {call}: tallies differ"
    assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated"


def test_noalloc_limits_and_status(env):
    g4, torch, ctx = env
    sc = synth.scenes.tiny_scene()
    src = synth.scenes.tiny_source()
    gid = g4.build_scene(ctx, sc)
    nb, stride = 10, sc.n_volumes + 2
    too_many = g4.make_items([(gid, 1, k, src, 0) for k in range(g4.G4N_NOALLOC_MAX_ITEMS + 1)])
    out = _outputs(torch, g4, nb, stride, g4.G4N_NOALLOC_MAX_ITEMS + 1)
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_transport_batch_noalloc(ctx, too_many, 1, *out, n_batches=nb)
    assert e.value.code == g4.G4N_ERR_ARG and "G4N_NOALLOC_MAX_ITEMS" in g4.g4n_last_error(ctx)
    # a step cap that every track reaches shows up in the status slot of the call that hit it
    items = g4.make_items([(gid, 300, 0, src, 0)])
    out = _outputs(torch, g4, nb, stride, 300)
    g4.g4n_transport_batch_noalloc(ctx, items, 1, *out, n_batches=nb, max_steps=1)
    torch.cuda.synchronize()
    assert out[1].cpu().numpy()[g4.G4N_NOALLOC_STATUS_SLOT] & 1
    out = _outputs(torch, g4, nb, stride, 300)
    g4.g4n_transport_batch_noalloc(ctx, items, 1, *out, n_batches=nb)
    torch.cuda.synchronize()
    assert out[1].cpu().numpy()[g4.G4N_NOALLOC_STATUS_SLOT] == 0
