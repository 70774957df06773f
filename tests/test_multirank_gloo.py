"""The multi-GPU path on CPU: two gloo ranks each transport their track-id shard (with the
oracle standing in for the device), reduce tallies and counters, and must reproduce the
single-process result.  Exercises the sharding and reduction logic without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1209_5235_gb300.shard import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, n, seed, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1209_5235_gb300.shard import reduce_results
    sc = synth.scenes.tiny_scene()
    g = oracle.Geometry(sc)
    tid0, count = shard_range(n, rank, world)
    r = g.transport(synth.scenes.tiny_source(), seed, count, tid0=tid0, threads=1)
    tally = torch.tensor(r["tally"])
    cnt = torch.tensor(r["counters"].astype(np.int64))
    reduce_results(tally, cnt)
    np.save(os.path.join(out_dir, f"h{rank}.npy"), r["hashes"])
    if rank == 0:
        np.save(os.path.join(out_dir, "tally.npy"), tally.numpy())
        np.save(os.path.join(out_dir, "cnt.npy"), cnt.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 1001):
        for w in (1, 2, 3, 8):
            parts = [shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and sum(c for _, c in parts) == n
            for (s0, c0), (s1, _) in zip(parts, parts[1:]):
                assert s0 + c0 == s1
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1


def test_two_gloo_ranks_match_single_process(tmp_path):
    import oracle
    import synth
    n, seed, world = 3001, 123, 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, seed, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g = oracle.Geometry(synth.scenes.tiny_scene())
    ref = g.transport(synth.scenes.tiny_source(), seed, n, threads=1)
    hashes = np.concatenate([np.load(tmp_path / f"h{r}.npy") for r in range(world)])
    assert np.array_equal(hashes, ref["hashes"])
    assert np.array_equal(np.load(tmp_path / "cnt.npy").astype(np.uint64), ref["counters"])
    assert np.allclose(np.load(tmp_path / "tally.npy"), ref["tally"], rtol=1e-12, atol=1e-12)
