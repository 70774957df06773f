"""Benchmark: gamma transport with Geant4-style navigation on one GB300.

Workload (default): the sampling calorimeter -- 5000 lead/scintillator box
cells in two-level voxels -- with 10^6 gamma tracks, energy uniform in
[0.1, 10] MeV, along +z with a 10 mm Gaussian spot; plain FP64 navigator.  One
step = one g4n_transport_batch over the whole batch (source generation,
locate, safety, boundary search, move/relocate, interactions, tallies).

Metric: navigation steps/s (every track advance, geometry- or physics-limited)
with tracks/s beside it.  Inputs (geometry tables) are resident before the
timed region; L2 is flushed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--tracks T] [--workload W]
                  [--autotune 0 --mode M --block B --blocks-per-sm S --refill-min R --interact-min I
                   --walk-budget K --regroup P]

With --impl reference the FP64 CPU oracle is timed instead, on the host cores,
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "navigation steps/sec and γ tracks/sec on 1 GB300; chosen vs plain at matched results"
WORKLOAD = ("sampling calorimeter: 50 alternating 5 mm lead-like / 10 mm scintillator-like layers x 10x10 "
            "box cells of 100x100 mm (5000 cells) in a 2 m vacuum world, smart voxels; "
            "gamma energy U(0.1, 10) MeV along +z, Gaussian spot sigma 10 mm; Compton (Kahn) + photoabsorption, "
            "10 keV cutoff; per-cell energy deposit in 100 batches")

# Algorithmic FP64 work per counted event (flops: add/sub/mul/compare/min/max = 1, fma = 2, div/sqrt = 1), from the
# formulas of each test.  An Inside test of a world-aligned box answered by exact coordinate keys (key_inside) counts
# as the FP64 box test whose answer it gives, and a relocation answered by a face record (face_reloc) as the two
# Inside tests (mother, entered volume) the method needs at least: the work the method defines, not the instructions
# the kernel executes.  DistanceToOut and Inside of tubes and cones (the *_curved counts, also included in dist_out
# and inside) add their surplus over the box's: a tube segment's exit takes ~163 (z plane ~30, the two cylinders'
# quadratics with their range tests ~69 with the shared a, b, r^2, the two phi planes ~64), its Inside ~40.
FLOPS = {"steps": 40, "dist_out": 12, "cand_box": 56, "cand_orb": 40, "cand_tube": 90, "cand_cone": 100, "inside": 24,
         "key_inside": 24, "face_reloc": 48, "vox_nodes": 14, "phys_steps": 60, "dist_out_curved": 151,
         "inside_curved": 16}
SCHEDULES = {0: "persistent", 1: "staged"}
# bytes of one track's state in the staged schedule's queues (16 doubles, hash, id, 6 ints)
STAGED_STATE_BYTES = 168
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12   # 152 SMs x 2.07 GHz x 4 FP64 flops/clk/SM (2 DFMA) = 1.2586


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one transport batch, per workload, mode and schedule,
# from single-pass ncu captures run without the L2 flush before the batch (--no-flush; the flush changes the figure by
# < 1 %): the sum over the staged schedule's kernels of a batch (launch list of nine batches, divided by nine).
# Summaries in profiles/.  Reported only while the CUDA sources, comments left out, hash to the value they had when
# the captures were taken (else the kernels may have changed since).
NCU_TRAFFIC = {"sources_sha256": "129d2cac6870f4ba898b119e5c9838caebb38c4b252f679d9108f3efd85e506a",
               # barrel: captured on the plain barrel workload (same scene and 10^7 tracks, another seed), which the
               # learned workload's line times with the same kernels; staged+reloc: the staged schedule with its
               # relocation kernel.  The calorimeter's batch was captured one commit earlier: its kernels (the
               # staged step kernel without the relocation option, finish, drain) have not changed since, only the
               # relocation kernel's launch bounds.  (The persistent kernel's figures, 1.01 GB per barrel launch and
               # 42.5 MB per calorimeter launch, were taken before its step code was shared with the staged kernels:
               # see profiles/.)
               "bytes_per_launch": {"barrel/fp32_recheck/staged+reloc": 93113306112,
                                    "barrel_learned/fp32_recheck/staged+reloc": 93113306112,
                                    "calorimeter/fp64/staged": 4296949248}}


def cuda_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1209_5235_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    for f in files + [os.path.join(ROOT, "include", "g4nav.h")]:
        with open(f, encoding="utf-8") as fh:
            h.update(os.path.basename(f).encode())
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()


def code_only(src: str) -> str:
    """C/C++/CUDA source without its comments and with runs of white space collapsed: what the compiler sees,
    so that editing a comment does not invalidate a capture of the kernels."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":                       # string or character literal, escapes kept
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def measured_traffic(workload: str, mode: str, schedule: str = "persistent"):
    """The captured DRAM bytes of one launch of (workload, mode, schedule), or None (not captured, or sources
    changed)."""
    per = NCU_TRAFFIC["bytes_per_launch"] or {}
    if NCU_TRAFFIC["sources_sha256"] != cuda_sources_sha256():
        return None
    return per.get(f"{workload}/{mode}" + ("" if schedule == "persistent" else "/" + schedule))


def algorithmic_flops(c: dict) -> float:
    return float(sum(FLOPS[k] * c[k] for k in FLOPS))


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


WORKLOADS = {
    "tiny": "tiny scene: 1 m water-like cube with 10 boxes (2-10 cm), 8x8x8 voxels; 10^4 gamma at 1 MeV isotropic",
    "batched": "256 independent water-like 1 m worlds with log-uniform 10-5000 mixed boxes/tubes/orbs rotated about z, "
               "smart voxels; 10^3-10^5 gamma each (5.65e6 total), log-uniform 0.05-5 MeV, one persistent launch",
    "barrel": "cylindrical barrel: 30 tube shells (r 50-1500 mm, 3 m) x 64 phi segments + 2000 lead-like orbs, smart "
              "voxels; 10^7 gamma log-uniform 0.02-20 MeV isotropic from points on the axis",
    "barrel_learned": "barrel scene with the learned candidate proposal (MLP trained on steps logged by the plain "
                      "navigator); 10^7 gamma",
    "stack": "24 aluminium-like plates (80 x 80 x 5 mm, pitch 40 mm) in a 200 x 200 x 1000 mm vacuum box, numbered from "
             "the far end, no voxels; 10^6 gamma 0.1-3 MeV log-uniform along +z from below, 15 mm spot; learned proposal "
             "trained on steps logged by the plain navigator",
    "barrel_nested": "barrel with deep nesting: 30 full tubes each inside the previous (the shells' annuli tiled by "
                     "64 phi segments inside each), 2000 lead-like orbs in the segments, hierarchy depth 32, smart "
                     "voxels; 10^7 gamma log-uniform 0.02-20 MeV isotropic from points on the axis",
    "spheres_regular": "Spheres (Sec. 3.4): 8000 aluminium balls r 100 mm on a 250 mm grid in a 5 m vacuum cube, smart "
                       "voxels, mu = rho x 0.06146 cm^2/g; 10^5 rays from the centre towards a 400 x 250 grid on the +z "
                       "face, Y = 1; free path T of Algorithm 1 per ray (the raytraced image)",
    "spheres_random": "Spheres (Sec. 3.4) as above; 10^5 rays from the centre, isotropic directions, Y ~ Exp(1); free "
                      "path T of Algorithm 1 per ray",
}

# The paper's Table 1 times for these inputs (GTX 470 / 2 x 6-core Opteron 2427; 10^5 particles, compute phase only).
PAPER_SPHERES_MS = {"spheres_regular": {"gpu_gtx470": 33.0, "cpu_1_thread": 442.0, "cpu_12_threads": 54.0},
                    "spheres_random": {"gpu_gtx470": 114.0, "cpu_1_thread": 458.0, "cpu_12_threads": 56.0}}
FREE_PATH_METRIC = "free paths (Algorithm 1) per second on 1 GB300, navigation steps/s beside it"


def parse_voxel(spec: str):
    """'default' | 'smart' | 'fixed:AXES:SLICES' e.g. fixed:2,0:51,11 (z then x)."""
    from synth.scenes import VoxelSpec
    if spec in ("default", ""):
        return None
    if spec == "smart":
        return VoxelSpec(mode="smart")
    _, axes, slices = spec.split(":")
    return VoxelSpec(mode="fixed", axes=tuple(int(a) for a in axes.split(",")),
                     slices=tuple(int(x) for x in slices.split(",")))


def calorimeter(voxel: str = "default"):
    import synth
    sc = synth.scenes.calorimeter_scene(voxel=parse_voxel(voxel))
    return sc, synth.scenes.calorimeter_source(), synth.scenes.CONFIG_SEEDS[1][1]


def _oracle_rate(og, src, seed, threads: int, target_s: float, tid: int, n0: int) -> dict:
    """Steps/s and tracks/s of oracle transports of growing batches of the following track ids, until
    target_s of wall time."""
    n, n_done, dt, steps = n0, 0, 0.0, 0
    used = threads
    while dt < target_s and n_done < 50_000_000:
        t0 = time.perf_counter()
        r = og.transport(src, seed, n, tid0=tid, want_hash=False, want_len=False, threads=threads)
        dt += time.perf_counter() - t0
        steps += int(r["counters"][1])
        used = int(r["threads"])
        tid += n
        n_done += n
        n *= 2
    return {"value": steps / dt, "unit": "steps/s", "cores": used, "tracks_per_s": n_done / dt, "seconds": dt,
            "histories": n_done, "next_tid": tid}


def cpu_baseline(sc, src, seed, target_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores, on bounded samples of the same workload: its uniform-grid timing
    mode (results identical to its brute-force search) on all cores and on one thread, and the brute-force
    search itself on all cores beside it."""
    import oracle
    threads = os.cpu_count() or 1
    og = oracle.Geometry(sc)
    og.use_grids(True)
    main = _oracle_rate(og, src, seed, threads, target_s, 10_000_000, 4096)
    one = _oracle_rate(og, src, seed, 1, target_s / 4, main["next_tid"], 256)
    brute = _oracle_rate(oracle.Geometry(sc), src, seed, threads, target_s / 3, one["next_tid"], 4096)
    out = {"value": main["value"], "unit": "steps/s", "cores": main["cores"], "kind": "oracle",
           "tracks_per_s": main["tracks_per_s"], "seconds": main["seconds"],
           "sample": f"{main['histories']} histories (track ids from 10^7) of the same workload, FP64 oracle in its "
                     f"uniform-grid timing mode (histories identical to its brute-force search), OpenMP over tracks"}
    out["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "tracks_per_s", "seconds")}
    out["single_thread"]["sample"] = f"{one['histories']} histories, one thread, timing mode"
    out["brute_force"] = {k: brute[k] for k in ("value", "unit", "cores", "tracks_per_s", "seconds")}
    out["brute_force"]["sample"] = f"{brute['histories']} histories, all cores, brute-force search (every daughter)"
    return out


def cpu_baseline_batched(target_s: float = 12.0) -> dict:
    """The oracle on the batched worlds: a bounded sample of each geometry's tracks, geometries in order, until
    the time target; steps/s over the whole sample."""
    import oracle
    import synth
    threads = os.cpu_count() or 1
    src, seed = synth.scenes.batched_source(), synth.scenes.CONFIG_SEEDS[2][1]
    dt, steps, n_tracks, n_geo = 0.0, 0, 0, 0
    for s2, nt in synth.scenes.batched_scenes():
        if dt >= target_s:
            break
        og = oracle.Geometry(s2)
        og.use_grids(True)
        n = min(nt, 2000)
        t0 = time.perf_counter()
        r = og.transport(src, seed, n, tid0=n_tracks, want_hash=False, want_len=False, threads=threads)
        dt += time.perf_counter() - t0
        steps += int(r["counters"][1])
        n_tracks += n
        n_geo += 1
    return {"value": steps / dt, "unit": "steps/s", "cores": threads, "kind": "oracle", "tracks_per_s": n_tracks / dt,
            "seconds": dt, "sample": f"up to 2000 tracks of each of the first {n_geo} of the 256 worlds ({n_tracks} "
                                     f"histories), FP64 oracle in its uniform-grid timing mode, OpenMP over tracks"}


def reference_workload(args):
    """(scene, source, seed, description) of the transport workload the reference arm times."""
    import synth
    w = args.workload
    if w == "calorimeter":
        sc, src, seed = calorimeter(args.voxel)
        return sc, src, seed, WORKLOAD
    if w == "tiny":
        return (synth.scenes.tiny_scene(), synth.scenes.tiny_source(), synth.scenes.CONFIG_SEEDS[0][1],
                WORKLOADS["tiny"])
    if w in ("barrel", "barrel_learned", "barrel_nested"):
        sc = synth.scenes.nested_barrel_scene() if w == "barrel_nested" else synth.scenes.barrel_scene()
        return (sc, synth.scenes.barrel_source(), synth.scenes.CONFIG_SEEDS[4 if w == "barrel_learned" else 3][1],
                WORKLOADS[w])
    return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ref = reference_workload(args)
    if ref is None:
        print(json.dumps({"impl": "reference", "unavailable": f"the reference arm times transport workloads; "
                                                              f"{args.workload} is not one"}))
        return
    sc, src, seed, workload = ref
    import oracle
    og = oracle.Geometry(sc)
    og.use_grids(True)
    threads = os.cpu_count() or 1
    n = args.ref_tracks or {"barrel": 1_000_000, "barrel_learned": 1_000_000, "barrel_nested": 500_000,
                            "calorimeter": 200_000, "tiny": 20_000}.get(args.workload, 100_000)
    n = max(64, n)
    times, steps = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = og.transport(src, seed + k, n, want_hash=False, want_len=False, threads=threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            steps.append(int(r["counters"][1]))
    tot = sum(times)
    val = sum(steps) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "tracks_per_step": n,
                       "mode": "FP64 oracle, uniform-grid timing mode (histories identical to its brute-force search)"},
            "tracks_per_s": n * args.steps / tot,
            "cpu_baseline": {"value": val, "unit": "steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{n} histories per step of the same workload"},
            "e2e": {"value": val, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def time_mode(g4, torch, ctx, items, seed, mode, args, edep, cnt, flush, stream, launch, barrier=None):
    """W warm-up launches, then K timed launches (CUDA events on the launch stream, L2 flushed between),
    bracketed by a synchronize and (several ranks) a barrier on both sides."""
    for k in range(args.warmup):
        g4.g4n_transport_batch(ctx, items, seed + 1000 + k, edep, cnt, n_batches=edep.shape[0], mode=mode,
                               stream=stream, **launch)
    g4.g4n_sync(ctx, stream)
    edep.zero_()
    cnt.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if barrier:
        barrier()
    launches0 = g4.g4n_kernel_launches(ctx)
    t_wall = time.perf_counter()
    for k in range(args.steps):
        if not getattr(args, "no_flush", False):
            flush.fill_(float(k))
        ev[k][0].record(stream)
        g4.g4n_transport_batch(ctx, items, seed + k, edep, cnt, n_batches=edep.shape[0], mode=mode, stream=stream,
                               **launch)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    t_wall = time.perf_counter() - t_wall
    launches = g4.g4n_kernel_launches(ctx) - launches0
    g4.g4n_sync(ctx, stream)
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, g4.counters_dict(cnt), t_wall, launches


def time_graph(g4, torch, ctx, items, seed, mode, args, edep, cnt, flush, stream, launch):
    """The same K timed launches replayed from a CUDA graph of the batch."""
    graph = g4.g4n_graph_create(ctx, items, seed, edep, cnt, n_batches=edep.shape[0], mode=mode, **launch)
    try:
        for k in range(args.warmup):
            g4.g4n_graph_launch(graph, seed + 1000 + k, stream)
        g4.g4n_sync(ctx, stream)
        edep.zero_()
        cnt.zero_()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            g4.g4n_graph_launch(graph, seed + k, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        g4.g4n_sync(ctx, stream)
    finally:
        g4.g4n_graph_destroy(graph)
    ms = [a.elapsed_time(b) for a, b in ev]
    c = g4.counters_dict(cnt)
    return c["steps"] / (sum(ms) / 1e3)


def setup_workload(g4, ctx, args, rank):
    """(items, stride, seed, n_tracks, description, modes) of the chosen workload on this rank."""
    import synth
    w = args.workload
    if w == "calorimeter":
        sc, src, seed = calorimeter(args.voxel)
        gid = g4.build_scene(ctx, sc)
        n = args.tracks
        return g4.make_items([(gid, n, rank * n, src, 0)]), sc.n_volumes + 2, seed, n, WORKLOAD, ["fp64", "fp32_recheck"]
    if w == "stack":
        # where list order misleads: the learned proposal against the FP32 bounds alone
        from synth.mlp_init import mlp_init
        sc, src = synth.scenes.reversed_stack_scene(), synth.scenes.reversed_stack_source()
        gid = g4.build_scene(ctx, sc)
        n = args.tracks
        log_items = g4.make_items([(gid, 100_000, 50_000_000, src, 0)])
        seed = 0x7A0C0020
        feat, label, ncand = g4.g4n_mlp_log(ctx, log_items, seed + 7, 2_000_000, sc.n_volumes + 2)
        g4.g4n_mlp_load(ctx, mlp_init(15))
        args.train_losses = g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=4, batch=2048, lr=2e-3, seed=6).tolist()
        args.train_samples = int(feat.shape[0])
        del feat, label, ncand
        return (g4.make_items([(gid, n, rank * n, src, 0)]), sc.n_volumes + 2, seed, n, WORKLOADS["stack"],
                ["fp64", "fp32_recheck", "learned"])
    if w == "tiny":
        sc = synth.scenes.tiny_scene()
        gid = g4.build_scene(ctx, sc)
        n = 10_000
        return (g4.make_items([(gid, n, rank * n, synth.scenes.tiny_source(), 0)]), sc.n_volumes + 2,
                synth.scenes.CONFIG_SEEDS[0][1], n, WORKLOADS["tiny"], ["fp64", "fp32_recheck"])
    if w == "batched":
        entries, off, tid = [], 0, 0
        for s2, nt in synth.scenes.batched_scenes():
            gid = g4.build_scene(ctx, s2)
            nt = max(1, int(round(nt * args.track_scale)))
            entries.append((gid, nt, rank * 10_000_000 + tid, synth.scenes.batched_source(), off))
            off += s2.n_volumes + 2
            tid += nt
        return g4.make_items(entries), off, synth.scenes.CONFIG_SEEDS[2][1], tid, WORKLOADS["batched"], \
            ["fp64", "fp32_recheck"]
    sc = synth.scenes.nested_barrel_scene() if w == "barrel_nested" else synth.scenes.barrel_scene()
    gid = g4.build_scene(ctx, sc)
    n = int(round(10_000_000 * args.track_scale))
    items = g4.make_items([(gid, n, rank * n, synth.scenes.barrel_source(), 0)])
    seed = synth.scenes.CONFIG_SEEDS[4 if w == "barrel_learned" else 3][1]
    modes = ["fp64", "fp32_recheck"]
    if w == "barrel_learned":
        # the proposal network: 10^7 steps logged by the plain navigator (10^7 histories give a little more; the
        # log keeps the first 10^7), trained by the library's kernels
        from synth.mlp_init import mlp_init
        log_items = g4.make_items([(gid, 10_000_000, 50_000_000, synth.scenes.barrel_source(), 0)])
        feat, label, ncand = g4.g4n_mlp_log(ctx, log_items, seed + 7, 10_000_000, sc.n_volumes + 2)
        g4.g4n_mlp_load(ctx, mlp_init(41))
        args.train_losses = g4.g4n_mlp_train(ctx, feat, label, ncand, epochs=2, batch=4096, lr=2e-3, seed=5).tolist()
        args.train_samples = int(feat.shape[0])
        del feat, label, ncand
        modes = ["fp64", "fp32_recheck", "learned"]
    return items, sc.n_volumes + 2, seed, n, WORKLOADS[w], modes


def run_gpu(args):
    import torch
    import paper_1209_5235_gb300 as g4
    from paper_1209_5235_gb300 import build as b
    from paper_1209_5235_gb300.autotune import autotune, DEFAULT
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    b.build()
    ctx = g4.g4n_create(local)
    items, stride, seed, n, workload, mode_names = setup_workload(g4, ctx, args, rank)
    nb = 100
    stream = torch.cuda.current_stream()
    edep = torch.zeros((nb, stride), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    code = {"fp64": g4.G4N_MODE_FP64, "fp32_recheck": g4.G4N_MODE_FP32_RECHECK, "learned": g4.G4N_MODE_LEARNED}
    if args.mode != "auto":
        mode_names = [args.mode]
    # launch shape per mode: autotuned on the same workload (untimed), or given
    tuned = {}
    if args.autotune:
        tune = autotune(ctx, items, stride, seed + 500, modes=[code[m] for m in mode_names], budget_s=args.tune_s,
                        stream=stream)
        for m in mode_names:
            tuned[m] = tune["per_mode"][code[m]]["cfg"]
    manual = dict(block_size=args.block, blocks_per_sm=args.blocks_per_sm, refill_min=args.refill_min,
                  interact_min=args.interact_min, walk_budget=args.walk_budget, regroup_period=args.regroup,
                  schedule=g4.G4N_SCHEDULE_STAGED if args.schedule == "staged" else g4.G4N_SCHEDULE_PERSISTENT,
                  pool_tracks=args.pool, drain_tracks=args.drain,
                  staged_flags=g4.G4N_STAGED_RELOCATION_KERNEL if args.reloc_kernel else 0)
    launch = {m: tuned.get(m, manual) for m in mode_names}
    # matched results: the same histories, bit for bit, in every mode (one launch with hashes each)
    ref_h = None
    matched = True
    for m in mode_names:
        h = torch.zeros(n, dtype=torch.int64, device="cuda")
        e2 = torch.zeros_like(edep)
        c2 = torch.zeros_like(cnt)
        g4.g4n_transport_batch(ctx, items, seed, e2, c2, h, n_batches=nb, mode=code[m], stream=stream, **launch[m])
        g4.g4n_sync(ctx, stream)
        if ref_h is None:
            ref_h = h
        else:
            matched = matched and bool(torch.equal(h, ref_h))
        del h, e2, c2
    del ref_h
    results = {}
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for m in mode_names:
            ms, c, t_wall, launches = time_mode(g4, torch, ctx, items, seed, code[m], args, edep, cnt, flush, stream,
                                                launch[m], barrier=dist.barrier if dist else None)
            t_dev = sum(ms) / 1e3
            steps_total, tracks_total = c["steps"], c["tracks"]
            if dist:
                tt = torch.tensor([t_dev], device="cuda")
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                t_dev = float(tt.item())
                st = torch.tensor([steps_total, tracks_total], dtype=torch.int64, device="cuda")
                dist.all_reduce(st)
                steps_total, tracks_total = int(st[0].item()), int(st[1].item())
            results[m] = {"steps_per_s": steps_total / t_dev, "tracks_per_s": tracks_total / t_dev,
                          "ms_per_step": 1e3 * t_dev / args.steps, "ms_launch_mean": float(np.mean(ms)),
                          "steps_per_track": steps_total / max(tracks_total, 1), "launch": launch[m],
                          "schedule": SCHEDULES[launch[m].get("schedule", 0)], "gpu_launches": launches,
                          "interactions": c["photo"] + c["compton"]}
    chosen = max(results, key=lambda k: results[k]["steps_per_s"]) if matched else "fp64"
    mode = code[chosen]
    graph_value = time_graph(g4, torch, ctx, items, seed, mode, args, edep, cnt, flush, stream, launch[chosen])
    # algorithmic work of one launch: a counting launch with the timed seed (outside the timed region)
    cnt.zero_()
    edep.zero_()
    g4.g4n_transport_batch(ctx, items, seed, edep, cnt, n_batches=nb, mode=mode, stream=stream, diagnostics=True,
                           **launch[chosen])
    g4.g4n_sync(ctx, stream)
    cdiag = g4.counters_dict(cnt)
    # end to end through the host-buffer entry point: H2D of the batch description, D2H of the tallies
    # the host result buffers are pinned (page-locked) memory, as a caller streaming results would use
    out = {"edep": torch.zeros((nb, stride), dtype=torch.float64).pin_memory().numpy(),
           "counters": torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64).pin_memory().numpy().view(np.uint64),
           "hashes": None, "lengths": None}
    e2e_steps, e2e_t = 0, 0.0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        out = g4.g4n_transport_batch_host(ctx, items, seed + k, stride, n_batches=nb, mode=mode, stream=stream,
                                          out=out, **launch[chosen])
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            e2e_t += dt
            e2e_steps += int(out["counters"][1])
    if dist:
        tt = torch.tensor([e2e_t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    e2e = {"value": e2e_steps * world / e2e_t, "unit": "steps/s",
           "h2d_bytes_per_step": int(len(items) * ctypes.sizeof(g4.g4n_work_item) + ctypes.sizeof(g4.g4n_batch_desc)),
           "d2h_bytes_per_step": int(nb * stride * 8 + g4.G4N_N_COUNTERS * 8)}
    g4.g4n_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    R = results[chosen]
    flops = algorithmic_flops(cdiag)               # per launch (this rank)
    t_launch = R["ms_launch_mean"] / 1e3
    achieved = flops / t_launch / 1e12
    hbm_bytes = (nb * stride * 8) * 2              # tallies read + written once per launch; tables stay in L2
    staged = R["schedule"] == "staged"
    reloc_kernel = staged and bool(R["launch"].get("staged_flags", 0) & g4.G4N_STAGED_RELOCATION_KERNEL)
    if staged:
        # the queues: every step and every interaction reads a state and writes one back, every start writes one;
        # with the relocation kernel every relocation search (a crossing no face record answers) one more of each
        hbm_bytes += STAGED_STATE_BYTES * (2 * cdiag["steps"] + 2 * (cdiag["photo"] + cdiag["compton"])
                                           + cdiag["tracks"])
        if reloc_kernel:
            hbm_bytes += (STAGED_STATE_BYTES + 4) * 2 * (cdiag["geom_steps"] - cdiag["face_reloc"])
    line = {
        "metric": METRIC, "value": R["steps_per_s"], "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "tracks_per_gpu": n, "mode": chosen,
                   "schedule": R["schedule"] + (" + relocation kernel" if reloc_kernel else ""),
                   "l2": ("not flushed (DRAM-traffic capture run)" if args.no_flush
                          else "flushed between timed steps (256 MB write)"), "launch": launch[chosen],
                   "autotuned": bool(args.autotune), "voxel": args.voxel if args.workload == "calorimeter" else "smart"},
        "tracks_per_s": R["tracks_per_s"],
        "steps_per_track": R["steps_per_track"],
        "modes": results,
        "matched_results": matched,
        "plain_fp64_steps_per_s": results.get("fp64", {}).get("steps_per_s"),
        "graph_replay_steps_per_s": graph_value,
        "gpu_launches": R["gpu_launches"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": measured_traffic(args.workload, chosen,
                                                 R["schedule"] + ("+reloc" if reloc_kernel else "")),
                     "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flops/clk/SM (recipe nominal 1.25 TFLOP/s)",
                     "kernel": (("k_staged_step + k_staged_reloc + k_staged_finish + k_staged_drain" if reloc_kernel
                                 else "k_staged_step + k_staged_finish + k_staged_drain") + " (one transport batch)"
                                if staged else "k_transport"), "flops_per_launch": flops},
        "hbm": {"algorithmic_bytes_per_launch": hbm_bytes, "achieved_gbs": hbm_bytes / t_launch / 1e9,
                "peak_gbs": peaks.get("hbm_gbs"),
                "frac": (hbm_bytes / t_launch / 1e9) / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None},
        "clocks": clk.summary(),
        "e2e": e2e,
        "counters": {k: cdiag[k] for k in ("steps", "geom_steps", "phys_steps", "safety_skips", "cand_box",
                                           "cand_tube", "cand_orb", "inside", "inside_curved", "key_inside",
                                           "face_reloc", "vox_nodes", "dist_out", "dist_out_curved", "rechecks",
                                           "proposals", "pruned")},
    }
    if getattr(args, "train_losses", None):
        line["learned"] = {"train_samples": args.train_samples, "epoch_losses": args.train_losses}
    if not args.no_cpu_baseline and world == 1:
        import synth
        if args.workload == "calorimeter":
            line["cpu_baseline"] = cpu_baseline(*calorimeter(args.voxel))
        elif args.workload == "batched":
            line["cpu_baseline"] = cpu_baseline_batched()
        elif args.workload.startswith("barrel"):
            sc = synth.scenes.nested_barrel_scene() if args.workload == "barrel_nested" else synth.scenes.barrel_scene()
            line["cpu_baseline"] = cpu_baseline(sc, synth.scenes.barrel_source(), seed)
        elif args.workload == "stack":
            line["cpu_baseline"] = cpu_baseline(synth.scenes.reversed_stack_scene(),
                                                synth.scenes.reversed_stack_source(), seed)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_free_path(args):
    """The Spheres benchmark: Algorithm 1 free paths of 10^5 rays (g4n_free_path), compute phase timed."""
    import torch
    import paper_1209_5235_gb300 as g4
    from paper_1209_5235_gb300 import build as b
    import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    b.build()
    ctx = g4.g4n_create(local)
    sc = synth.scenes.spheres_scene()
    gid = g4.build_scene(ctx, sc)
    kind = args.workload.split("_")[1]
    p, v, Y = synth.scenes.spheres_rays(kind, seed=0x7A0C0005 + rank)
    n, E = len(Y), synth.scenes.SPHERES_ENERGY
    pos = torch.tensor(np.ascontiguousarray(p.T), dtype=torch.float64, device="cuda")
    dirs = torch.tensor(np.ascontiguousarray(v.T), dtype=torch.float64, device="cuda")
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    T = torch.empty(n, dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    code = {"fp64": g4.G4N_MODE_FP64, "fp32_recheck": g4.G4N_MODE_FP32_RECHECK}
    modes = ["fp64", "fp32_recheck"] if args.mode == "auto" else [args.mode]
    ref = None
    matched = True
    for m in modes:
        g4.g4n_free_path(ctx, gid, pos, dirs, Yd, E, mode=code[m], out_T=T, out_steps=st, stream=stream)
        g4.g4n_sync(ctx, stream)
        if ref is None:
            ref = T.clone()
        else:
            matched = matched and bool(torch.equal(torch.nan_to_num(T, posinf=-1.0), torch.nan_to_num(ref, posinf=-1.0)))
    results = {}
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for m in modes:
            for k in range(args.warmup):
                g4.g4n_free_path(ctx, gid, pos, dirs, Yd, E, mode=code[m], out_T=T, out_steps=st, stream=stream)
            g4.g4n_sync(ctx, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                g4.g4n_free_path(ctx, gid, pos, dirs, Yd, E, mode=code[m], out_T=T, out_steps=st, stream=stream)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            g4.g4n_sync(ctx, stream)
            ms = [a.elapsed_time(c) for a, c in ev]
            t_dev = sum(ms) / 1e3
            if dist:
                tt = torch.tensor([t_dev], device="cuda")
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                t_dev = float(tt.item())
            segs = int(st.to(torch.int64).sum().item())
            results[m] = {"rays_per_s": world * n * args.steps / t_dev, "nav_steps_per_s": world * segs * args.steps / t_dev,
                          "ms_per_step": 1e3 * t_dev / args.steps, "ms_launch_mean": float(np.mean(ms)),
                          "steps_per_ray": segs / n}
    chosen = max(results, key=lambda k: results[k]["rays_per_s"]) if matched else "fp64"
    R = results[chosen]
    cnt = torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    g4.g4n_free_path(ctx, gid, pos, dirs, Yd, E, mode=code[chosen], counters=cnt, diagnostics=True, out_T=T,
                     out_steps=st, stream=stream)
    g4.g4n_sync(ctx, stream)
    cdiag = g4.counters_dict(cnt)
    escaped = int(torch.isinf(T).sum().item())
    # end to end through the public API: pinned host inputs copied in, T copied out, every step
    hp = torch.from_numpy(np.ascontiguousarray(p.T)).pin_memory()
    hv = torch.from_numpy(np.ascontiguousarray(v.T)).pin_memory()
    hY = torch.from_numpy(Y.copy()).pin_memory()
    hT = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_t = 0.0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pos.copy_(hp, non_blocking=True)
        dirs.copy_(hv, non_blocking=True)
        Yd.copy_(hY, non_blocking=True)
        g4.g4n_free_path(ctx, gid, pos, dirs, Yd, E, mode=code[chosen], out_T=T, out_steps=st, stream=stream)
        hT.copy_(T, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_t += time.perf_counter() - t0
    g4.g4n_sync(ctx, stream)
    g4.g4n_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    flops = (FLOPS["steps"] * cdiag["steps"] + FLOPS["dist_out"] * cdiag["dist_out"] + FLOPS["cand_orb"] *
             cdiag["cand_orb"] + FLOPS["cand_box"] * cdiag["cand_box"] + FLOPS["inside"] * (cdiag["inside"] + cdiag["key_inside"])
             + FLOPS["face_reloc"] * cdiag["face_reloc"] + FLOPS["vox_nodes"] * cdiag["vox_nodes"])
    t_launch = R["ms_launch_mean"] / 1e3
    paper = PAPER_SPHERES_MS[args.workload]
    line = {
        "metric": FREE_PATH_METRIC, "value": R["rays_per_s"], "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": R["rays_per_s"] / world / (1e5 / (paper["gpu_gtx470"] / 1e3)), "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "rays_per_gpu": n, "mode": chosen,
                   "l2": "flushed between timed steps (256 MB write)", "energy_mev": E},
        "nav_steps_per_s": R["nav_steps_per_s"], "steps_per_ray": R["steps_per_ray"], "escaped": escaped,
        "modes": results, "matched_results": matched, "gpu_launches": args.steps,
        "paper_table1_ms": paper,
        "vs_baseline_note": "rays/s per GPU over the paper's GTX 470 rays/s (10^5 rays / its time): another machine, context",
        "roofline": {"bound": "alu", "achieved": flops / t_launch / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": flops / t_launch / 1e12 / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_free_path",
                     "flops_per_launch": flops},
        "clocks": clk.summary(),
        "e2e": {"value": world * n * args.steps / e2e_t, "unit": "rays/s", "h2d_bytes_per_step": int(7 * 8 * n),
                "d2h_bytes_per_step": int(8 * n)},
        "counters": {k: cdiag[k] for k in ("tracks", "steps", "geom_steps", "phys_steps", "escaped", "dist_out",
                                           "cand_orb", "key_inside", "inside", "vox_nodes")},
    }
    if not args.no_cpu_baseline and world == 1:
        import oracle
        og = oracle.Geometry(sc)
        og.use_grids(True)          # the oracle's timing mode: free paths identical to its brute-force search
        t0 = time.perf_counter()
        _, _, used = og.free_path_many(p, v, E, Y)
        dt_all = time.perf_counter() - t0
        t0 = time.perf_counter()
        og.free_path_many(p, v, E, Y, threads=1)
        dt_1 = time.perf_counter() - t0
        ob = oracle.Geometry(sc)    # brute force: every step tests all 8000 balls
        m1 = 20000
        t0 = time.perf_counter()
        ob.free_path_many(p[:m1], v[:m1], E, Y[:m1])
        dt_b = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / dt_all, "unit": "rays/s", "cores": int(used), "kind": "oracle",
                                "single_thread_rays_per_s": n / dt_1, "brute_force_rays_per_s": m1 / dt_b,
                                "sample": f"all {n} rays on {used} threads and on 1 thread, FP64 oracle in its "
                                          f"uniform-grid timing mode; the first {m1} rays by its brute-force search "
                                          f"on {used} threads"}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


QUERY_METRIC = "navigation queries/sec on 1 GB300 (the two navigation problems of Sec. 3.2: locate, compute_step)"


def run_queries(args):
    """Throughput of the query entry points g4n_locate / g4n_compute_step on resident SoA inputs: 10^7
    points uniform in a box around the detector with isotropic directions (compute_step: from their
    located paths, with a physics proposal per query), L2 flushed between timed launches."""
    import torch
    import paper_1209_5235_gb300 as g4
    from paper_1209_5235_gb300 import build as b
    import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    b.build()
    ctx = g4.g4n_create(local)
    scene = args.scene
    sc = calorimeter(args.voxel)[0] if scene == "calorimeter" else synth.scenes.barrel_scene()   # smart voxels
    gid = g4.build_scene(ctx, sc)
    n = args.queries
    p, v = synth.scenes.query_points(scene, n, seed=0x7A0C0010 + rank)
    pos = torch.from_numpy(p).cuda()
    dirs = torch.from_numpy(v).cuda()
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    path = torch.empty((g4.G4N_DMAX, n), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    g4.g4n_locate(ctx, gid, pos, dirs, depth, path, stream=stream)
    g4.g4n_sync(ctx, stream)
    prop = torch.from_numpy(np.random.default_rng(0x7A0C0011 + rank).exponential(100.0, n)).cuda()
    kind = args.workload
    modes = {"fp64": g4.G4N_MODE_FP64, "fp32_recheck": g4.G4N_MODE_FP32_RECHECK}
    if kind == "locate":
        modes = {"fp64": g4.G4N_MODE_FP64}       # the descent is the same code in every mode
        in_b, out_b = 48, 4 + 4 * g4.G4N_DMAX     # pos, dir | depth, path (all G4N_DMAX levels written)

        def launch(mode):
            g4.g4n_locate(ctx, gid, pos, dirs, depth, path, stream=stream)
    else:
        in_b, out_b = 48 + 4 + 4 + 8, 8 + 8 + 4   # pos, dir, depth, the leaf's path entry, proposal | step, safety, limiter
        outs = {m: (torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda"),
                    torch.empty(n, dtype=torch.int32, device="cuda")) for m in modes.values()}

        def launch(mode):
            g4.g4n_compute_step(ctx, gid, pos, dirs, depth, path, prop, mode=mode, stream=stream, out=outs[mode])
    results = {}
    ref = None
    matched = True
    with ClockSampler(local) as clk:
        for name, mode in modes.items():
            launch(mode)
            g4.g4n_sync(ctx, stream)
            if kind == "compute_step":
                got = tuple(x.clone() for x in outs[mode][::2])   # step, limiter
                if ref is None:
                    ref = got
                else:
                    matched = matched and all(bool(torch.equal(a, c)) for a, c in zip(got, ref))
            for k in range(args.warmup):
                launch(mode)
            g4.g4n_sync(ctx, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                launch(mode)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            g4.g4n_sync(ctx, stream)
            ms = [a.elapsed_time(c) for a, c in ev]
            t_dev = sum(ms) / 1e3
            if dist:
                tt = torch.tensor([t_dev], device="cuda")
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                t_dev = float(tt.item())
            results[name] = {"queries_per_s": world * n * args.steps / t_dev, "ms_per_step": 1e3 * t_dev / args.steps,
                             "ms_launch_mean": float(np.mean(ms))}
    chosen = max(results, key=lambda k: results[k]["queries_per_s"]) if matched else "fp64"
    R = results[chosen]
    # end to end: pinned host inputs in, outputs back, every step
    hp = torch.from_numpy(p).pin_memory()
    hv = torch.from_numpy(v).pin_memory()
    if kind == "locate":
        hout = [torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty((g4.G4N_DMAX, n), dtype=torch.int32).pin_memory()]
    else:
        hd = depth.cpu().pin_memory()
        hpath = path.cpu().pin_memory()
        hprop = prop.cpu().pin_memory()
        hout = [torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory(),
                torch.empty(n, dtype=torch.int32).pin_memory()]
    e2e_t = 0.0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pos.copy_(hp, non_blocking=True)
        dirs.copy_(hv, non_blocking=True)
        if kind == "locate":
            g4.g4n_locate(ctx, gid, pos, dirs, depth, path, stream=stream)
            devs = [depth, path]
        else:
            depth.copy_(hd, non_blocking=True)
            path.copy_(hpath, non_blocking=True)
            prop.copy_(hprop, non_blocking=True)
            devs = list(g4.g4n_compute_step(ctx, gid, pos, dirs, depth, path, prop, mode=modes[chosen], stream=stream,
                                            out=outs[modes[chosen]]))
        for h, d in zip(hout, devs):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_t += time.perf_counter() - t0
    g4.g4n_sync(ctx, stream)
    h2d = n * (48 if kind == "locate" else 48 + 4 + 4 * g4.G4N_DMAX + 8)
    d2h = n * (4 + 4 * g4.G4N_DMAX if kind == "locate" else 20)
    g4.g4n_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks = load_peaks()
    t_launch = R["ms_launch_mean"] / 1e3
    algo = n * (in_b + out_b)
    achieved = algo / t_launch / 1e9
    peak = peaks.get("hbm_gbs")
    line = {
        "metric": QUERY_METRIC, "value": R["queries_per_s"], "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{kind}: {n} queries on the {scene} scene, points uniform in the box "
                               f"{synth.scenes.QUERY_BOXES[scene]} mm, isotropic directions"
                               + ("" if kind == "locate" else ", from their located paths, physics proposal "
                                                               "~ Exp(mean 100 mm)"),
                   "queries_per_gpu": n, "mode": chosen, "l2": "flushed between timed steps (256 MB write)"},
        "modes": results, "matched_results": matched, "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": None,
                     "kernel": "k_locate" if kind == "locate" else "k_compute_step",
                     "algorithmic_bytes_per_query": in_b + out_b, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "clocks": clk.summary(),
        "e2e": {"value": world * n * args.steps / e2e_t, "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed launches per mode (default 10 for the 10^7-track barrel workloads, else 20)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tracks", type=int, default=1_000_000)
    ap.add_argument("--track-scale", type=float, default=1.0,
                    help="batched / barrel workloads: fraction of their track counts (profiling a smaller case)")
    ap.add_argument("--ref-tracks", type=int, default=0,
                    help="reference arm: histories per step (default: about a second of the oracle on 16 cores)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--refill-min", type=int, default=0)
    ap.add_argument("--interact-min", type=int, default=0)
    ap.add_argument("--walk-budget", type=int, default=0)
    ap.add_argument("--regroup", type=int, default=0)
    ap.add_argument("--mode", default="auto", choices=["auto", "fp64", "fp32_recheck"])
    ap.add_argument("--voxel", default="smart")
    ap.add_argument("--workload", default="barrel_learned",
                    choices=["calorimeter", "tiny", "batched", "barrel", "barrel_learned", "barrel_nested", "stack",
                             "spheres_regular", "spheres_random", "locate", "compute_step"])
    ap.add_argument("--scene", default="calorimeter", choices=["calorimeter", "barrel"],
                    help="locate / compute_step workloads: the scene queried")
    ap.add_argument("--queries", type=int, default=10_000_000)
    ap.add_argument("--schedule", default="staged", choices=["staged", "persistent"],
                    help="schedule of the transport when --autotune 0 (the tuner chooses it otherwise)")
    ap.add_argument("--pool", type=int, default=0, help="staged schedule: tracks in flight (0 = default)")
    ap.add_argument("--drain", type=int, default=0, help="staged schedule: drain point (0 = default, -1 = never)")
    ap.add_argument("--reloc-kernel", type=int, default=0,
                    help="staged schedule: relocation searches in a kernel of their own (1) or in the step kernel (0)")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--tune-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-flush", action="store_true",
                    help="no L2 flush between timed launches: only for the DRAM-traffic capture of a launch in the "
                         "steady state (the flush's dirty lines would otherwise be written back during the launch)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.workload.startswith("barrel") else 20
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("spheres_"):
        run_free_path(args)
    elif args.workload in ("locate", "compute_step"):
        run_queries(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
