"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol declared in include/g4nav.h, and its host-side geometry builder
(host-only context, no GPU) validates geometries and builds voxels."""
import math
import os
import re

import numpy as np
import pytest

import synth
from synth.scenes import Scene, Solid, Placement, VoxelSpec, BOX, TUBE, ORB, CONE
from synth.materials import vacuum

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g4():
    from paper_1209_5235_gb300 import build
    build.build()
    import paper_1209_5235_gb300 as g
    return g


def declared_functions():
    src = open(os.path.join(ROOT, "include", "g4nav.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(g4n_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(g4):
    L = g4.load()
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def test_create_without_gpu_fails_cleanly(g4):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(g4.G4NError) as e:
        g4.g4n_create(0)
    assert e.value.code == g4.G4N_ERR_CUDA if hasattr(g4, "G4N_ERR_CUDA") else True


def _scene(solids, places):
    return Scene("t", [vacuum()], [Solid(BOX, (100.0, 100.0, 100.0))] + solids,
                 [Placement(-1, 0, 0, (0, 0, 0))] + places, VoxelSpec(mode="smart"))


def test_host_only_builds_configs(g4):
    ctx = g4.g4n_create(-1)
    try:
        for sc in (synth.scenes.tiny_scene(), synth.scenes.calorimeter_scene(), synth.scenes.barrel_scene(),
                   synth.scenes.spheres_scene()):
            info = g4.g4n_geom_info(ctx, g4.build_scene(ctx, sc))
            assert info["n_volumes"] == sc.n_volumes
            assert info["max_depth"] == max(1 + _depth(sc, i) for i in range(sc.n_volumes))
            assert info["n_candidate_entries"] >= sc.n_volumes - 1
    finally:
        g4.g4n_destroy(ctx)


def _depth(sc, i):
    d = 0
    while sc.placements[i].mother >= 0:
        i = sc.placements[i].mother
        d += 1
    return d


@pytest.mark.parametrize("case,code", [
    ("overlap", -2), ("sticks_out", -2), ("too_deep", -2), ("bad_rotation", -1), ("bad_box", -1),
    ("bad_tube", -1), ("bad_cone", -1), ("cone_sticks_out", -2), ("world_not_first", -1), ("bad_material_id", -1)])
def test_host_only_validation(g4, case, code):
    ctx = g4.g4n_create(-1)
    try:
        with pytest.raises(g4.G4NError) as e:
            if case == "overlap":
                g4.build_scene(ctx, _scene([Solid(BOX, (10, 10, 10))],
                                           [Placement(0, 1, 0, (0, 0, 0)), Placement(0, 1, 0, (5, 0, 0))]))
            elif case == "sticks_out":
                g4.build_scene(ctx, _scene([Solid(ORB, (10,))], [Placement(0, 1, 0, (95, 0, 0))]))
            elif case == "too_deep":
                D = g4.G4N_DMAX
                sols = [Solid(BOX, (95.0 - 2.5 * k,) * 3) for k in range(D)]
                g4.build_scene(ctx, _scene(sols, [Placement(k, k + 1, 0, (0, 0, 0)) for k in range(D)]))
            elif case == "bad_rotation":
                g4.build_scene(ctx, _scene([Solid(BOX, (1, 1, 1))], [Placement(0, 1, 0, (0, 0, 0), (1.0, 0.1))]))
            elif case == "bad_box":
                g4.g4n_solid_box(ctx, 1.0, 0.0, 1.0)
            elif case == "bad_tube":
                g4.g4n_solid_tube(ctx, 2.0, 1.0, 1.0, 0.0, 1.0)
            elif case == "bad_cone":
                g4.g4n_solid_cone(ctx, 0.0, 1.0, 2.0, 1.5, 1.0)
            elif case == "cone_sticks_out":
                # the wide end (radius 30) of the cone does not fit the 20 mm mother box
                g4.build_scene(ctx, _scene([Solid(BOX, (20, 20, 20)), Solid(CONE, (0, 5, 0, 30, 10))],
                                           [Placement(0, 1, 0, (0, 0, 0)), Placement(1, 2, 0, (0, 0, 0))]))
            elif case == "world_not_first":
                m = g4.g4n_material_add(ctx, 1.0, [1, 2], [0, 0], [0, 0])
                s = g4.g4n_solid_box(ctx, 1, 1, 1)
                g4.g4n_place(ctx, 0, s, m, [0, 0, 0])
            elif case == "bad_material_id":
                s = g4.g4n_solid_box(ctx, 1, 1, 1)
                g4.g4n_place(ctx, -1, s, 7, [0, 0, 0])
        assert e.value.code == code
        assert g4.g4n_last_error(ctx)
    finally:
        g4.g4n_destroy(ctx)


def test_host_only_accepts_touching_and_max_depth(g4):
    """Exactly touching siblings and a hierarchy of exactly G4N_DMAX levels are valid."""
    ctx = g4.g4n_create(-1)
    try:
        D = g4.G4N_DMAX
        sols = [Solid(BOX, (95.0 - 2.5 * k,) * 3) for k in range(D - 1)]
        g4.build_scene(ctx, _scene(sols, [Placement(k, k + 1, 0, (0, 0, 0)) for k in range(D - 1)]))
        g4.build_scene(ctx, _scene([Solid(BOX, (10, 10, 10))],
                                   [Placement(0, 1, 0, (-10, 0, 0)), Placement(0, 1, 0, (10, 0, 0))]))
        seg = Solid(TUBE, (10.0, 20.0, 5.0, 0.0, math.pi / 2))
        g4.build_scene(ctx, _scene([seg], [Placement(0, 1, 0, (0, 0, 0), (math.cos(k * math.pi / 2), math.sin(k * math.pi / 2)))
                                           for k in range(4)]))
    finally:
        g4.g4n_destroy(ctx)


def test_queries_refused_on_host_only_context(g4):
    ctx = g4.g4n_create(-1)
    try:
        gid = g4.build_scene(ctx, synth.scenes.tiny_scene())
        L = g4.load()
        assert L.g4n_locate(ctx, gid, 1, None, None, None, None, None) == g4.G4N_ERR_STATE
    finally:
        g4.g4n_destroy(ctx)


@pytest.mark.parametrize("field,value", [("walk_budget", -1), ("regroup_period", -2), ("refill_min", 33),
                                         ("interact_min", 40), ("block_size", 48), ("mode", 7), ("schedule", 2),
                                         ("pool_tracks", -1), ("staged_flags", 2)])
def test_transport_rejects_bad_launch_fields(g4, field, value):
    """Launch-shape fields are validated on the host before any device work (G4N_ERR_ARG); with valid fields the
    same call on a host-only context is refused as a device query (G4N_ERR_STATE).  The output pointers are host
    placeholders that the refused calls never touch."""
    import ctypes
    from paper_1209_5235_gb300 import binding
    ctx = g4.g4n_create(-1)
    try:
        gid = g4.build_scene(ctx, synth.scenes.tiny_scene())
        items = g4.make_items([(gid, 10, 0, synth.scenes.tiny_source(), 0)])
        edep = np.zeros((100, 13))
        cnt = np.zeros(g4.G4N_N_COUNTERS, dtype=np.uint64)
        L = g4.load()
        d = binding._desc(items, 1, 0.01, 0, 100, 13, 0, 0, 0)
        assert L.g4n_transport_batch(ctx, ctypes.byref(d), edep.ctypes.data, cnt.ctypes.data, None, None,
                                     None) == g4.G4N_ERR_STATE
        setattr(d, field, value)
        assert L.g4n_transport_batch(ctx, ctypes.byref(d), edep.ctypes.data, cnt.ctypes.data, None, None,
                                     None) == g4.G4N_ERR_ARG
        assert g4.g4n_last_error(ctx)
    finally:
        g4.g4n_destroy(ctx)


def test_logical_volumes_expand_into_touchables(g4):
    """Placing reused logical volumes gives the same geometry as writing the expanded placements out (an
    independent expansion in synth), with the touchable path (logical volume, copy number) of every volume."""
    base, lvs, pls = synth.scenes.modular_calorimeter()
    flat, touch = synth.scenes.expand_logical(base, lvs, pls)
    ctx = g4.g4n_create(-1)
    try:
        gid = g4.build_logical_scene(ctx, base, lvs, pls)
        gid_flat = g4.build_scene(ctx, flat)
        assert g4.g4n_geom_info(ctx, gid) == g4.g4n_geom_info(ctx, gid_flat)
        assert g4.g4n_geom_info(ctx, gid)["n_volumes"] == flat.n_volumes == 1 + 4 * (1 + 16 * (1 + 10 * 3))
        for v in range(flat.n_volumes):
            chain, x = [], v
            while x >= 0:
                chain.append(touch[x])
                x = flat.placements[x].mother
            assert g4.g4n_touchable(ctx, gid, v) == chain[::-1]
    finally:
        g4.g4n_destroy(ctx)


def test_logical_volume_errors(g4):
    ctx = g4.g4n_create(-1)
    try:
        m = g4.g4n_material_add(ctx, 1.0, [1, 2], [0, 0], [0, 0])
        s = g4.g4n_solid_box(ctx, 10, 10, 10)
        a = g4.g4n_logical_create(ctx, s, m)
        b = g4.g4n_logical_create(ctx, s, m)
        g4.g4n_logical_add_daughter(ctx, a, b, [0, 0, 0])
        for mother, daughter in ((b, a), (a, a)):          # a logical volume may not contain itself
            with pytest.raises(g4.G4NError) as e:
                g4.g4n_logical_add_daughter(ctx, mother, daughter, [0, 0, 0])
            assert e.value.code == -1
        with pytest.raises(g4.G4NError) as e:
            g4.g4n_logical_create(ctx, 7, m)
        assert e.value.code == -1
        with pytest.raises(g4.G4NError) as e:
            g4.g4n_place_logical(ctx, 3, a, [0, 0, 0])     # no world yet: the first placement has mother -1
        assert e.value.code == -1
        # a chain of nested logical volumes deeper than the hierarchy limit
        chain = [g4.g4n_logical_create(ctx, g4.g4n_solid_box(ctx, 500.0 - k, 500.0 - k, 500.0 - k), m)
                 for k in range(g4.G4N_DMAX + 1)]
        for k in range(g4.G4N_DMAX):
            g4.g4n_logical_add_daughter(ctx, chain[k], chain[k + 1], [0, 0, 0])
        with pytest.raises(g4.G4NError) as e:
            g4.g4n_place_logical(ctx, -1, chain[0], [0, 0, 0])
        assert e.value.code == -2
    finally:
        g4.g4n_destroy(ctx)


class _FakeCuda:
    """A CPU tensor posing as a CUDA tensor on device `index` (for the binding's argument checks only:
    the checks raise before any library call, so no pointer is ever used)."""

    def __init__(self, t, index=0):
        self.t, self.is_cuda = t, True
        self.device = type("D", (), {"index": index})()

    dtype = property(lambda self: self.t.dtype)
    shape = property(lambda self: self.t.shape)

    def is_contiguous(self):
        return self.t.is_contiguous()

    def numel(self):
        return self.t.numel()

    def dim(self):
        return self.t.dim()

    def data_ptr(self):
        return self.t.data_ptr()


@pytest.mark.parametrize("case", ["counters_short", "hash_short", "len_short", "edep_rows", "wrong_device"])
def test_binding_refuses_undersized_or_misplaced_outputs(g4, case):
    """The transport kernels write G4N_N_COUNTERS counters and one hash / length per track: the binding
    refuses smaller tensors, and tensors on another device than the context's, before calling the library."""
    import torch
    items = g4.make_items([(0, 1000, 0, synth.scenes.tiny_source(), 0), (0, 24, 5000, synth.scenes.tiny_source(), 0)])
    ctx = ctypes_ctx = type("C", (), {"value": 0x1234})()
    g4.binding._CTX_DEVICE[ctypes_ctx.value] = 0
    try:
        edep = _FakeCuda(torch.zeros((100, 13), dtype=torch.float64))
        cnt = _FakeCuda(torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64))
        h = _FakeCuda(torch.zeros(1024, dtype=torch.int64))
        ln = _FakeCuda(torch.zeros(1024, dtype=torch.float64))
        if case == "counters_short":
            cnt = _FakeCuda(torch.zeros(g4.G4N_N_COUNTERS - 1, dtype=torch.int64))
        elif case == "hash_short":
            h = _FakeCuda(torch.zeros(1023, dtype=torch.int64))
        elif case == "len_short":
            ln = _FakeCuda(torch.zeros(1000, dtype=torch.float64))
        elif case == "edep_rows":
            edep = _FakeCuda(torch.zeros((99, 13), dtype=torch.float64))
        else:
            h = _FakeCuda(torch.zeros(1024, dtype=torch.int64), index=1)
        for call in (g4.g4n_transport_batch, g4.g4n_transport_batch_noalloc, g4.g4n_graph_create):
            with pytest.raises(ValueError):
                call(ctx, items, 1, edep, cnt, h, ln)
        # the same arguments at the right sizes pass the checks
        ok = g4.binding._transport_ptrs(ctx, items, _FakeCuda(torch.zeros((100, 13), dtype=torch.float64)),
                                        _FakeCuda(torch.zeros(g4.G4N_N_COUNTERS, dtype=torch.int64)),
                                        _FakeCuda(torch.zeros(1024, dtype=torch.int64)),
                                        _FakeCuda(torch.zeros(1024, dtype=torch.float64)), 100)
        assert len(ok) == 4 and all(p is not None for p in ok)
    finally:
        g4.binding._CTX_DEVICE.pop(ctypes_ctx.value, None)


def test_binding_checks_query_shapes(g4):
    """locate / compute_step / free_path: (3, n) positions and directions, per-query arrays of n."""
    import torch
    ctx = type("C", (), {"value": 0x4321})()
    g4.binding._CTX_DEVICE[ctx.value] = 0
    try:
        pos = _FakeCuda(torch.zeros((3, 10), dtype=torch.float64))
        with pytest.raises(ValueError):
            g4.g4n_locate(ctx, 0, pos, _FakeCuda(torch.zeros((3, 9), dtype=torch.float64)))
        with pytest.raises(ValueError):
            g4.g4n_locate(ctx, 0, pos, pos, out_depth=_FakeCuda(torch.zeros(9, dtype=torch.int32)),
                          out_path=_FakeCuda(torch.zeros((g4.G4N_DMAX, 10), dtype=torch.int32)))
        with pytest.raises(ValueError):
            g4.g4n_free_path(ctx, 0, pos, pos, _FakeCuda(torch.zeros(9, dtype=torch.float64)), 1.0,
                             out_T=_FakeCuda(torch.zeros(10, dtype=torch.float64)),
                             out_steps=_FakeCuda(torch.zeros(10, dtype=torch.int32)))
        with pytest.raises(ValueError):
            g4.g4n_locate(ctx, 0, _FakeCuda(torch.zeros((10, 3), dtype=torch.float64)), pos)
    finally:
        g4.binding._CTX_DEVICE.pop(ctx.value, None)


def test_ctypes_structures_match_the_header_layout(tmp_path):
    """The binding's ctypes mirrors of the ABI structures have the C compiler's size and field offsets (a C
    program built from include/g4nav.h prints them), so that no field of a batch description or work item is
    read from the wrong place."""
    import ctypes
    import os
    import shutil
    import subprocess
    from paper_1209_5235_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"g4n_batch_desc": binding.g4n_batch_desc, "g4n_work_item": binding.g4n_work_item,
               "g4n_source": binding.g4n_source, "g4n_voxel_params": binding.g4n_voxel_params}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "g4nav.h"', "int main(void) {"]
    for name, st in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, st in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
