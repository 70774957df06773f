"""ctypes binding of libg4nav: the C-ABI entry points under the same names.

Every function here only converts arguments (torch tensors -> device
pointers, numpy/sequences -> host arrays, the current torch stream ->
cudaStream_t) and raises ``G4NError`` on a non-zero status.  No navigation,
physics or fallback computation happens in Python: if the shared library is
missing the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libg4nav.so")

G4N_OK, G4N_ERR_ARG, G4N_ERR_GEOM, G4N_ERR_OOM, G4N_ERR_CUDA = 0, -1, -2, -3, -4
G4N_ERR_STEP_LIMIT, G4N_ERR_TIMEOUT, G4N_ERR_QUEUE, G4N_ERR_STATE = -5, -6, -7, -8
G4N_BOX, G4N_TUBE, G4N_ORB, G4N_CONE = 0, 1, 2, 3
G4N_MODE_FP64, G4N_MODE_FP32_RECHECK, G4N_MODE_LEARNED = 0, 1, 2
G4N_LIM_PHYSICS, G4N_LIM_MOTHER = -2, -1
G4N_DMAX = 32
G4N_N_COUNTERS = 32
G4N_FLAG_DIAGNOSTICS = 1
G4N_SCHEDULE_PERSISTENT, G4N_SCHEDULE_STAGED = 0, 1
G4N_STAGED_RELOCATION_KERNEL = 1
G4N_NOALLOC_MAX_ITEMS = 256
G4N_MLP_N_PARAMS = 6880
G4N_NOALLOC_STATUS_SLOT = G4N_N_COUNTERS - 1
COUNTER_NAMES = {0: "tracks", 1: "steps", 2: "geom_steps", 3: "phys_steps", 4: "photo", 5: "compton", 6: "escaped",
                 7: "cutoff", 8: "pushes", 9: "step_limit", 10: "walk_yields", 11: "cand_cone", 12: "dist_out_curved",
                 13: "inside_curved", 14: "face_reloc", 15: "key_inside", 16: "safety_skips", 17: "cand_box", 18: "cand_tube",
                 19: "cand_orb", 20: "dist_out", 21: "inside", 22: "vox_nodes", 23: "rechecks", 24: "proposals",
                 25: "pruned", 26: "cyc_refill", 27: "cyc_interact", 28: "cyc_step", 29: "step_lanes",
                 30: "step_phases"}
PARITY_COUNTERS = ["tracks", "steps", "geom_steps", "phys_steps", "photo", "compton", "escaped", "cutoff", "pushes",
                   "step_limit"]

EXPORTED = ["g4n_create", "g4n_destroy", "g4n_last_error", "g4n_set_tolerance_scale", "g4n_sync", "g4n_set_loop_caps",
            "g4n_kernel_launches",
            "g4n_material_add",
            "g4n_solid_box", "g4n_solid_tube", "g4n_solid_orb", "g4n_solid_cone", "g4n_place",
            "g4n_logical_create", "g4n_logical_add_daughter", "g4n_place_logical", "g4n_touchable", "g4n_voxelize", "g4n_geom_finalize",
            "g4n_geom_info", "g4n_locate", "g4n_compute_step", "g4n_free_path", "g4n_transport_batch", "g4n_transport_batch_host",
            "g4n_transport_batch_noalloc", "g4n_mlp_load", "g4n_mlp_get", "g4n_mlp_log", "g4n_mlp_train",
            "g4n_mlp_grad", "g4n_mlp_predict", "g4n_graph_create", "g4n_graph_launch", "g4n_graph_destroy"]

__all__ = EXPORTED + ["G4N_FLAG_DIAGNOSTICS", "G4N_SCHEDULE_PERSISTENT", "G4N_SCHEDULE_STAGED", "G4N_STAGED_RELOCATION_KERNEL", "G4NError", "load", "lib_path", "build_scene", "build_logical_scene", "make_items", "counters_dict", "voxel_params",
                      "COUNTER_NAMES", "PARITY_COUNTERS", "G4N_DMAX", "G4N_N_COUNTERS", "G4N_MODE_FP64",
                      "G4N_MODE_FP32_RECHECK", "G4N_MODE_LEARNED", "G4N_LIM_PHYSICS", "G4N_LIM_MOTHER",
                      "G4N_ERR_ARG", "G4N_ERR_GEOM", "G4N_ERR_OOM", "G4N_ERR_CUDA", "G4N_ERR_STEP_LIMIT", "G4N_ERR_TIMEOUT", "G4N_ERR_STATE",
                      "G4N_NOALLOC_MAX_ITEMS", "G4N_NOALLOC_STATUS_SLOT", "G4N_MLP_N_PARAMS",
                      "g4n_voxel_params", "g4n_source", "g4n_work_item", "g4n_batch_desc"]


class G4NError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libg4nav error {code}: {msg}")
        self.code = code


class g4n_voxel_params(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_levels", ctypes.c_int32), ("axes", ctypes.c_int32 * 3),
                ("slices", ctypes.c_int32 * 3), ("smartless", ctypes.c_double), ("max_slices", ctypes.c_int32),
                ("refine_above", ctypes.c_int32)]


class g4n_source(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("spot_sigma", ctypes.c_double), ("has_z", ctypes.c_int32),
                ("z0", ctypes.c_double), ("z1", ctypes.c_double), ("isotropic", ctypes.c_int32),
                ("dir", ctypes.c_double * 3), ("e_kind", ctypes.c_int32), ("e0", ctypes.c_double),
                ("e1", ctypes.c_double)]


class g4n_work_item(ctypes.Structure):
    _fields_ = [("geom", ctypes.c_int32), ("n_tracks", ctypes.c_int64), ("track_id0", ctypes.c_int64),
                ("source", g4n_source), ("tally_offset", ctypes.c_int64)]


class g4n_batch_desc(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("items", ctypes.POINTER(g4n_work_item)), ("seed", ctypes.c_uint64),
                ("cutoff", ctypes.c_double), ("mode", ctypes.c_int32), ("n_tally_batches", ctypes.c_int32),
                ("tally_stride", ctypes.c_int64), ("max_steps", ctypes.c_int64), ("block_size", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("refill_min", ctypes.c_int32), ("interact_min", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("walk_budget", ctypes.c_int32), ("regroup_period", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("staged_flags", ctypes.c_int32), ("pool_tracks", ctypes.c_int64),
                ("drain_tracks", ctypes.c_int64)]


_lib = None


def lib_path() -> str:
    return LIB_PATH


def load():
    """Load libg4nav.so (built by ``paper_1209_5235_gb300.build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libg4nav.so is not built ({LIB_PATH}); run paper_1209_5235_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "g4n_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int],
        "g4n_destroy": [vp], "g4n_set_tolerance_scale": [vp, d], "g4n_sync": [vp, vp],
        "g4n_set_loop_caps": [vp, i32, i32],
        "g4n_material_add": [vp, d, i32, vp, vp, vp, vp],
        "g4n_solid_box": [vp, d, d, d, vp], "g4n_solid_tube": [vp, d, d, d, d, d, vp], "g4n_solid_orb": [vp, d, vp],
        "g4n_solid_cone": [vp, d, d, d, d, d, vp],
        "g4n_logical_create": [vp, i32, i32, vp], "g4n_logical_add_daughter": [vp, i32, i32, vp, vp, vp],
        "g4n_place_logical": [vp, i32, i32, vp, vp, vp, vp], "g4n_touchable": [vp, i32, i32, i32, vp, vp, vp],
        "g4n_place": [vp, i32, i32, i32, vp, vp, vp], "g4n_voxelize": [vp, ctypes.POINTER(g4n_voxel_params)],
        "g4n_geom_finalize": [vp, vp], "g4n_geom_info": [vp, i32, vp],
        "g4n_locate": [vp, i32, i64, vp, vp, vp, vp, vp],
        "g4n_compute_step": [vp, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp],
        "g4n_free_path": [vp, i32, i64, vp, vp, vp, d, vp, vp, vp, i32, i64, i32, vp],
        "g4n_transport_batch": [vp, ctypes.POINTER(g4n_batch_desc), vp, vp, vp, vp, vp],
        "g4n_transport_batch_host": [vp, ctypes.POINTER(g4n_batch_desc), vp, vp, vp, vp, vp],
        "g4n_transport_batch_noalloc": [vp, ctypes.POINTER(g4n_batch_desc), vp, vp, vp, vp, vp],
        "g4n_mlp_load": [vp, vp], "g4n_mlp_get": [vp, vp],
        "g4n_mlp_log": [vp, ctypes.POINTER(g4n_batch_desc), vp, vp, vp, i64, vp, vp],
        "g4n_mlp_train": [vp, i64, vp, vp, vp, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp],
        "g4n_mlp_grad": [vp, i64, vp, vp, vp, i32, vp, vp],
        "g4n_mlp_predict": [vp, i64, vp, vp, vp],
        "g4n_graph_create": [vp, ctypes.POINTER(g4n_batch_desc), vp, vp, vp, vp, ctypes.POINTER(ctypes.c_void_p)],
        "g4n_graph_launch": [vp, ctypes.c_uint64, vp], "g4n_graph_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.g4n_last_error.argtypes = [vp]
    L.g4n_last_error.restype = ctypes.c_char_p
    L.g4n_kernel_launches.argtypes = [vp]
    L.g4n_kernel_launches.restype = ctypes.c_int64
    _lib = L
    return L


def _check(ctx, rc: int):
    if rc != G4N_OK:
        msg = load().g4n_last_error(ctx) if ctx else b""
        raise G4NError(rc, (msg or b"").decode())
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


_CTX_DEVICE = {}   # context handle -> its CUDA device (set by g4n_create)


def _dptr(t, dtype, name, min_numel: int = 0, device: Optional[int] = None):
    """Device pointer of a contiguous CUDA tensor of the given dtype (None -> NULL), holding at least
    `min_numel` elements and, when `device` is given, on that CUDA device.  The kernels write every
    element they are told exists, so an undersized or misplaced tensor is refused here."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA tensor of {dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: {t.numel()} elements, need at least {min_numel}")
    if device is not None and t.device.index is not None and t.device.index != device:
        raise ValueError(f"{name}: tensor on cuda:{t.device.index}, the context is on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


def _ctx_device(ctx) -> Optional[int]:
    return _CTX_DEVICE.get(getattr(ctx, "value", ctx))


def _n_tracks(items) -> int:
    return int(sum(max(0, int(items[k].n_tracks)) for k in range(len(items))))


def _transport_ptrs(ctx, items, edep, counters, track_hash, track_len, n_batches):
    """Checked device pointers of a transport's outputs: edep (n_batches, stride) float64, counters
    (>= G4N_N_COUNTERS) int64, per-track hash / length (>= the batch's track count), all on the
    context's device."""
    import torch
    if edep.dim() != 2 or edep.shape[0] != n_batches:
        raise ValueError("edep: need shape (n_batches, tally_stride)")
    dev = _ctx_device(ctx)
    n = _n_tracks(items)
    return (_dptr(edep, torch.float64, "edep", n_batches * edep.shape[1], dev),
            _dptr(counters, torch.int64, "counters", G4N_N_COUNTERS, dev),
            _dptr(track_hash, torch.int64, "track_hash", n, dev),
            _dptr(track_len, torch.float64, "track_len", n, dev))


def _soa3(t, name, n=None):
    """A (3, n) structure-of-arrays tensor; returns n."""
    if t.dim() != 2 or t.shape[0] != 3 or (n is not None and t.shape[1] != n):
        raise ValueError(f"{name}: need shape (3, n)" + (f" with n = {n}" if n is not None else ""))
    return int(t.shape[1])


def _host(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


# ---------------------------------------------------------------- context

def g4n_create(device: int = 0):
    ctx = ctypes.c_void_p()
    rc = load().g4n_create(ctypes.byref(ctx), int(device))
    if rc != G4N_OK:
        raise G4NError(rc, "g4n_create failed (no CUDA device?)")
    if int(device) >= 0:
        _CTX_DEVICE[ctx.value] = int(device)
    return ctx


def g4n_destroy(ctx) -> None:
    _CTX_DEVICE.pop(getattr(ctx, "value", ctx), None)
    load().g4n_destroy(ctx)


def g4n_last_error(ctx) -> str:
    return (load().g4n_last_error(ctx) or b"").decode()


def g4n_set_tolerance_scale(ctx, scale: float) -> None:
    _check(ctx, load().g4n_set_tolerance_scale(ctx, float(scale)))


def g4n_sync(ctx, stream=None) -> None:
    _check(ctx, load().g4n_sync(ctx, _stream(stream)))


def g4n_kernel_launches(ctx) -> int:
    """Kernels the context has launched so far (a monotonic count)."""
    return int(load().g4n_kernel_launches(ctx))


def g4n_set_loop_caps(ctx, max_walk_nodes: int = 0, max_sampler_trials: int = 0) -> None:
    """Caps of the device loops (0 = default: 65536 voxel nodes per search, 1000 sampler trials)."""
    _check(ctx, load().g4n_set_loop_caps(ctx, int(max_walk_nodes), int(max_sampler_trials)))


# ---------------------------------------------------------------- geometry build

def g4n_material_add(ctx, density: float, energies, mu_compton, mu_photo) -> int:
    e, c, p = _host(energies, np.float64), _host(mu_compton, np.float64), _host(mu_photo, np.float64)
    out = ctypes.c_int32()
    _check(ctx, load().g4n_material_add(ctx, float(density), int(e.shape[0]), e.ctypes.data, c.ctypes.data,
                                        p.ctypes.data, ctypes.byref(out)))
    return out.value


def g4n_solid_box(ctx, hx: float, hy: float, hz: float) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_solid_box(ctx, float(hx), float(hy), float(hz), ctypes.byref(out)))
    return out.value


def g4n_solid_tube(ctx, rmin: float, rmax: float, hz: float, sphi: float, dphi: float) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_solid_tube(ctx, float(rmin), float(rmax), float(hz), float(sphi), float(dphi),
                                      ctypes.byref(out)))
    return out.value


def g4n_solid_cone(ctx, rmin1: float, rmax1: float, rmin2: float, rmax2: float, hz: float) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_solid_cone(ctx, float(rmin1), float(rmax1), float(rmin2), float(rmax2), float(hz),
                                      ctypes.byref(out)))
    return out.value


def g4n_solid_orb(ctx, r: float) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_solid_orb(ctx, float(r), ctypes.byref(out)))
    return out.value


def g4n_place(ctx, mother: int, solid: int, mat: int, t: Sequence[float], rot: Optional[Sequence[float]] = None) -> int:
    tt = _host(t, np.float64)
    rr = _host(rot, np.float64) if rot is not None else None
    out = ctypes.c_int32()
    _check(ctx, load().g4n_place(ctx, int(mother), int(solid), int(mat), tt.ctypes.data,
                                 rr.ctypes.data if rr is not None else None, ctypes.byref(out)))
    return out.value


def _rot(rot):
    return (ctypes.c_double * 2)(*[float(x) for x in rot]) if rot is not None else None


def g4n_logical_create(ctx, solid: int, mat: int) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_logical_create(ctx, int(solid), int(mat), ctypes.byref(out)))
    return out.value


def g4n_logical_add_daughter(ctx, mother_lv: int, daughter_lv: int, t: Sequence[float],
                             rot: Optional[Sequence[float]] = None) -> int:
    tt = (ctypes.c_double * 3)(*[float(x) for x in t])
    out = ctypes.c_int32()
    _check(ctx, load().g4n_logical_add_daughter(ctx, int(mother_lv), int(daughter_lv), tt, _rot(rot), ctypes.byref(out)))
    return out.value


def g4n_place_logical(ctx, mother: int, lv: int, t: Sequence[float], rot: Optional[Sequence[float]] = None):
    """Returns (first volume id, number of volumes) of the expanded subtree."""
    tt = (ctypes.c_double * 3)(*[float(x) for x in t])
    first, n = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, load().g4n_place_logical(ctx, int(mother), int(lv), tt, _rot(rot), ctypes.byref(first), ctypes.byref(n)))
    return first.value, n.value


def g4n_touchable(ctx, geom: int, vol: int):
    """[(logical volume, copy number)] from the world down to vol."""
    lv = (ctypes.c_int32 * G4N_DMAX)()
    cp = (ctypes.c_int32 * G4N_DMAX)()
    depth = ctypes.c_int32()
    _check(ctx, load().g4n_touchable(ctx, int(geom), int(vol), G4N_DMAX, lv, cp, ctypes.byref(depth)))
    return [(lv[k], cp[k]) for k in range(depth.value)]


def build_logical_scene(ctx, base, logicals, placements) -> int:
    """Marshal a scene whose base placements are given directly and whose logical volumes
    (synth.scenes.LogicalVolume) are placed through the logical-volume calls; geometry id."""
    mats = [g4n_material_add(ctx, m.density, m.energies, m.mu_compton, m.mu_photo) for m in base.materials]
    solids = []
    for s in base.solids:
        f = {G4N_BOX: g4n_solid_box, G4N_TUBE: g4n_solid_tube, G4N_CONE: g4n_solid_cone}.get(s.kind, g4n_solid_orb)
        solids.append(f(ctx, *s.params))
    for pl in base.placements:
        g4n_place(ctx, pl.mother, solids[pl.solid], mats[pl.material], pl.t, pl.rot)
    lvs = [g4n_logical_create(ctx, solids[lv.solid], mats[lv.material]) for lv in logicals]
    for k, lv in enumerate(logicals):
        for d in lv.daughters:
            g4n_logical_add_daughter(ctx, lvs[k], lvs[d.lv], d.t, d.rot)
    for p in placements:
        g4n_place_logical(ctx, p.mother, lvs[p.lv], p.t, p.rot)
    g4n_voxelize(ctx, voxel_params(base.voxel))
    return g4n_geom_finalize(ctx)


def voxel_params(spec) -> g4n_voxel_params:
    """g4n_voxel_params from a synth.VoxelSpec-like object."""
    p = g4n_voxel_params()
    p.mode = {"smart": 0, "fixed": 1, "none": 2}[spec.mode]
    p.n_levels = len(spec.axes) if spec.mode == "fixed" else getattr(spec, "max_levels", 3)
    for k, a in enumerate(spec.axes):
        p.axes[k] = a
    for k, s in enumerate(spec.slices):
        p.slices[k] = s
    p.smartless = float(spec.smartless)
    p.max_slices = int(spec.max_slices)
    p.refine_above = int(spec.refine_above)
    return p


def g4n_voxelize(ctx, params: g4n_voxel_params) -> None:
    _check(ctx, load().g4n_voxelize(ctx, ctypes.byref(params)))


def g4n_geom_finalize(ctx) -> int:
    out = ctypes.c_int32()
    _check(ctx, load().g4n_geom_finalize(ctx, ctypes.byref(out)))
    return out.value


def g4n_geom_info(ctx, geom: int) -> dict:
    out = np.zeros(8, dtype=np.int64)
    _check(ctx, load().g4n_geom_info(ctx, int(geom), out.ctypes.data))
    keys = ["n_volumes", "n_voxel_headers", "n_voxel_slices", "n_candidate_lists", "n_candidate_entries",
            "device_bytes", "max_depth", "n_materials"]
    return dict(zip(keys, out.tolist()))


def build_scene(ctx, scene) -> int:
    """Marshal a synth.Scene through the geometry-build calls; returns the geometry id."""
    mats = [g4n_material_add(ctx, m.density, m.energies, m.mu_compton, m.mu_photo) for m in scene.materials]
    solids = []
    for s in scene.solids:
        if s.kind == G4N_BOX:
            solids.append(g4n_solid_box(ctx, *s.params))
        elif s.kind == G4N_TUBE:
            solids.append(g4n_solid_tube(ctx, *s.params))
        elif s.kind == G4N_CONE:
            solids.append(g4n_solid_cone(ctx, *s.params))
        else:
            solids.append(g4n_solid_orb(ctx, *s.params))
    for pl in scene.placements:
        g4n_place(ctx, pl.mother, solids[pl.solid], mats[pl.material], pl.t, pl.rot)
    g4n_voxelize(ctx, voxel_params(scene.voxel))
    return g4n_geom_finalize(ctx)


# ---------------------------------------------------------------- queries

def g4n_locate(ctx, geom: int, pos, dir, out_depth=None, out_path=None, stream=None):
    """pos, dir: (3, n) float64 CUDA tensors (SoA).  Returns (depth (n,) int32, path (G4N_DMAX, n) int32)."""
    import torch
    n = _soa3(pos, "pos")
    _soa3(dir, "dir", n)
    if out_depth is None:
        out_depth = torch.empty(n, dtype=torch.int32, device=pos.device)
    if out_path is None:
        out_path = torch.empty((G4N_DMAX, n), dtype=torch.int32, device=pos.device)
    dev = _ctx_device(ctx)
    args = (_dptr(pos, torch.float64, "pos", 3 * n, dev), _dptr(dir, torch.float64, "dir", 3 * n, dev),
            _dptr(out_depth, torch.int32, "out_depth", n, dev), _dptr(out_path, torch.int32, "out_path", G4N_DMAX * n, dev))
    _check(ctx, load().g4n_locate(ctx, int(geom), int(n), *args, _stream(stream)))
    return out_depth, out_path


def g4n_compute_step(ctx, geom: int, pos, dir, depth, path, proposed=None, mode: int = G4N_MODE_FP64, stream=None,
                     out=None):
    """Returns (step (n,) f64, safety (n,) f64, limiter (n,) int32); `out` may give those three tensors."""
    import torch
    n = _soa3(pos, "pos")
    _soa3(dir, "dir", n)
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, device=pos.device), torch.empty(n, dtype=torch.float64, device=pos.device),
               torch.empty(n, dtype=torch.int32, device=pos.device))
    step, saf, lim = out
    dev = _ctx_device(ctx)
    args = (_dptr(pos, torch.float64, "pos", 3 * n, dev), _dptr(dir, torch.float64, "dir", 3 * n, dev),
            _dptr(depth, torch.int32, "depth", n, dev), _dptr(path, torch.int32, "path", G4N_DMAX * n, dev),
            _dptr(proposed, torch.float64, "proposed", n, dev), _dptr(step, torch.float64, "step", n, dev),
            _dptr(saf, torch.float64, "safety", n, dev), _dptr(lim, torch.int32, "limiter", n, dev))
    _check(ctx, load().g4n_compute_step(ctx, int(geom), int(n), *args, int(mode), _stream(stream)))
    return step, saf, lim


def g4n_free_path(ctx, geom: int, pos, dir, Y, energy: float, mode: int = G4N_MODE_FP64, counters=None,
                  max_steps: int = 0, diagnostics: bool = False, want_steps: bool = True, out_T=None, out_steps=None,
                  stream=None):
    """Free path T of Algorithm 1 per ray.  Returns (T (n,) f64, steps (n,) int32 or None); `counters`
    (G4N_N_COUNTERS int64 device tensor) is accumulated if given."""
    import torch
    n = _soa3(pos, "pos")
    _soa3(dir, "dir", n)
    T = out_T if out_T is not None else torch.empty(n, dtype=torch.float64, device=pos.device)
    st = out_steps if out_steps is not None else (torch.empty(n, dtype=torch.int32, device=pos.device) if want_steps
                                                  else None)
    dev = _ctx_device(ctx)
    args = (_dptr(pos, torch.float64, "pos", 3 * n, dev), _dptr(dir, torch.float64, "dir", 3 * n, dev),
            _dptr(Y, torch.float64, "Y", n, dev), float(energy), _dptr(T, torch.float64, "T", n, dev),
            _dptr(st, torch.int32, "steps", n, dev), _dptr(counters, torch.int64, "counters", G4N_N_COUNTERS, dev))
    _check(ctx, load().g4n_free_path(ctx, int(geom), int(n), *args, int(mode), int(max_steps),
                                     G4N_FLAG_DIAGNOSTICS if diagnostics else 0, _stream(stream)))
    return T, st


def make_items(entries) -> "ctypes.Array":
    """Work items from (geom, n_tracks, track_id0, synth.Source, tally_offset) tuples."""
    arr = (g4n_work_item * len(entries))()
    for k, (geom, n, tid0, src, off) in enumerate(entries):
        w = arr[k]
        w.geom, w.n_tracks, w.track_id0, w.tally_offset = int(geom), int(n), int(tid0), int(off)
        s = w.source
        for i in range(3):
            s.pos[i] = float(src.pos[i])
            s.dir[i] = float(src.direction[i])
        s.spot_sigma = float(src.spot_sigma)
        s.has_z = 1 if src.z_range is not None else 0
        s.z0, s.z1 = (float(src.z_range[0]), float(src.z_range[1])) if src.z_range is not None else (0.0, 0.0)
        s.isotropic = 1 if src.isotropic else 0
        s.e_kind = {"mono": 0, "uniform": 1, "loguniform": 2}[src.e_kind]
        s.e0, s.e1 = float(src.e0), float(src.e1)
    return arr


def _desc(items, seed, cutoff, mode, n_batches, stride, max_steps, block_size, blocks_per_sm, refill_min=0,
          interact_min=0, diagnostics=False, walk_budget=0, regroup_period=0, schedule=0, pool_tracks=0,
          drain_tracks=0, staged_flags=0):
    d = g4n_batch_desc()
    d.n_items = len(items)
    d.items = ctypes.cast(items, ctypes.POINTER(g4n_work_item))
    d.seed = ctypes.c_uint64(seed).value
    d.cutoff = float(cutoff)
    d.mode = int(mode)
    d.n_tally_batches = int(n_batches)
    d.tally_stride = int(stride)
    d.max_steps = int(max_steps)
    d.block_size, d.blocks_per_sm = int(block_size), int(blocks_per_sm)
    d.refill_min, d.interact_min = int(refill_min), int(interact_min)
    d.flags = G4N_FLAG_DIAGNOSTICS if diagnostics else 0
    d.walk_budget = int(walk_budget)
    d.regroup_period = int(regroup_period)
    d.schedule = int(schedule)
    d.pool_tracks = int(pool_tracks)
    d.drain_tracks = int(drain_tracks)
    d.staged_flags = int(staged_flags)
    return d


def g4n_transport_batch(ctx, items, seed: int, edep, counters, track_hash=None, track_len=None, cutoff: float = 0.01,
                        mode: int = G4N_MODE_FP64, n_batches: int = 100, max_steps: int = 0, block_size: int = 0,
                        blocks_per_sm: int = 0, refill_min: int = 0, interact_min: int = 0,
                        diagnostics: bool = False, stream=None, walk_budget: int = 0, regroup_period: int = 0,
        schedule: int = 0, pool_tracks: int = 0, drain_tracks: int = 0,
        staged_flags: int = 0) -> None:
    """Device outputs (accumulated): edep (n_batches, stride) f64, counters (32,) int64 (as uint64 bits)."""
    ptrs = _transport_ptrs(ctx, items, edep, counters, track_hash, track_len, n_batches)
    d = _desc(items, seed, cutoff, mode, n_batches, edep.shape[1], max_steps, block_size, blocks_per_sm, refill_min,
              interact_min, diagnostics, walk_budget, regroup_period, schedule, pool_tracks,
              drain_tracks, staged_flags)
    _check(ctx, load().g4n_transport_batch(ctx, ctypes.byref(d), *ptrs, _stream(stream)))


def g4n_transport_batch_noalloc(ctx, items, seed: int, edep, counters, track_hash=None, track_len=None,
                                cutoff: float = 0.01, mode: int = G4N_MODE_FP64, n_batches: int = 100,
                                max_steps: int = 0, block_size: int = 0, blocks_per_sm: int = 0, refill_min: int = 0,
                                interact_min: int = 0, diagnostics: bool = False, stream=None,
                                walk_budget: int = 0, regroup_period: int = 0,
        schedule: int = 0, pool_tracks: int = 0, drain_tracks: int = 0,
        staged_flags: int = 0) -> None:
    """The allocation-free variant of g4n_transport_batch (at most G4N_NOALLOC_MAX_ITEMS items).

    For callers that must not allocate device memory while running: the library keeps this call's
    scratch in a fixed device array instead of a cudaMalloc'd workspace.  Device-side errors are
    written to counters[G4N_NOALLOC_STATUS_SLOT] (0 = none) instead of being reported by g4n_sync.
    """
    ptrs = _transport_ptrs(ctx, items, edep, counters, track_hash, track_len, n_batches)
    d = _desc(items, seed, cutoff, mode, n_batches, edep.shape[1], max_steps, block_size, blocks_per_sm, refill_min,
              interact_min, diagnostics, walk_budget, regroup_period, schedule, pool_tracks,
              drain_tracks, staged_flags)
    _check(ctx, load().g4n_transport_batch_noalloc(ctx, ctypes.byref(d), *ptrs, _stream(stream)))


def g4n_transport_batch_host(ctx, items, seed: int, stride: int, n_tracks: int = 0, want_hash: bool = False,
                             want_len: bool = False, cutoff: float = 0.01, mode: int = G4N_MODE_FP64,
                             n_batches: int = 100, max_steps: int = 0, block_size: int = 0, blocks_per_sm: int = 0,
                             refill_min: int = 0, interact_min: int = 0, diagnostics: bool = False, stream=None,
                             out=None, walk_budget: int = 0, regroup_period: int = 0,
        schedule: int = 0, pool_tracks: int = 0, drain_tracks: int = 0,
        staged_flags: int = 0):
    """Host-buffer variant: returns dict of numpy arrays (edep, counters, hashes, lengths)."""
    d = _desc(items, seed, cutoff, mode, n_batches, stride, max_steps, block_size, blocks_per_sm, refill_min,
              interact_min, diagnostics, walk_budget, regroup_period, schedule, pool_tracks,
              drain_tracks, staged_flags)
    if out is None:
        out = {"edep": np.zeros((n_batches, stride)), "counters": np.zeros(G4N_N_COUNTERS, dtype=np.uint64),
               "hashes": np.zeros(n_tracks, dtype=np.uint64) if want_hash else None,
               "lengths": np.zeros(n_tracks) if want_len else None}
    rc = load().g4n_transport_batch_host(ctx, ctypes.byref(d), out["edep"].ctypes.data, out["counters"].ctypes.data,
                                         out["hashes"].ctypes.data if out["hashes"] is not None else None,
                                         out["lengths"].ctypes.data if out["lengths"] is not None else None,
                                         _stream(stream))
    _check(ctx, rc)
    return out


def counters_dict(counters) -> dict:
    """Name -> value for a counter array (numpy uint64 or torch int64)."""
    a = counters.cpu().numpy() if hasattr(counters, "cpu") else np.asarray(counters)
    a = a.view(np.uint64) if a.dtype == np.int64 else a
    return {name: int(a[k]) for k, name in COUNTER_NAMES.items()}


# ---------------------------------------------------------------- learned proposal

def g4n_mlp_load(ctx, params) -> None:
    """Load packed FP32 parameters (G4N_MLP_N_PARAMS floats)."""
    a = _host(params, np.float32)
    if a.size != G4N_MLP_N_PARAMS:
        raise ValueError("need G4N_MLP_N_PARAMS parameters")
    _check(ctx, load().g4n_mlp_load(ctx, a.ctypes.data))


def g4n_mlp_get(ctx) -> np.ndarray:
    out = np.zeros(G4N_MLP_N_PARAMS, dtype=np.float32)
    _check(ctx, load().g4n_mlp_get(ctx, out.ctypes.data))
    return out


def g4n_mlp_log(ctx, items, seed: int, capacity: int, stride: int, cutoff: float = 0.01, n_batches: int = 100,
                stream=None):
    """Samples logged by the plain navigator: (feat (n, 9) f32, label (n,) i32, ncand (n,) i32) CUDA tensors."""
    import torch
    feat = torch.empty((capacity, 9), dtype=torch.float32, device="cuda")
    label = torch.empty(capacity, dtype=torch.int32, device="cuda")
    ncand = torch.empty(capacity, dtype=torch.int32, device="cuda")
    d = _desc(items, seed, cutoff, G4N_MODE_FP64, n_batches, stride, 0, 0, 0)
    count = ctypes.c_int64()
    _check(ctx, load().g4n_mlp_log(ctx, ctypes.byref(d), _dptr(feat, torch.float32, "feat"),
                                   _dptr(label, torch.int32, "label"), _dptr(ncand, torch.int32, "ncand"),
                                   int(capacity), ctypes.byref(count), _stream(stream)))
    n = count.value
    return feat[:n], label[:n], ncand[:n]


def g4n_mlp_train(ctx, feat, label, ncand, epochs: int = 1, batch: int = 4096, lr: float = 1e-3, seed: int = 1,
                  stream=None) -> np.ndarray:
    """Train in place on device samples; returns the mean loss of each epoch."""
    import torch
    out = np.zeros(epochs, dtype=np.float32)
    _check(ctx, load().g4n_mlp_train(ctx, int(feat.shape[0]), _dptr(feat, torch.float32, "feat"),
                                     _dptr(label, torch.int32, "label"), _dptr(ncand, torch.int32, "ncand"),
                                     int(epochs), int(batch), float(lr), ctypes.c_uint64(seed), out.ctypes.data,
                                     _stream(stream)))
    return out


def g4n_mlp_grad(ctx, feat, label, ncand, precision: int = 0):
    """(mean loss, gradient (G4N_MLP_N_PARAMS,) float32) at the current parameters; precision 0 BF16, 1 FP32."""
    import torch
    g = np.zeros(G4N_MLP_N_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _check(ctx, load().g4n_mlp_grad(ctx, int(feat.shape[0]), _dptr(feat, torch.float32, "feat"),
                                    _dptr(label, torch.int32, "label"), _dptr(ncand, torch.int32, "ncand"),
                                    int(precision), g.ctypes.data, ctypes.byref(loss)))
    return loss.value, g


def g4n_mlp_predict(ctx, feat, stream=None):
    """Logits (n, 32) float32 CUDA tensor for feature rows (n, 9)."""
    import torch
    out = torch.empty((feat.shape[0], 32), dtype=torch.float32, device=feat.device)
    _check(ctx, load().g4n_mlp_predict(ctx, int(feat.shape[0]), _dptr(feat, torch.float32, "feat"),
                                       _dptr(out, torch.float32, "logits"), _stream(stream)))
    return out


# ---------------------------------------------------------------- CUDA graphs

def g4n_graph_create(ctx, items, seed: int, edep, counters, track_hash=None, track_len=None, cutoff: float = 0.01,
                     mode: int = G4N_MODE_FP64, n_batches: int = 100, max_steps: int = 0, block_size: int = 0,
                     blocks_per_sm: int = 0, refill_min: int = 0, interact_min: int = 0, diagnostics: bool = False,
                     walk_budget: int = 0, regroup_period: int = 0,
        schedule: int = 0, pool_tracks: int = 0, drain_tracks: int = 0,
        staged_flags: int = 0):
    """Record the batch as a CUDA graph writing into the given device outputs; returns the handle."""
    ptrs = _transport_ptrs(ctx, items, edep, counters, track_hash, track_len, n_batches)
    d = _desc(items, seed, cutoff, mode, n_batches, edep.shape[1], max_steps, block_size, blocks_per_sm, refill_min,
              interact_min, diagnostics, walk_budget, regroup_period, schedule, pool_tracks,
              drain_tracks, staged_flags)
    h = ctypes.c_void_p()
    _check(ctx, load().g4n_graph_create(ctx, ctypes.byref(d), *ptrs, ctypes.byref(h)))
    return (ctx, h)


def g4n_graph_launch(graph, seed: int, stream=None) -> None:
    ctx, h = graph
    _check(ctx, load().g4n_graph_launch(h, ctypes.c_uint64(seed), _stream(stream)))


def g4n_graph_destroy(graph) -> None:
    ctx, h = graph
    load().g4n_graph_destroy(h)
