"""Plain FP64 CPU oracle for the navigation/transport path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library neither imports nor
links it and shares no code with it; both consume the scene descriptions of
the ``synth`` package.

The arithmetic lives in ``g4oracle.c`` (plain C, IEEE double, contraction
off); this module compiles it with gcc and wraps it with ctypes.

Parity status of each function (how it is pinned, see ``tests/test_oracle_*``):
  * solids (box, orb, tube segment, cone): closed-form ray/solid distances, a
    bisection march on Inside() for segments, cones and rotated solids, a cone
    with equal end radii against the tube, safety checked against sampled
    distances;
  * locate / compute_step / relocate: brute force is the definition itself;
    checked by invariants (locate/step consistency, jitter stability, hand
    built scenes with known answers);
  * Philox4x32-10: known-answer vectors of the published generator;
  * FNV-1a: the published test vectors;
  * attenuation / free path (Eqs. 2-8): uncollided fraction through a slab vs
    exp(-mu x), and the free-path CDF of a two-layer medium (KS test);
  * Kahn sampling: histogram of E'/E vs the Klein-Nishina differential law;
  * Compton direction change (rotate): unit norm, u.u' = cos theta of Compton's
    relation from the recorded energies, azimuth uniform and right-handed in an
    independently built frame, the u = +-z special cases;
  * transport: energy conservation and the closed-form slab limits; the trace
    is the transport loop with a recorder, and its hashed records reproduce the
    history hash, step count and path length.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "g4oracle.c")
_LIB_PATH = os.path.join(_HERE, "libg4oracle.so")
_lock = threading.Lock()
_lib = None

N_COUNTERS = 16
COUNTER_NAMES = ["tracks", "steps", "geom_steps", "phys_steps", "photo", "compton", "escaped", "cutoff",
                 "pushes", "step_limit", "dist_in_evals", "inside_tests"]
DMAX = 32
LIM_PHYS, LIM_MOTHER = -2, -1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, -ffp-contract=off, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                   "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        d, i, i64, u64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        sig = {
            "o_set_scale": (None, [d]), "o_tolerance": (d, []),
            "o_new_geom": (i, []), "o_free_all": (None, []),
            "o_add_material": (i, [i, d, i, vp, vp, vp]), "o_add_solid": (i, [i, i, vp]),
            "o_add_volume": (i, [i, i, i, i, vp, d, d]), "o_finalize": (i, [i]), "o_n_volumes": (i, [i]),
            "o_solid_inside": (i, [i, i, vp, vp]), "o_solid_dist_in": (d, [i, i, vp, vp]),
            "o_solid_dist_out": (d, [i, i, vp, vp]), "o_solid_safety_in": (d, [i, i, vp]),
            "o_solid_safety_out": (d, [i, i, vp]),
            "o_locate": (i, [i, vp, vp, vp]), "o_relocate": (i, [i, vp, i, vp, vp]),
            "o_compute_step": (i, [i, i, vp, vp, vp, d, vp, vp, vp]),
            "o_philox4x32_10": (None, [vp, vp, vp]), "o_uniform": (d, [u64, i64, ctypes.c_uint32, ctypes.c_uint32]),
            "o_uniform_pair": (None, [u64, i64, ctypes.c_uint32, ctypes.c_uint32, vp]),
            "o_fnv1a": (u64, [vp, i64]), "o_mu": (None, [i, i, d, vp]),
            "o_kahn_sample": (i, [d, u64, i64, i64, vp, vp]),
            "o_source_sample": (None, [vp, u64, i64, i64, vp, vp, vp]),
            "o_transport": (i, [i, vp, u64, i64, i64, d, i64, i, vp, vp, vp, vp, i]),
            "o_free_path": (d, [i, vp, vp, d, d, vp]),
            "o_free_path_many": (i, [i, i64, vp, vp, d, vp, vp, vp, i]),
            "o_locate_many": (None, [i, i64, vp, vp, vp, vp]),
            "o_transport_trace": (i, [i, vp, u64, i64, d, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      vp, vp]),
            "o_rotate": (None, [vp, d, d, d, vp]),
            "o_use_grids": (None, [i, i]),
            "o_compute_step_many": (None, [i, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def set_scale(scale: float) -> None:
    lib().o_set_scale(float(scale))


class Geometry:
    """A scene loaded into the oracle (brute-force navigation, no voxels)."""

    def __init__(self, scene):
        L = lib()
        self.scene = scene
        self.gid = L.o_new_geom()
        if self.gid < 0:
            raise RuntimeError("oracle: too many geometries")
        for m in scene.materials:
            e, c, p = _f64(m.energies), _f64(m.mu_compton), _f64(m.mu_photo)
            if L.o_add_material(self.gid, float(m.density), int(e.shape[0]), _p(e), _p(c), _p(p)) < 0:
                raise ValueError(f"oracle: bad material {m.name}")
        for s in scene.solids:
            par = _f64(list(s.params) + [0.0] * (5 - len(s.params)))
            if L.o_add_solid(self.gid, int(s.kind), _p(par)) < 0:
                raise ValueError(f"oracle: bad solid {s}")
        for pl in scene.placements:
            t = _f64(pl.t)
            if L.o_add_volume(self.gid, int(pl.mother), int(pl.solid), int(pl.material), _p(t),
                              float(pl.rot[0]), float(pl.rot[1])) < 0:
                raise ValueError(f"oracle: bad placement {pl}")
        rc = L.o_finalize(self.gid)
        if rc != 0:
            raise ValueError(f"oracle: finalize failed ({rc})")
        self.n_volumes = L.o_n_volumes(self.gid)

    def use_grids(self, on: bool = True) -> None:
        """Timing mode: uniform grids over the daughters of every mother with 8 or more (results unchanged)."""
        lib().o_use_grids(self.gid, 1 if on else 0)

    # -- solids (local frame) -------------------------------------------------
    def solid_inside(self, solid: int, p, v) -> bool:
        return bool(lib().o_solid_inside(self.gid, solid, _p(_f64(p)), _p(_f64(v))))

    def solid_dist_in(self, solid: int, p, v) -> float:
        return lib().o_solid_dist_in(self.gid, solid, _p(_f64(p)), _p(_f64(v)))

    def solid_dist_out(self, solid: int, p, v) -> float:
        return lib().o_solid_dist_out(self.gid, solid, _p(_f64(p)), _p(_f64(v)))

    def solid_safety_in(self, solid: int, p) -> float:
        return lib().o_solid_safety_in(self.gid, solid, _p(_f64(p)))

    def solid_safety_out(self, solid: int, p) -> float:
        return lib().o_solid_safety_out(self.gid, solid, _p(_f64(p)))

    # -- navigation ----------------------------------------------------------
    def locate(self, p, v):
        path = np.full(DMAX, -1, dtype=np.int32)
        depth = lib().o_locate(self.gid, _p(_f64(p)), _p(_f64(v)), _p(path))
        return depth, path

    def locate_many(self, pos: np.ndarray, dirs: np.ndarray):
        """pos, dirs: (n, 3).  Returns depth (n,) and paths (n, DMAX)."""
        n = pos.shape[0]
        depth = np.zeros(n, dtype=np.int32)
        paths = np.full((n, DMAX), -1, dtype=np.int32)
        lib().o_locate_many(self.gid, int(n), _p(_f64(pos)), _p(_f64(dirs)), _p(depth), _p(paths))
        return depth, paths

    def trace(self, source, seed: int, tid: int, cutoff: float = 0.01, cap: int = 100000,
              max_steps: int = 1_000_000):
        """One history as the transport computes it (the same loop, with a recorder): per step the state
        before it (pos, dir, E, path, depth, sphys = Y / mu) and its outcome (step, limiter, event); the
        hashed (leaf, limiter, event) records in order; the history's hash, path length and step count."""
        src = _f64(source.as_array())
        pos, dirs = np.zeros((cap, 3)), np.zeros((cap, 3))
        E, steps, sph = np.zeros(cap), np.zeros(cap), np.zeros(cap)
        paths = np.zeros((cap, DMAX), dtype=np.int32)
        depth, lim, ev = np.zeros(cap, dtype=np.int32), np.zeros(cap, dtype=np.int32), np.zeros(cap, dtype=np.int32)
        rec = np.zeros((2 * cap + 2, 3), dtype=np.int32)
        nrec, nsteps = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64)
        h, ln = np.zeros(1, dtype=np.uint64), np.zeros(1)
        n = lib().o_transport_trace(self.gid, _p(src), ctypes.c_uint64(seed), int(tid), float(cutoff), int(max_steps),
                                    int(cap), _p(pos), _p(dirs), _p(E), _p(paths), _p(depth), _p(steps), _p(lim),
                                    _p(sph), _p(ev), _p(rec), _p(nrec), _p(h), _p(ln), _p(nsteps))
        return {"pos": pos[:n], "dir": dirs[:n], "E": E[:n], "path": paths[:n], "depth": depth[:n],
                "step": steps[:n], "limiter": lim[:n], "event": ev[:n], "sphys": sph[:n],
                "records": rec[:int(nrec[0])], "hash": int(h[0]), "length": float(ln[0]), "n_steps": int(nsteps[0])}

    def compute_step_many(self, pos, dirs, depth, paths, proposed=None):
        """Brute-force steps for n queries; returns (step, limiter, safety)."""
        n = pos.shape[0]
        step = np.zeros(n)
        lim = np.zeros(n, dtype=np.int32)
        saf = np.zeros(n)
        prop = _f64(proposed) if proposed is not None else None
        lib().o_compute_step_many(self.gid, int(n), _p(_f64(pos)), _p(_f64(dirs)),
                                  _p(np.ascontiguousarray(depth, dtype=np.int32)),
                                  _p(np.ascontiguousarray(paths, dtype=np.int32)),
                                  _p(prop) if prop is not None else None, _p(step), _p(lim), _p(saf))
        return step, lim, saf

    def relocate(self, path, depth: int, p, v):
        path = np.ascontiguousarray(np.asarray(path, dtype=np.int32)).copy()
        nd = lib().o_relocate(self.gid, _p(path), int(depth), _p(_f64(p)), _p(_f64(v)))
        return nd, path

    def compute_step(self, depth: int, path, p, v, proposed: float = np.inf, safety: bool = True):
        path = np.ascontiguousarray(np.asarray(path, dtype=np.int32))
        step = np.zeros(1)
        lim = np.zeros(1, dtype=np.int32)
        saf = np.zeros(1)
        rc = lib().o_compute_step(self.gid, int(depth), _p(path), _p(_f64(p)), _p(_f64(v)), float(proposed),
                                  _p(step), _p(lim), _p(saf) if safety else None)
        if rc != 0:
            raise ValueError("oracle: compute_step outside the world")
        return float(step[0]), int(lim[0]), float(saf[0])

    def mu(self, mat: int, E: float):
        out = np.zeros(2)
        lib().o_mu(self.gid, mat, float(E), _p(out))
        return float(out[0]), float(out[1])

    def free_path(self, p, v, E: float, Y: float):
        ns = np.zeros(1, dtype=np.int64)
        T = lib().o_free_path(self.gid, _p(_f64(p)), _p(_f64(v)), float(E), float(Y), _p(ns))
        return T, int(ns[0])

    def free_path_many(self, p, v, E: float, Y, threads: int = 0):
        """Algorithm 1 free paths of n rays (p, v: (n, 3)); returns (T (n,), steps (n,), threads used)."""
        p, v, Y = _f64(p), _f64(v), _f64(Y)
        n = p.shape[0]
        T = np.empty(n)
        ns = np.zeros(n, dtype=np.int64)
        used = lib().o_free_path_many(self.gid, n, _p(p), _p(v), float(E), _p(Y), _p(T), _p(ns), int(threads))
        return T, ns, used

    def transport(self, source, seed: int, n: int, tid0: int = 0, cutoff: float = 0.01, max_steps: int = 1_000_000,
                  n_batches: int = 100, want_hash: bool = True, want_len: bool = True, threads: int = 0):
        """Transport ``n`` histories; returns dict(tally, counters, hashes, lengths, threads)."""
        src = _f64(source.as_array())
        stride = self.n_volumes + 2
        tally = np.zeros((n_batches, stride))
        cnt = np.zeros(N_COUNTERS, dtype=np.uint64)
        hashes = np.zeros(n, dtype=np.uint64) if want_hash else None
        lens = np.zeros(n) if want_len else None
        used = lib().o_transport(self.gid, _p(src), ctypes.c_uint64(seed), int(tid0), int(n), float(cutoff),
                                 int(max_steps), int(n_batches), _p(tally), _p(cnt),
                                 _p(hashes) if hashes is not None else None,
                                 _p(lens) if lens is not None else None, int(threads))
        return {"tally": tally, "counters": cnt, "hashes": hashes, "lengths": lens, "threads": used}


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().o_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniform(seed: int, tid: int, stream: int, draw: int) -> float:
    return lib().o_uniform(ctypes.c_uint64(seed), int(tid), stream, draw)


def uniform_pair(seed: int, tid: int, stream: int, draw: int):
    out = np.zeros(2)
    lib().o_uniform_pair(ctypes.c_uint64(seed), int(tid), stream, draw, _p(out))
    return float(out[0]), float(out[1])


def fnv1a(data: bytes) -> int:
    buf = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(1, dtype=np.uint8)
    return int(lib().o_fnv1a(_p(buf), len(data)))


def rotate(u, ct: float, cph: float, sph: float) -> np.ndarray:
    """The Compton direction rotation: u turned to polar cosine ct and azimuth (cph, sph) about itself."""
    out = np.zeros(3)
    lib().o_rotate(_p(_f64(u)), float(ct), float(cph), float(sph), _p(out))
    return out


def kahn_sample(E: float, seed: int, n: int, tid0: int = 0):
    eta = np.zeros(n)
    cost = np.zeros(n)
    if lib().o_kahn_sample(float(E), ctypes.c_uint64(seed), int(tid0), int(n), _p(eta), _p(cost)) != 0:
        raise RuntimeError("kahn: trial cap")
    return eta, cost


def source_sample(source, seed: int, n: int, tid0: int = 0):
    src = _f64(source.as_array())
    pos = np.zeros((n, 3))
    dirs = np.zeros((n, 3))
    E = np.zeros(n)
    lib().o_source_sample(_p(src), ctypes.c_uint64(seed), int(tid0), int(n), _p(pos), _p(dirs), _p(E))
    return pos, dirs, E
