"""Independent geometric references used to pin the oracle's solids and navigator.

Formulated differently from the oracle on purpose: plain strict-inside
predicates (atan2 for the phi range, explicit rotation matrices for the
placements), interval arithmetic for closed-form ray/solid intersections, and
a march plus bisection along rays for everything else.
"""
import math

import numpy as np

BOX, TUBE, ORB, CONE = 0, 1, 2, 3


def inside_strict(kind, par, p):
    """Vectorised strict point-in-solid test in the solid's local frame; p: (..., 3)."""
    p = np.asarray(p, dtype=np.float64)
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    if kind == BOX:
        return (np.abs(x) < par[0]) & (np.abs(y) < par[1]) & (np.abs(z) < par[2])
    if kind == ORB:
        return x * x + y * y + z * z < par[0] ** 2
    if kind == CONE:
        # radii interpolated linearly from the -hz end (rmin1, rmax1) to the +hz end (rmin2, rmax2)
        rmin1, rmax1, rmin2, rmax2, hz = par
        f = (z + hz) / (2.0 * hz)
        r = np.hypot(x, y)
        return (np.abs(z) < hz) & (r < rmax1 + (rmax2 - rmax1) * f) & (r > rmin1 + (rmin2 - rmin1) * f)
    rmin, rmax, hz, sphi, dphi = par
    r = np.hypot(x, y)
    ok = (r < rmax) & (r > rmin) & (np.abs(z) < hz)
    if dphi < 2 * math.pi - 1e-12:
        ang = np.mod(np.arctan2(y, x) - sphi, 2 * math.pi)
        ok &= (ang > 0) & (ang < dphi)
    return ok


def slab_interval(p, v, lo, hi):
    """Parameter interval where lo < p + t v < hi along one axis (None if empty)."""
    if v == 0.0:
        return (-math.inf, math.inf) if lo < p < hi else None
    a, b = (lo - p) / v, (hi - p) / v
    return (min(a, b), max(a, b))


def cyl_interval(px, py, vx, vy, R):
    a = vx * vx + vy * vy
    c = px * px + py * py - R * R
    if a == 0.0:
        return (-math.inf, math.inf) if c < 0 else None
    b = px * vx + py * vy
    disc = b * b - a * c
    if disc <= 0:
        return None
    s = math.sqrt(disc)
    return ((-b - s) / a, (-b + s) / a)


def _isect(i1, i2):
    if i1 is None or i2 is None:
        return None
    lo, hi = max(i1[0], i2[0]), min(i1[1], i2[1])
    return (lo, hi) if lo < hi else None


def inside_intervals(kind, par, p, v):
    """Intervals of t along the ray p + t v that lie in the (full-phi) solid, by interval arithmetic."""
    if kind == BOX:
        iv = (-math.inf, math.inf)
        for k in range(3):
            iv = _isect(iv, slab_interval(p[k], v[k], -par[k], par[k]))
        return [iv] if iv else []
    if kind == ORB:
        b = float(np.dot(p, v))
        c = float(np.dot(p, p)) - par[0] ** 2
        disc = b * b - c
        if disc <= 0:
            return []
        s = math.sqrt(disc)
        return [(-b - s, -b + s)]
    rmin, rmax, hz, sphi, dphi = par
    assert dphi >= 2 * math.pi - 1e-12
    outer = _isect(cyl_interval(p[0], p[1], v[0], v[1], rmax), slab_interval(p[2], v[2], -hz, hz))
    if outer is None:
        return []
    if rmin == 0.0:
        return [outer]
    inner = cyl_interval(p[0], p[1], v[0], v[1], rmin)
    if inner is None:
        return [outer]
    out = []
    if outer[0] < inner[0]:
        out.append((outer[0], min(outer[1], inner[0])))
    if outer[1] > inner[1]:
        out.append((max(outer[0], inner[1]), outer[1]))
    return [iv for iv in out if iv[0] < iv[1]]


def first_entry_closed_form(kind, par, p, v):
    ivs = [iv for iv in inside_intervals(kind, par, p, v) if iv[1] > 0]
    ivs.sort()
    return (ivs[0][0], ivs[0][1] - max(ivs[0][0], 0.0)) if ivs else (math.inf, 0.0)


def first_exit_closed_form(kind, par, p, v):
    for lo, hi in inside_intervals(kind, par, p, v):
        if lo <= 0.0 <= hi:
            return hi
    return None


def march_entry(pred, p, v, tmax, dt):
    """First t in (0, tmax] at which pred flips False -> True, refined by bisection; (t, chord)."""
    ts = np.arange(dt, tmax + dt, dt)
    pts = p[None, :] + ts[:, None] * v[None, :]
    ins = pred(pts)
    idx = np.nonzero(ins)[0]
    if idx.size == 0:
        return math.inf, 0.0
    k = idx[0]
    lo, hi = (ts[k - 1] if k > 0 else 0.0), ts[k]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if pred(p + mid * v):
            hi = mid
        else:
            lo = mid
    t_in = hi
    outs = np.nonzero(~ins[k:])[0]
    chord = (ts[k + outs[0]] - t_in) if outs.size else (tmax - t_in)
    return t_in, chord


def march_exit(pred, p, v, tmax, dt):
    """First t at which pred flips True -> False, starting inside."""
    ts = np.arange(dt, tmax + dt, dt)
    pts = p[None, :] + ts[:, None] * v[None, :]
    ins = pred(pts)
    idx = np.nonzero(~ins)[0]
    k = idx[0]
    lo, hi = (ts[k - 1] if k > 0 else 0.0), ts[k]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if pred(p + mid * v):
            lo = mid
        else:
            hi = mid
    return lo


def rot_matrix(c, s):
    """Rotation about z taking local to mother coordinates."""
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def random_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]
