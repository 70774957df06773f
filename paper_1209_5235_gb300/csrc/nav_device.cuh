// nav_device.cuh -- device-side navigation (sm_103a): solids, locate, the voxel
// walk of compute_step, relocation, attenuation tables, Philox and the step hash.
//
// Navigation problems (Sec. 3.2): (1) which volumes contain a point; (2) the
// distance to the next boundary along a direction.  Conventions shared with the
// host side of the library:
//  * tolerance band +-half around every surface (half = 0.5e-9 mm x scale);
//  * Inside is direction aware: a point in the band of a surface belongs to the
//    solid iff the direction points strictly inward through every surface
//    whose band holds the point;
//  * DistanceToIn from a point that is not inside only reports crossings
//    beyond the band; ties in compute_step go to the daughter over the mother
//    and to the lower daughter id;
//  * every distance here is FP64; the FP32 variants live in nav_fp32.cuh.
#pragma once

#include <cstdint>

#include "g4n_internal.h"

namespace g4n {
namespace dev {

constexpr double kInf = __builtin_huge_val();

struct V3 {
  double x, y, z;
};

__device__ __forceinline__ double comp(const V3 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Per-thread event counters (registers), flushed once per warp at the end.
struct Counters {
  uint32_t c[G4N_N_COUNTERS];
};

// ---------------------------------------------------------------- frames

__device__ __forceinline__ void to_local(const DVol &v, const V3 &pm, const V3 &vm, V3 &pl, V3 &vl) {
  const double dx = pm.x - v.tx, dy = pm.y - v.ty;
  pl.x = v.c * dx + v.s * dy;
  pl.y = v.c * dy - v.s * dx;
  pl.z = pm.z - v.tz;
  vl.x = v.c * vm.x + v.s * vm.y;
  vl.y = v.c * vm.y - v.s * vm.x;
  vl.z = vm.z;
}

__device__ __forceinline__ void world_to_local(const DWorld &w, const V3 &p, const V3 &u, V3 &pl, V3 &vl) {
  const double dx = p.x - w.tx, dy = p.y - w.ty;
  pl.x = w.c * dx + w.s * dy;
  pl.y = w.c * dy - w.s * dx;
  pl.z = p.z - w.tz;
  vl.x = w.c * u.x + w.s * u.y;
  vl.y = w.c * u.y - w.s * u.x;
  vl.z = u.z;
}

// ---------------------------------------------------------------- box

__device__ __forceinline__ bool box_inside(const double *h, const V3 &p, const V3 &v, double half) {
  const double ax = fabs(p.x) - h[0], ay = fabs(p.y) - h[1], az = fabs(p.z) - h[2];
  const double m = fmax(ax, fmax(ay, az));
  if (m > half) return false;
  if (m < -half) return true;
  if (ax >= -half && p.x * v.x >= 0.0) return false;
  if (ay >= -half && p.y * v.y >= 0.0) return false;
  if (az >= -half && p.z * v.z >= 0.0) return false;
  return true;
}

__device__ __forceinline__ double box_dist_in(const double *h, const V3 &p, const V3 &v, double half) {
  if ((fabs(p.x) - h[0] >= -half && p.x * v.x >= 0.0) || (fabs(p.y) - h[1] >= -half && p.y * v.y >= 0.0) ||
      (fabs(p.z) - h[2] >= -half && p.z * v.z >= 0.0))
    return kInf;
  double tin = -kInf, tout = kInf;
  const double pp[3] = {p.x, p.y, p.z}, vv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (vv[i] != 0.0) {
      const double a = (-h[i] - pp[i]) / vv[i], b = (h[i] - pp[i]) / vv[i];
      tin = fmax(tin, fmin(a, b));
      tout = fmin(tout, fmax(a, b));
    }
  }
  if (!(tout > tin + half)) return kInf;
  return fmax(tin, 0.0);
}

__device__ __forceinline__ double box_dist_out(const double *h, const V3 &p, const V3 &v) {
  double t = kInf;
  if (v.x != 0.0) t = fmin(t, (copysign(h[0], v.x) - p.x) / v.x);
  if (v.y != 0.0) t = fmin(t, (copysign(h[1], v.y) - p.y) / v.y);
  if (v.z != 0.0) t = fmin(t, (copysign(h[2], v.z) - p.z) / v.z);
  return fmax(t, 0.0);
}

__device__ __forceinline__ double box_safety_in(const double *h, const V3 &p) {
  return fmax(fmax(fabs(p.x) - h[0], fmax(fabs(p.y) - h[1], fabs(p.z) - h[2])), 0.0);
}

__device__ __forceinline__ double box_safety_out(const double *h, const V3 &p) {
  return fmax(fmin(h[0] - fabs(p.x), fmin(h[1] - fabs(p.y), h[2] - fabs(p.z))), 0.0);
}

// ---------------------------------------------------------------- orb

// Roots of a t^2 + 2 b t + c = 0 without cancellation; false if the discriminant is not positive.
__device__ __forceinline__ bool quad_roots(double a, double b, double c, double &lo, double &hi) {
  const double disc = b * b - a * c;
  if (!(disc > 0.0)) return false;
  const double sq = sqrt(disc);
  const double q = -(b + copysign(sq, b));
  const double r1 = q / a, r2 = c / q;
  lo = fmin(r1, r2);
  hi = fmax(r1, r2);
  return true;
}

__device__ __forceinline__ bool orb_inside(double R, const V3 &p, const V3 &v, double half) {
  const double r2 = p.x * p.x + p.y * p.y + p.z * p.z;
  const double ro = R + half, ri = R - half;
  if (r2 > ro * ro) return false;
  if (r2 < ri * ri) return true;
  return p.x * v.x + p.y * v.y + p.z * v.z < 0.0;
}

__device__ __forceinline__ double orb_dist_in(double R, const V3 &p, const V3 &v, double half) {
  const double b = p.x * v.x + p.y * v.y + p.z * v.z;
  const double c = p.x * p.x + p.y * p.y + p.z * p.z - R * R;
  double lo, hi;
  if (!quad_roots(1.0, b, c, lo, hi)) return kInf;
  return lo > half ? lo : kInf;
}

__device__ __forceinline__ double orb_dist_out(double R, const V3 &p, const V3 &v) {
  const double b = p.x * v.x + p.y * v.y + p.z * v.z;
  const double c = p.x * p.x + p.y * p.y + p.z * p.z - R * R;
  double lo, hi;
  if (!quad_roots(1.0, b, c, lo, hi)) return 0.0;
  return fmax(hi, 0.0);
}

__device__ __forceinline__ double orb_safety_in(double R, const V3 &p) {
  return fmax(sqrt(p.x * p.x + p.y * p.y + p.z * p.z) - R, 0.0);
}

__device__ __forceinline__ double orb_safety_out(double R, const V3 &p) {
  return fmax(R - sqrt(p.x * p.x + p.y * p.y + p.z * p.z), 0.0);
}

// ---------------------------------------------------------------- tube segment
// q[0..6] = rmin, rmax, hz, cos(sphi), sin(sphi), cos(ephi), sin(ephi).
// ps = cross(u_start, p) and pe = cross(p, u_end) are the signed distances to the
// lines of the two phi half-planes, positive on the solid's side.

__device__ __forceinline__ bool tube_phi_ok(const double *q, int flags, double x, double y, double tol) {
  if (!(flags & kSeg)) return true;
  const double ps = q[3] * y - q[4] * x, pe = q[6] * x - q[5] * y;
  return (flags & kWide) ? (ps >= -tol || pe >= -tol) : (ps >= -tol && pe >= -tol);
}

__device__ __forceinline__ bool tube_r_ok(const double *q, int flags, double x, double y, double half) {
  const double r2 = x * x + y * y, ro = q[1] + half;
  if (r2 > ro * ro) return false;
  if (flags & kHasRmin) {
    const double ri = q[0] - half;
    if (r2 < ri * ri) return false;
  }
  return true;
}

__device__ __noinline__ bool tube_inside(const double *q, int flags, const V3 &p, const V3 &v, double half) {
  const double sz = fabs(p.z) - q[2];
  if (sz > half) return false;
  const double r2 = p.x * p.x + p.y * p.y;
  const double ro = q[1] + half;
  if (r2 > ro * ro) return false;
  bool nz = sz >= -half;
  const double rmi = q[1] - half;
  bool nrmax = r2 >= rmi * rmi;
  bool nrmin = false;
  if (flags & kHasRmin) {
    const double ri = q[0] - half, rio = q[0] + half;
    if (r2 < ri * ri) return false;
    nrmin = r2 <= rio * rio;
  }
  bool ns = false, ne = false;
  if (flags & kSeg) {
    const double ps = q[3] * p.y - q[4] * p.x, pe = q[6] * p.x - q[5] * p.y;
    if (!(flags & kWide)) {
      if (ps < -half || pe < -half) return false;
      ns = ps <= half;
      ne = pe <= half;
    } else {
      const double m = fmax(ps, pe);
      if (m < -half) return false;
      if (m <= half) {
        if (ps >= pe) ns = true;
        else ne = true;
      }
    }
  }
  if (!(nz || nrmax || nrmin || ns || ne)) return true;
  const double vr = p.x * v.x + p.y * v.y;
  if (nz && !(p.z * v.z < 0.0)) return false;
  if (nrmax && !(vr < 0.0)) return false;
  if (nrmin && !(vr > 0.0)) return false;
  if (ns && !(q[4] * v.x - q[3] * v.y < 0.0)) return false;
  if (ne && !(q[5] * v.y - q[6] * v.x < 0.0)) return false;
  return true;
}

// enter = true: first entering crossing with t > half (DistanceToIn);
// enter = false: first exiting crossing with t > -half (DistanceToOut, clamped by the caller).
__device__ __noinline__ double tube_cross(const double *q, int flags, const V3 &p, const V3 &v, double half, bool enter) {
  const double tmin = enter ? half : -half;
  double best = kInf;
  if (v.z != 0.0) {
    // the z plane this ray can enter (enter) or leave (exit) through
    const double sg = ((v.z < 0.0) == enter) ? 1.0 : -1.0;
    const double t = (sg * q[2] - p.z) / v.z;
    if (t > tmin) {
      const double qx = p.x + t * v.x, qy = p.y + t * v.y;
      if (tube_r_ok(q, flags, qx, qy, half) && tube_phi_ok(q, flags, qx, qy, half)) best = t;
    }
  }
  const double a = v.x * v.x + v.y * v.y;
  if (a > 0.0) {
    const double b = p.x * v.x + p.y * v.y;
    const double r2 = p.x * p.x + p.y * p.y;
    double lo, hi;
    if (quad_roots(a, b, r2 - q[1] * q[1], lo, hi)) {
      const double t = enter ? lo : hi;
      if (t > tmin && t < best && fabs(p.z + t * v.z) <= q[2] + half &&
          tube_phi_ok(q, flags, p.x + t * v.x, p.y + t * v.y, half))
        best = t;
    }
    if ((flags & kHasRmin) && quad_roots(a, b, r2 - q[0] * q[0], lo, hi)) {
      const double t = enter ? hi : lo;
      if (t > tmin && t < best && fabs(p.z + t * v.z) <= q[2] + half &&
          tube_phi_ok(q, flags, p.x + t * v.x, p.y + t * v.y, half))
        best = t;
    }
  }
  if (flags & kSeg) {
    const double dn = q[4] * v.x - q[3] * v.y;  // v . outward normal of the start plane
    if (dn != 0.0 && ((dn < 0.0) == enter)) {
      const double t = (q[3] * p.y - q[4] * p.x) / dn;
      if (t > tmin && t < best) {
        const double qx = p.x + t * v.x, qy = p.y + t * v.y;
        if (q[3] * qx + q[4] * qy >= -half && tube_r_ok(q, flags, qx, qy, half) && fabs(p.z + t * v.z) <= q[2] + half)
          best = t;
      }
    }
    const double de = q[5] * v.y - q[6] * v.x;  // end plane
    if (de != 0.0 && ((de < 0.0) == enter)) {
      const double t = (q[6] * p.x - q[5] * p.y) / de;
      if (t > tmin && t < best) {
        const double qx = p.x + t * v.x, qy = p.y + t * v.y;
        if (q[5] * qx + q[6] * qy >= -half && tube_r_ok(q, flags, qx, qy, half) && fabs(p.z + t * v.z) <= q[2] + half)
          best = t;
      }
    }
  }
  return best;
}

__device__ __forceinline__ double tube_safety_in(const double *q, int flags, const V3 &p) {
  const double r = sqrt(p.x * p.x + p.y * p.y);
  double m = fmax(r - q[1], fabs(p.z) - q[2]);
  if (flags & kHasRmin) m = fmax(m, q[0] - r);
  if (flags & kSeg) {
    const double a = q[4] * p.x - q[3] * p.y, b = q[5] * p.y - q[6] * p.x;
    m = fmax(m, (flags & kWide) ? fmin(a, b) : fmax(a, b));
  }
  return fmax(m, 0.0);
}

__device__ __forceinline__ double tube_safety_out(const double *q, int flags, const V3 &p) {
  const double r = sqrt(p.x * p.x + p.y * p.y);
  double m = fmin(q[1] - r, q[2] - fabs(p.z));
  if (flags & kHasRmin) m = fmin(m, r - q[0]);
  if (flags & kSeg) m = fmin(m, fmin(fabs(q[3] * p.y - q[4] * p.x), fabs(q[6] * p.x - q[5] * p.y)));
  return fmax(m, 0.0);
}

// ---------------------------------------------------------------- dispatch on the solid kind

__device__ __forceinline__ bool vol_inside(const DVol &d, const V3 &p, const V3 &v, double half) {
  if (d.kind == kBox) return box_inside(d.p, p, v, half);
  if (d.kind == kOrb) return orb_inside(d.p[0], p, v, half);
  return tube_inside(d.p, d.flags, p, v, half);
}

__device__ __forceinline__ double vol_dist_in(const DVol &d, const V3 &p, const V3 &v, double half) {
  if (d.kind == kBox) return box_dist_in(d.p, p, v, half);
  if (d.kind == kOrb) return orb_dist_in(d.p[0], p, v, half);
  return tube_cross(d.p, d.flags, p, v, half, true);
}

__device__ __forceinline__ double vol_dist_out(const DVol &d, const V3 &p, const V3 &v, double half) {
  if (d.kind == kBox) return box_dist_out(d.p, p, v);
  if (d.kind == kOrb) return orb_dist_out(d.p[0], p, v);
  const double t = tube_cross(d.p, d.flags, p, v, half, false);
  return t == kInf ? 0.0 : fmax(t, 0.0);
}

__device__ __forceinline__ double vol_safety_in(const DVol &d, const V3 &p) {
  if (d.kind == kBox) return box_safety_in(d.p, p);
  if (d.kind == kOrb) return orb_safety_in(d.p[0], p);
  return tube_safety_in(d.p, d.flags, p);
}

__device__ __forceinline__ double vol_safety_out(const DVol &d, const V3 &p) {
  if (d.kind == kBox) return box_safety_out(d.p, p);
  if (d.kind == kOrb) return orb_safety_out(d.p[0], p);
  return tube_safety_out(d.p, d.flags, p);
}

// Conservative FP32 test: can the mother-frame point claim daughter box b?
__device__ __forceinline__ bool box32_contains(const DBox32 &b, const V3 &p) {
  const float x = (float)p.x, y = (float)p.y, z = (float)p.z;
  return x >= b.lo[0] && x <= b.hi[0] && y >= b.lo[1] && y <= b.hi[1] && z >= b.lo[2] && z <= b.hi[2];
}

// ---------------------------------------------------------------- voxels

__device__ __forceinline__ int slice_of(const DVoxHdr &H, double coord) {
  double f = floor((coord - H.lo) * H.inv_width);
  f = fmin(fmax(f, 0.0), (double)(H.nslices - 1));
  return (int)f;
}

// Candidate list of the voxel node holding p (mother frame).
__device__ __forceinline__ int vox_lookup(const DGeom &G, int h, const V3 &p) {
#pragma unroll 1
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    const DVoxHdr H = G.hdr[h];
    const DVoxSlice S = G.slice[H.slice_base + slice_of(H, comp(p, H.axis))];
    if (S.child >= 0) return S.child;
    h = -S.child - 1;
  }
  return 0;
}

// Descend from volume m (p, v in m's frame) into the first daughter, in id order,
// that contains the point; repeat.  Returns the deepest volume.
__device__ __noinline__ int descend(const DGeom &G, int m, V3 p, V3 v, Counters &cnt) {
#pragma unroll 1
  for (int lev = 0; lev < kDMax; ++lev) {
    const int h = G.vol[m].vox;
    if (h < 0) return m;
    const DCandList L = G.clist[vox_lookup(G, h, p)];
    int found = -1;
    V3 fp, fv;
#pragma unroll 1
    for (int i = 0; i < L.count; ++i) {
      const int d = G.cand[L.offset + i];
      if (!box32_contains(G.box[d], p)) continue;
      const DVol &D = G.vol[d];
      V3 dp, dv;
      to_local(D, p, v, dp, dv);
      cnt.c[G4N_C_INSIDE]++;
      if (vol_inside(D, dp, dv, G.half)) {
        found = d;
        fp = dp;
        fv = dv;
        break;
      }
    }
    if (found < 0) return m;
    m = found;
    p = fp;
    v = fv;
  }
  return m;
}

// Locate from the world: returns the leaf, or -1 outside the world.
__device__ __forceinline__ int locate_world(const DGeom &G, const V3 &x, const V3 &u, Counters &cnt) {
  V3 p, v;
  world_to_local(G.wxf[0], x, u, p, v);
  cnt.c[G4N_C_INSIDE]++;
  if (!vol_inside(G.vol[0], p, v, G.half)) return -1;
  return descend(G, 0, p, v, cnt);
}

// After a move: leave every volume that no longer contains the point, then descend.
__device__ __noinline__ int relocate(const DGeom &G, int leaf, const V3 &x, const V3 &u, Counters &cnt) {
#pragma unroll 1
  while (leaf >= 0) {
    V3 p, v;
    world_to_local(G.wxf[leaf], x, u, p, v);
    const DVol &L = G.vol[leaf];
    cnt.c[G4N_C_INSIDE]++;
    if (vol_inside(L, p, v, G.half)) return descend(G, leaf, p, v, cnt);
    leaf = L.mother;
  }
  return -1;
}

// Voxel walk state: per level the header, the merged node's slice range.
struct Chain {
  int h[kMaxLevels];
  int k0[kMaxLevels], k1[kMaxLevels];
  int nlev;
  int list;
};

__device__ __forceinline__ void chain_fill(const DGeom &G, Chain &ch, int lev, int h, const V3 &p) {
#pragma unroll 1
  for (; lev < kMaxLevels; ++lev) {
    const DVoxHdr H = G.hdr[h];
    const DVoxSlice S = G.slice[H.slice_base + slice_of(H, comp(p, H.axis))];
    ch.h[lev] = h;
    ch.k0[lev] = S.k0;
    ch.k1[lev] = S.k1;
    if (S.child >= 0) {
      ch.nlev = lev + 1;
      ch.list = S.child;
      return;
    }
    h = -S.child - 1;
  }
  ch.nlev = kMaxLevels;
  ch.list = 0;
}

// Geometric step inside `leaf` from local point p along v (Sec. 3.2, problem 2):
// DistanceToOut of the leaf, then DistanceToIn of the daughters listed in the
// voxel nodes the ray crosses, stopping once the node exit lies beyond the best
// distance or `limit`.  Returns the step, *lim = daughter id or -1 (mother).
// If want_safety, *safety = isotropic lower bound (mother, the first node's
// candidates and that node's slab boundaries).  Sets *timeout on a runaway walk.
__device__ __noinline__ double geom_step(const DGeom &G, int leaf, const V3 &p, const V3 &v, double limit, int *lim,
                                         double *safety, bool want_safety, Counters &cnt, bool *timeout) {
  const DVol &V = G.vol[leaf];
  const double half = G.half;
  cnt.c[G4N_C_DIST_OUT]++;
  double best = vol_dist_out(V, p, v, half);
  int bl = G4N_LIM_MOTHER;
  double saf = want_safety ? vol_safety_out(V, p) : 0.0;
  if (V.vox >= 0) {
    Chain ch;
    chain_fill(G, ch, 0, V.vox, p);
    bool first = true;
#pragma unroll 1
    for (int it = 0; it < 1 << 16; ++it) {
      cnt.c[G4N_C_VOX_NODES]++;
      const DCandList L = G.clist[ch.list];
#pragma unroll 1
      for (int i = 0; i < L.count; ++i) {
        const int d = G.cand[L.offset + i];
        const DVol &D = G.vol[d];
        V3 dp, dv;
        to_local(D, p, v, dp, dv);
        cnt.c[G4N_C_CAND_BOX + D.kind]++;
        const double t = vol_dist_in(D, dp, dv, half);
        if (t < kInf && (t < best || (t == best && (bl < 0 || d < bl)))) {
          best = t;
          bl = d;
        }
        if (first && want_safety) saf = fmin(saf, vol_safety_in(D, dp));
      }
      // exit of the current node along the ray; node slab boundaries bound the safety
      double texit = kInf;
      int lstar = -1;
#pragma unroll 1
      for (int l = 0; l < ch.nlev; ++l) {
        const DVoxHdr H = G.hdr[ch.h[l]];
        const double pa = comp(p, H.axis), va = comp(v, H.axis);
        const double blo = H.lo + ch.k0[l] * H.width, bhi = H.lo + (ch.k1[l] + 1) * H.width;
        if (first && want_safety) saf = fmin(saf, fmax(fmin(pa - blo, bhi - pa), 0.0));
        double t = kInf;
        if (va > 0.0) t = (bhi - pa) / va;
        else if (va < 0.0) t = (blo - pa) / va;
        if (t < texit) {
          texit = t;
          lstar = l;
        }
      }
      first = false;
      if (!(texit < fmin(best, limit))) break;
      // step into the neighbouring node at level lstar; deeper levels are looked up again
      const DVoxHdr H = G.hdr[ch.h[lstar]];
      const int nk = comp(v, H.axis) > 0.0 ? ch.k1[lstar] + 1 : ch.k0[lstar] - 1;
      if (nk < 0 || nk >= H.nslices) break;
      const DVoxSlice S = G.slice[H.slice_base + nk];
      ch.k0[lstar] = S.k0;
      ch.k1[lstar] = S.k1;
      if (S.child >= 0) {
        ch.nlev = lstar + 1;
        ch.list = S.child;
      } else {
        const V3 qpt{p.x + texit * v.x, p.y + texit * v.y, p.z + texit * v.z};
        chain_fill(G, ch, lstar + 1, -S.child - 1, qpt);
      }
      if (it == (1 << 16) - 1) *timeout = true;
    }
  }
  *lim = bl;
  if (want_safety) *safety = saf;
  return best;
}

// ---------------------------------------------------------------- attenuation table

// Binary search for E_k <= E < E_{k+1}, lin-lin interpolation, clamped at the ends.
__device__ __forceinline__ void mu_lookup(const DGeom &G, int mat, double E, double &mu_tot, double &mu_pe) {
  const int off = G.mat_off[mat], n = G.mat_n[mat];
  const double *Eg = G.matE + off, *C = G.matC + off, *P = G.matP + off;
  double mc, mp;
  if (E <= Eg[0]) {
    mc = C[0];
    mp = P[0];
  } else if (E >= Eg[n - 1]) {
    mc = C[n - 1];
    mp = P[n - 1];
  } else {
    int lo = 0, hi = n - 1;
#pragma unroll 1
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (Eg[mid] <= E) lo = mid;
      else hi = mid;
    }
    const double f = (E - Eg[lo]) / (Eg[lo + 1] - Eg[lo]);
    mc = C[lo] + f * (C[lo + 1] - C[lo]);
    mp = P[lo] + f * (P[lo + 1] - P[lo]);
  }
  mu_tot = mc + mp;
  mu_pe = mp;
}

// ---------------------------------------------------------------- Philox4x32-10 and FNV-1a

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform in (0, 1] from one Philox block: counter (draw, id lo, id hi, stream).
__device__ __forceinline__ double philox_uniform(uint64_t seed, int64_t tid, uint32_t stream, uint32_t &draw) {
  const uint4 x = philox4x32_10(make_uint4(draw++, (uint32_t)(uint64_t)tid, (uint32_t)((uint64_t)tid >> 32), stream),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint64_t w = ((uint64_t)x.y << 32) | x.x;
  return (double)((w >> 11) + 1) * 0x1.0p-53;
}

__device__ __forceinline__ uint64_t fnv_word(uint64_t h, uint32_t w) {
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    h ^= (w >> (8 * b)) & 0xffu;
    h *= 0x100000001b3ull;
  }
  return h;
}

__device__ __forceinline__ uint64_t hash_step(uint64_t h, int32_t leaf, int32_t limiter, int32_t event) {
  h = fnv_word(h, (uint32_t)leaf);
  h = fnv_word(h, (uint32_t)limiter);
  return fnv_word(h, (uint32_t)event);
}

}  // namespace dev
}  // namespace g4n
