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
//    and to the lower daughter id.
//
// Precision modes.  kFP64: every distance in FP64.  kFP32: rigorous FP32
// interval bounds (directed rounding) on the padded bounding boxes decide which
// candidates can still matter and whether the physics step wins; only those
// candidates and the winning surface are evaluated in FP64, so every result is
// the FP64 one.  GB300's FP64 rate is ~1/72 of its FP32 rate, which is why the
// bounds are worth their extra FP32 work.
#pragma once

#include <cstdint>

#include "g4n_internal.h"
#include "mlp_device.cuh"

namespace g4n {
namespace dev {

constexpr double kInf = __builtin_huge_val();
constexpr float kInfF = __builtin_huge_valf();
enum Mode : int { kFP64 = 0, kFP32 = 1, kLearned = 2 };  // kLearned: FP32 bounds + proposal first

struct V3 {
  double x, y, z;
};

__device__ __forceinline__ double comp(const V3 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Per-thread event counters (registers; constant indices only), flushed once per warp.
struct Counters {
  uint32_t c[G4N_N_COUNTERS];
};

template <bool COUNT>
__device__ __forceinline__ void diag(Counters &c, int k) {
  if (COUNT) c.c[k]++;
}

template <bool COUNT>
__device__ __forceinline__ void diag_kind(Counters &c, int kind) {
  if (COUNT) {
    if (kind == kBox) c.c[G4N_C_CAND_BOX]++;
    else if (kind == kTube) c.c[G4N_C_CAND_TUBE]++;
    else if (kind == kCone) c.c[G4N_C_CAND_CONE]++;
    else c.c[G4N_C_CAND_ORB]++;
  }
}

// An FP64 DistanceToOut or Inside test of solid `kind`: tubes and cones are also counted apart (their
// formulas have several times the box's arithmetic).
template <bool COUNT>
__device__ __forceinline__ void diag_test(Counters &c, int which, int curved_which, int kind) {
  if (COUNT) {
    c.c[which]++;
    if (kind == kTube || kind == kCone) c.c[curved_which]++;
  }
}

// key(x): a double's bits as a signed integer with the negative half reflected, so that
// x < y <=> key(x) < key(y) for all non-NaN doubles (-0 < +0).
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}

// ---------------------------------------------------------------- frames

__device__ __forceinline__ void to_local(const DVol &v, const V3 &pm, const V3 &vm, V3 &pl, V3 &vl) {
  const double dx = pm.x - v.tx, dy = pm.y - v.ty;
  if (v.flags & kPlacedAligned) {
    pl = V3{dx, dy, pm.z - v.tz};
    vl = vm;
    return;
  }
  pl.x = v.c * dx + v.s * dy;
  pl.y = v.c * dy - v.s * dx;
  pl.z = pm.z - v.tz;
  vl.x = v.c * vm.x + v.s * vm.y;
  vl.y = v.c * vm.y - v.s * vm.x;
  vl.z = vm.z;
}

// World -> local frame of a volume; world-aligned volumes need only the translation.
__device__ __forceinline__ void world_to_local(const DWorld &w, bool aligned, const V3 &p, const V3 &u, V3 &pl,
                                               V3 &vl) {
  const double dx = p.x - w.tx, dy = p.y - w.ty;
  if (aligned) {
    pl = V3{dx, dy, p.z - w.tz};
    vl = u;
    return;
  }
  pl.x = w.c * dx + w.s * dy;
  pl.y = w.c * dy - w.s * dx;
  pl.z = p.z - w.tz;
  vl.x = w.c * u.x + w.s * u.y;
  vl.y = w.c * u.y - w.s * u.x;
  vl.z = u.z;
}

// Reciprocal direction components (0 where the component is 0: never used there).
struct Inv3 {
  double x, y, z;
};

__device__ __forceinline__ Inv3 inv_dir(const V3 &v) {
  return Inv3{v.x != 0.0 ? 1.0 / v.x : 0.0, v.y != 0.0 ? 1.0 / v.y : 0.0, v.z != 0.0 ? 1.0 / v.z : 0.0};
}

__device__ __forceinline__ double icomp(const Inv3 &v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

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

// DistanceToOut with the reciprocal direction of the same frame; *face = the exit face
// (2 axis + (v_axis > 0)) of the first axis attaining the minimum.  The zero tests of
// v, the minimum and the clamp at 0 are integer operations on the bit patterns (the
// order-preserving keys of doubles), which give the same value as fmin/fmax.
__device__ __forceinline__ bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }

__device__ __forceinline__ double box_dist_out(const double *h, const V3 &p, const V3 &v, const Inv3 &iv, int *face) {
  constexpr long long kKeyInf = 0x7FF0000000000000ll;  // key of +inf; NaN keys lie outside [key(-inf), key(+inf)]
  double t = kInf;
  long long kt = kKeyInf;
  int f = -1;
  const double pp[3] = {p.x, p.y, p.z}, vv[3] = {v.x, v.y, v.z}, ii[3] = {iv.x, iv.y, iv.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!nonzero_bits(vv[a])) continue;
    const double ta = (copysign(h[a], vv[a]) - pp[a]) * ii[a];
    const long long k = dkey(ta);
    if (k < kt && k >= -kKeyInf - 1) {
      kt = k;
      t = ta;
      f = 2 * a + (vv[a] > 0.0 ? 1 : 0);
    }
  }
  *face = f;
  return kt < 0 ? 0.0 : t;
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

// The crossings tube_cross takes the first of, one helper per surface: each returns its crossing
// parameter t when t lies in (tmin, best) and the crossing passes the surface's range tests, else
// +inf.
// z plane the ray enters (enter) or leaves (exit) through
__device__ __forceinline__ double tube_z_cand(const double *q, int flags, const V3 &p, const V3 &v, double half,
                                              bool enter, double tmin) {
  if (v.z == 0.0) return kInf;
  const double sg = ((v.z < 0.0) == enter) ? 1.0 : -1.0;
  const double t = (sg * q[2] - p.z) / v.z;
  if (!(t > tmin)) return kInf;
  const double qx = p.x + t * v.x, qy = p.y + t * v.y;
  return (tube_r_ok(q, flags, qx, qy, half) && tube_phi_ok(q, flags, qx, qy, half)) ? t : kInf;
}

// cylinder of radius R (outer: the root that enters / leaves the solid through rmax; inner: through rmin)
__device__ __forceinline__ double tube_cyl_cand(const double *q, int flags, const V3 &p, const V3 &v, double half,
                                                bool enter, double tmin, double best, bool outer) {
  const double a = v.x * v.x + v.y * v.y;
  if (!(a > 0.0)) return kInf;
  const double b = p.x * v.x + p.y * v.y;
  const double r2 = p.x * p.x + p.y * p.y;
  const double R = outer ? q[1] : q[0];
  double lo, hi;
  if (!quad_roots(a, b, r2 - R * R, lo, hi)) return kInf;
  const double t = (enter == outer) ? lo : hi;
  if (t > tmin && t < best && fabs(p.z + t * v.z) <= q[2] + half &&
      tube_phi_ok(q, flags, p.x + t * v.x, p.y + t * v.y, half))
    return t;
  return kInf;
}

// phi half-plane at the start (start = true) or end of the segment
__device__ __forceinline__ double tube_phi_cand(const double *q, int flags, const V3 &p, const V3 &v, double half,
                                                bool enter, double tmin, double best, bool start) {
  // v . outward normal of the plane, the signed distance to its line (positive on the solid's side)
  const double dn = start ? q[4] * v.x - q[3] * v.y : q[5] * v.y - q[6] * v.x;
  if (!(dn != 0.0 && ((dn < 0.0) == enter))) return kInf;
  const double t = (start ? q[3] * p.y - q[4] * p.x : q[6] * p.x - q[5] * p.y) / dn;
  if (!(t > tmin && t < best)) return kInf;
  const double qx = p.x + t * v.x, qy = p.y + t * v.y;
  const double along = start ? q[3] * qx + q[4] * qy : q[5] * qx + q[6] * qy;
  return (along >= -half && tube_r_ok(q, flags, qx, qy, half) && fabs(p.z + t * v.z) <= q[2] + half) ? t : kInf;
}

// enter = true: first entering crossing with t > half (DistanceToIn);
// enter = false: first exiting crossing with t > -half (DistanceToOut, clamped by the caller).
__device__ __noinline__ double tube_cross(const double *q, int flags, const V3 &p, const V3 &v, double half, bool enter) {
  const double tmin = enter ? half : -half;
  double best = tube_z_cand(q, flags, p, v, half, enter, tmin);
  best = fmin(best, tube_cyl_cand(q, flags, p, v, half, enter, tmin, best, true));
  if (flags & kHasRmin) best = fmin(best, tube_cyl_cand(q, flags, p, v, half, enter, tmin, best, false));
  if (flags & kSeg) {
    best = fmin(best, tube_phi_cand(q, flags, p, v, half, enter, tmin, best, true));
    best = fmin(best, tube_phi_cand(q, flags, p, v, half, enter, tmin, best, false));
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

// ---------------------------------------------------------------- cone (full in phi)
// q[0..6] = ki, ci, ko, co, hz, cos(inner half-angle), cos(outer half-angle): between
// z = -hz and +hz the solid is Rin(z) <= r <= Rout(z), Rout = ko z + co, Rin = ki z + ci
// (flag kHasRmin: inner surface present).  Bands along r at the point's z; outward normal of
// the outer surface along (x / r, y / r, -ko), of the inner one along (-x / r, -y / r, ki).

__device__ __noinline__ bool cone_inside(const double *q, int flags, const V3 &p, const V3 &v, double half) {
  const double sz = fabs(p.z) - q[4];
  if (sz > half) return false;
  const double r2 = p.x * p.x + p.y * p.y;
  const double ro = q[2] * p.z + q[3];
  const double rop = ro + half, rom = ro - half;
  if (r2 > rop * rop) return false;
  const bool nz = sz >= -half;
  const bool nrmax = r2 >= rom * rom;
  bool nrmin = false;
  if (flags & kHasRmin) {
    const double ri = q[0] * p.z + q[1];
    const double rim = ri - half, rip = ri + half;
    if (r2 < rim * rim) return false;
    nrmin = r2 <= rip * rip;
  }
  if (!(nz || nrmax || nrmin)) return true;
  const double r = sqrt(r2);
  const double vr = p.x * v.x + p.y * v.y;
  if (nz && !(p.z * v.z < 0.0)) return false;
  if (nrmax && !(vr - q[2] * r * v.z < 0.0)) return false;
  if (nrmin && !(vr - q[0] * r * v.z > 0.0)) return false;
  return true;
}

// enter = true: first entering crossing with t > half; enter = false: first exiting crossing
// with t > -half.  Conical surfaces: a t^2 + 2 b t + cc = 0 with d = a t + b half the rate of
// change of r^2 - R^2 along the ray (entering the solid: d < 0 at the outer surface, d > 0 at
// the inner one); roots on the other half of the double cone (R < 0) are not surface points.
__device__ __noinline__ double cone_cross(const double *q, int flags, const V3 &p, const V3 &v, double half, bool enter) {
  const double tmin = enter ? half : -half;
  const double hz = q[4];
  double best = kInf;
  if (v.z != 0.0) {
    const double sg = ((v.z < 0.0) == enter) ? 1.0 : -1.0;
    const double t = (sg * hz - p.z) / v.z;
    if (t > tmin) {
      const double qx = p.x + t * v.x, qy = p.y + t * v.y;
      const double r2 = qx * qx + qy * qy;
      const double ro = q[2] * (sg * hz) + q[3] + half;
      bool ok = r2 <= ro * ro;
      if (flags & kHasRmin) {
        const double ri = q[0] * (sg * hz) + q[1] - half;
        ok = ok && !(r2 < ri * ri);
      }
      if (ok) best = t;
    }
  }
  const int nw = (flags & kHasRmin) ? 2 : 1;
#pragma unroll 1
  for (int w = 0; w < nw; ++w) {
    const double k = w == 0 ? q[2] : q[0], c = w == 0 ? q[3] : q[1];
    const double rz = k * p.z + c;
    const double a = v.x * v.x + v.y * v.y - k * k * v.z * v.z;
    const double b = p.x * v.x + p.y * v.y - k * v.z * rz;
    const double cc = p.x * p.x + p.y * p.y - rz * rz;
    double t0 = kInf, t1 = kInf;
    if (a != 0.0) {
      const double disc = b * b - a * cc;
      if (disc > 0.0) {
        const double sq = sqrt(disc);
        const double qq = -(b + copysign(sq, b));
        t0 = qq / a;
        t1 = cc / qq;
      }
    } else if (b != 0.0) {
      t0 = -cc / (2.0 * b);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const double t = i == 0 ? t0 : t1;
      if (!(t > tmin && t < best)) continue;
      const double d = a * t + b;
      const bool into = w == 0 ? d < 0.0 : d > 0.0;
      if (into != enter) continue;
      const double qz = p.z + t * v.z;
      if (fabs(qz) > hz + half) continue;
      if (!(k * qz + c >= 0.0)) continue;
      best = t;
    }
  }
  return best;
}

__device__ __forceinline__ double cone_safety_in(const double *q, int flags, const V3 &p) {
  const double r = sqrt(p.x * p.x + p.y * p.y);
  double m = fmax(fabs(p.z) - q[4], (r - (q[2] * p.z + q[3])) * q[6]);
  if (flags & kHasRmin) m = fmax(m, ((q[0] * p.z + q[1]) - r) * q[5]);
  return fmax(m, 0.0);
}

__device__ __forceinline__ double cone_safety_out(const double *q, int flags, const V3 &p) {
  const double r = sqrt(p.x * p.x + p.y * p.y);
  double m = fmin(q[4] - fabs(p.z), ((q[2] * p.z + q[3]) - r) * q[6]);
  if (flags & kHasRmin) m = fmin(m, (r - (q[0] * p.z + q[1])) * q[5]);
  return fmax(m, 0.0);
}

// ---------------------------------------------------------------- dispatch on the solid kind

__device__ __forceinline__ bool vol_inside(const DVol &d, const V3 &p, const V3 &v, double half) {
  if (d.kind == kBox) return box_inside(d.p, p, v, half);
  if (d.kind == kOrb) return orb_inside(d.p[0], p, v, half);
  if (d.kind == kCone) return cone_inside(d.p, d.flags, p, v, half);
  return tube_inside(d.p, d.flags, p, v, half);
}

__device__ __forceinline__ double vol_dist_in(const DVol &d, const V3 &p, const V3 &v, double half) {
  if (d.kind == kBox) return box_dist_in(d.p, p, v, half);
  if (d.kind == kOrb) return orb_dist_in(d.p[0], p, v, half);
  if (d.kind == kCone) return cone_cross(d.p, d.flags, p, v, half, true);
  return tube_cross(d.p, d.flags, p, v, half, true);
}

__device__ __forceinline__ double vol_dist_out(const DVol &d, const V3 &p, const V3 &v, const Inv3 &iv, double half,
                                               int *face) {
  *face = -1;
  if (d.kind == kBox) return box_dist_out(d.p, p, v, iv, face);
  if (d.kind == kOrb) return orb_dist_out(d.p[0], p, v);
  const double t = d.kind == kCone ? cone_cross(d.p, d.flags, p, v, half, false) : tube_cross(d.p, d.flags, p, v, half, false);
  return t == kInf ? 0.0 : fmax(t, 0.0);
}

__device__ __forceinline__ double vol_safety_in(const DVol &d, const V3 &p) {
  if (d.kind == kBox) return box_safety_in(d.p, p);
  if (d.kind == kOrb) return orb_safety_in(d.p[0], p);
  if (d.kind == kCone) return cone_safety_in(d.p, d.flags, p);
  return tube_safety_in(d.p, d.flags, p);
}

__device__ __forceinline__ double vol_safety_out(const DVol &d, const V3 &p) {
  if (d.kind == kBox) return box_safety_out(d.p, p);
  if (d.kind == kOrb) return orb_safety_out(d.p[0], p);
  if (d.kind == kCone) return cone_safety_out(d.p, d.flags, p);
  return tube_safety_out(d.p, d.flags, p);
}

// ---------------------------------------------------------------- FP32 interval bounds
// A point p (FP64) is enclosed by [lo, hi] = the float neighbours of (float)p; a
// direction component by its float neighbours, whose reciprocals, rounded
// outward, enclose 1/v.  All products and differences below are rounded in the
// direction that keeps each bound valid, so every lower bound is <= the exact
// FP64 quantity it bounds (and every upper bound >=).

struct Ray32 {
  float plo[3], phi[3];
  float ilo[3], ihi[3];  // enclosure of 1/|v_a|
  int sgn[3];            // sign of v_a (0 if |v_a| < 1e-30)
};

__device__ __forceinline__ void enclose(double x, float &lo, float &hi) {
  const float f = (float)x;
  lo = nextafterf(f, -kInfF);
  hi = nextafterf(f, kInfF);
}

__device__ __forceinline__ Ray32 make_ray32(const V3 &p, const V3 &v) {
  Ray32 r;
  const double pp[3] = {p.x, p.y, p.z}, vv[3] = {v.x, v.y, v.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    enclose(pp[a], r.plo[a], r.phi[a]);
    const double w = fabs(vv[a]);
    if (w < 1e-30) {
      r.sgn[a] = 0;
      r.ilo[a] = r.ihi[a] = 0.f;
      continue;
    }
    r.sgn[a] = vv[a] > 0.0 ? 1 : -1;
    float wlo, whi;
    enclose(w, wlo, whi);
    r.ilo[a] = __frcp_rd(whi);
    r.ihi[a] = wlo > 0.f ? __frcp_ru(wlo) : kInfF;
  }
  return r;
}

// Lower/upper bound of num / |v_a| given num in [nlo, nhi] (scalar num bounds).
__device__ __forceinline__ float div_lo(float n, const Ray32 &r, int a) {
  return n >= 0.f ? __fmul_rd(n, r.ilo[a]) : __fmul_rd(n, r.ihi[a]);
}
__device__ __forceinline__ float div_hi(float n, const Ray32 &r, int a) {
  return n >= 0.f ? __fmul_ru(n, r.ihi[a]) : __fmul_ru(n, r.ilo[a]);
}

// Rigorous lower bound of the parameter at which the ray enters box [lo, hi]
// (same frame), +inf when the ray certainly misses it.  Also the exit upper bound.
__device__ __forceinline__ float box_entry_lb(const float *lo, const float *hi, const Ray32 &r, float *exit_ub) {
  float tlo = 0.f, thi = kInfF;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (r.sgn[a] == 0) {
      if (r.phi[a] < lo[a] || r.plo[a] > hi[a]) return kInfF;
      continue;
    }
    float en, ex;
    if (r.sgn[a] > 0) {
      en = div_lo(__fsub_rd(lo[a], r.phi[a]), r, a);
      ex = div_hi(__fsub_ru(hi[a], r.plo[a]), r, a);
    } else {
      en = div_lo(__fsub_rd(r.plo[a], hi[a]), r, a);
      ex = div_hi(__fsub_ru(r.phi[a], lo[a]), r, a);
    }
    tlo = fmaxf(tlo, en);
    thi = fminf(thi, ex);
  }
  if (exit_ub) *exit_ub = thi;
  return tlo > thi ? kInfF : tlo;
}

// Lower bound of the Euclidean distance from the point to box [lo, hi].
__device__ __forceinline__ float box_gap_lb(const float *lo, const float *hi, const Ray32 &r) {
  float d = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) d = fmaxf(d, fmaxf(__fsub_rd(lo[a], r.phi[a]), __fsub_rd(r.plo[a], hi[a])));
  return d;
}

__device__ __forceinline__ float absmax(float lo, float hi) { return fmaxf(fabsf(lo), fabsf(hi)); }
__device__ __forceinline__ float absmin(float lo, float hi) { return (lo <= 0.f && hi >= 0.f) ? 0.f : fminf(fabsf(lo), fabsf(hi)); }

// Bounds of the leaf's DistanceToOut in its own frame: [*lo, *hi].  Boxes get the
// directional interval; orbs and tubes the isotropic safety (lower) and the exit
// of their bounding box (upper).  Also a lower bound of the isotropic safety.
__device__ __forceinline__ void exit_bounds32(const DVol &V, const Ray32 &r, const V3 &p, float *lo, float *hi,
                                              float *safety) {
  float h[3];
  if (V.kind == kBox) {
    h[0] = __double2float_rd(V.p[0]);
    h[1] = __double2float_rd(V.p[1]);
    h[2] = __double2float_rd(V.p[2]);
    float tlo = kInfF, thi = kInfF, s = kInfF;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s = fminf(s, __fsub_rd(h[a], absmax(r.plo[a], r.phi[a])));
      if (r.sgn[a] == 0) continue;
      // exit through the face +h (v > 0) or -h (v < 0): distance (h - s p) / |v| with s = sign(v)
      const float hu = __double2float_ru(V.p[a]);
      float nlo, nhi;
      if (r.sgn[a] > 0) {
        nlo = __fsub_rd(h[a], r.phi[a]);
        nhi = __fsub_ru(hu, r.plo[a]);
      } else {
        nlo = __fadd_rd(h[a], r.plo[a]);
        nhi = __fadd_ru(hu, r.phi[a]);
      }
      tlo = fminf(tlo, div_lo(nlo, r, a));
      thi = fminf(thi, div_hi(nhi, r, a));
    }
    *lo = fmaxf(tlo, 0.f);
    *hi = fmaxf(thi, 0.f);
    *safety = fmaxf(s, 0.f);
    return;
  }
  float ax = absmax(r.plo[0], r.phi[0]), ay = absmax(r.plo[1], r.phi[1]), az = absmax(r.plo[2], r.phi[2]);
  float s;
  float ext[3];
  if (V.kind == kCone) {
    // no FP32 safety (0 bounds it); the exit lies within the bounding box of the end radii
    s = 0.f;
    const double rmax = fmax(V.p[3] - V.p[2] * V.p[4], V.p[3] + V.p[2] * V.p[4]);
    ext[0] = ext[1] = __double2float_ru(rmax);
    ext[2] = __double2float_ru(V.p[4]);
  } else if (V.kind == kOrb) {
    const float R = __double2float_rd(V.p[0]);
    const float rr = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)), __fmul_ru(az, az)));
    s = __fsub_rd(R, rr);
    ext[0] = ext[1] = ext[2] = __double2float_ru(V.p[0]);
  } else {
    const float rmax = __double2float_rd(V.p[1]), hz = __double2float_rd(V.p[2]);
    const float rup = __fsqrt_ru(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)));
    s = fminf(__fsub_rd(rmax, rup), __fsub_rd(hz, az));
    if (V.flags & kHasRmin) {
      const float mx = absmin(r.plo[0], r.phi[0]), my = absmin(r.plo[1], r.phi[1]);
      const float rdn = __fsqrt_rd(__fadd_rd(__fmul_rd(mx, mx), __fmul_rd(my, my)));
      s = fminf(s, __fsub_rd(rdn, __double2float_ru(V.p[0])));
    }
    if (V.flags & kSeg) {
      // phi planes: exact FP64 distances to the two lines, rounded down
      const double ds = fabs(V.p[3] * p.y - V.p[4] * p.x), de = fabs(V.p[6] * p.x - V.p[5] * p.y);
      s = fminf(s, __double2float_rd(fmin(ds, de)));
    }
    ext[0] = ext[1] = __double2float_ru(V.p[1]);
    ext[2] = __double2float_ru(V.p[2]);
  }
  const float mlo[3] = {-ext[0], -ext[1], -ext[2]};
  float xub = kInfF;
  box_entry_lb(mlo, ext, r, &xub);
  *safety = fmaxf(s, 0.f);
  *lo = *safety;
  *hi = xub;
}

// Is the point inside the solid by more than the tolerance band whatever the direction?
// (conservative: false when undecided).
__device__ __forceinline__ bool certainly_inside32(const DVol &V, const Ray32 &r, float band) {
  if (V.kind == kBox) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (!(absmax(r.plo[a], r.phi[a]) < __fsub_rd(__double2float_rd(V.p[a]), band))) return false;
    return true;
  }
  if (V.kind == kCone) return false;
  const float ax = absmax(r.plo[0], r.phi[0]), ay = absmax(r.plo[1], r.phi[1]), az = absmax(r.plo[2], r.phi[2]);
  if (V.kind == kOrb) {
    const float R = __fsub_rd(__double2float_rd(V.p[0]), band);
    return R > 0.f && __fadd_ru(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)), __fmul_ru(az, az)) < __fmul_rd(R, R);
  }
  if (V.flags & kSeg) return false;
  const float rmax = __fsub_rd(__double2float_rd(V.p[1]), band);
  if (!(az < __fsub_rd(__double2float_rd(V.p[2]), band))) return false;
  if (!(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)) < __fmul_rd(rmax, rmax))) return false;
  if (V.flags & kHasRmin) {
    const float rmin = __fadd_ru(__double2float_ru(V.p[0]), band);
    const float mx = absmin(r.plo[0], r.phi[0]), my = absmin(r.plo[1], r.phi[1]);
    if (!(__fadd_rd(__fmul_rd(mx, mx), __fmul_rd(my, my)) > __fmul_ru(rmin, rmin))) return false;
  }
  return true;
}

// Lower bound of the Euclidean distance from mother-frame point (x, y, z) to daughter D's
// solid, from FP32 copies of its placement and size: the FP32 local point is within
// `e` of the exact one (a generous allowance: 2^-20 of the magnitudes involved).
// Negative when the point may be inside.
__device__ __forceinline__ float iso_lb32(const DVol32 &D, float x, float y, float z) {
  const float dx = x - D.tx, dy = y - D.ty, lz = z - D.tz;
  float lx = dx, ly = dy;
  if (!(D.flags & kPlacedAligned)) {
    lx = D.c * dx + D.s * dy;
    ly = D.c * dy - D.s * dx;
  }
  const float e = 9.5367432e-7f * (fabsf(x) + fabsf(y) + fabsf(z) + D.scale) + 1e-30f;
  float d;
  if (D.kind == kBox) {
    d = fmaxf(fabsf(lx) - D.q0, fmaxf(fabsf(ly) - D.q1, fabsf(lz) - D.q2));
  } else if (D.kind == kOrb) {
    d = sqrtf(lx * lx + ly * ly + lz * lz) - D.q0;
  } else {
    const float r = sqrtf(lx * lx + ly * ly);
    d = fmaxf(r - D.q1, fabsf(lz) - D.q2);
    if (D.flags & kHasRmin) d = fmaxf(d, D.q0 - r);
  }
  return d - e;
}

// Conservative FP32 test: can the mother-frame point claim daughter box b?
__device__ __forceinline__ bool box32_contains(const DBox32 &b, float x, float y, float z) {
  return x >= b.lo[0] && x <= b.hi[0] && y >= b.lo[1] && y <= b.hi[1] && z >= b.lo[2] && z <= b.hi[2];
}

// ---------------------------------------------------------------- voxels

__device__ __forceinline__ int slice_of(const DVoxHdr &H, double coord) {
  double f = floor((coord - H.lo) * H.inv_width);
  f = fmin(fmax(f, 0.0), (double)(H.nslices - 1));
  return (int)f;
}

// ---------------------------------------------------------------- FP32 voxel walk
// The FP32 modes walk the voxel nodes with interval arithmetic on the headers' outward
// rounded FP32 copies (lo_dn/lo_up, w_dn/w_up, iw_dn/iw_up) and on the ray's enclosure
// (Ray32).  Every interval encloses the value the FP64 walk computes (each FP64 result
// is a double between two directed-rounded floats of the same operation), so a
// decision taken where the intervals do not overlap is the FP64 walk's decision; an
// overlapping case returns "undecided" and the FP64 code takes that node step.

__device__ __forceinline__ float sel3(float a, float b, float c, int i) { return i == 0 ? a : (i == 1 ? b : c); }
__device__ __forceinline__ int sel3i(int a, int b, int c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

// Slice index of every FP64 coordinate in [qlo, qhi] under slice_of, or -1 if they differ.
__device__ __forceinline__ int slice_of32(const DVoxHdr32 &H, float qlo, float qhi) {
  const float dlo = __fsub_rd(qlo, H.lo_up), dhi = __fsub_ru(qhi, H.lo_dn);
  const float slo = dlo >= 0.f ? __fmul_rd(dlo, H.iw_dn) : __fmul_rd(dlo, H.iw_up);
  const float shi = dhi >= 0.f ? __fmul_ru(dhi, H.iw_up) : __fmul_ru(dhi, H.iw_dn);
  const float top = (float)((H.n_axis >> 2) - 1);
  const float klo = fminf(fmaxf(floorf(slo), 0.f), top), khi = fminf(fmaxf(floorf(shi), 0.f), top);
  return klo == khi ? (int)klo : -1;
}

// Enclosure of the FP64 slab boundaries lo + k0 w and lo + (k1 + 1) w of a merged node.
__device__ __forceinline__ void slab32(const DVoxHdr32 &H, int k0, int k1, float &blo_dn, float &blo_up, float &bhi_dn,
                                       float &bhi_up) {
  const float a = (float)k0, b = (float)(k1 + 1);
  blo_dn = __fadd_rd(H.lo_dn, __fmul_rd(a, H.w_dn));
  blo_up = __fadd_ru(H.lo_up, __fmul_ru(a, H.w_up));
  bhi_dn = __fadd_rd(H.lo_dn, __fmul_rd(b, H.w_dn));
  bhi_up = __fadd_ru(H.lo_up, __fmul_ru(b, H.w_up));
}

// Enclosure [qlo, qhi] of the FP64 coordinate p_a + t v_a for t in [tl, th] (axis a of the ray).
// False when v_a is tiny but not zero (the FP32 enclosure does not hold it).
__device__ __forceinline__ bool advance32(const Ray32 &r, const V3 &v, int a, float tl, float th, float &qlo,
                                          float &qhi) {
  const float plo = sel3(r.plo[0], r.plo[1], r.plo[2], a), phi = sel3(r.phi[0], r.phi[1], r.phi[2], a);
  const int sg = sel3i(r.sgn[0], r.sgn[1], r.sgn[2], a);
  if (sg == 0) {
    qlo = plo;
    qhi = phi;
    return !nonzero_bits(comp(v, a));
  }
  // |v_a| lies in [1 / ihi, 1 / ilo]
  const float ilo = sel3(r.ilo[0], r.ilo[1], r.ilo[2], a), ihi = sel3(r.ihi[0], r.ihi[1], r.ihi[2], a);
  const float vlo = __frcp_rd(ihi), vhi = __frcp_ru(ilo);
  const float mlo = tl >= 0.f ? __fmul_rd(tl, vlo) : __fmul_rd(tl, vhi);
  const float mhi = th >= 0.f ? __fmul_ru(th, vhi) : __fmul_ru(th, vlo);
  if (sg > 0) {
    qlo = __fadd_rd(plo, mlo);
    qhi = __fadd_ru(phi, mhi);
  } else {
    qlo = __fsub_rd(plo, mhi);
    qhi = __fsub_ru(phi, mlo);
  }
  return true;
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

// ---------------------------------------------------------------- exact coordinate keys
// key(x): a double's bits as a signed integer with the negative half reflected,
// so that x < y <=> key(x) < key(y).  The geometry carries, for world-aligned
// boxes and for the voxel slices of world-aligned mothers, the keys at which the
// FP64 predicates (Inside bands, slice index) change value; comparing keys then
// gives the FP64 answer with integer instructions only.


// A float near x built from the high word of its bits (truncated; no FP64 instruction).
__device__ __forceinline__ float approx_float(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const int e = (int)((hi >> 20) & 0x7ffu);
  const unsigned sg = hi & 0x80000000u;
  if (e < 897) return __uint_as_float(sg);
  if (e > 1150) return __uint_as_float(sg | 0x7f7fffffu);
  return __uint_as_float(sg | ((unsigned)(e - 896) << 23) | ((hi & 0xfffffu) << 3));
}

// A world point and direction with the keys of the point and a float guess of it.
struct WPos {
  V3 x, u;
  long long k[3];
  float f[3];
};

__device__ __forceinline__ WPos make_wpos(const V3 &x, const V3 &u) {
  WPos W;
  W.x = x;
  W.u = u;
  W.k[0] = dkey(x.x);
  W.k[1] = dkey(x.y);
  W.k[2] = dkey(x.z);
  W.f[0] = approx_float(x.x);
  W.f[1] = approx_float(x.y);
  W.f[2] = approx_float(x.z);
  return W;
}

__device__ __forceinline__ long long kcomp(const long long *k, int a) { return a == 0 ? k[0] : (a == 1 ? k[1] : k[2]); }
__device__ __forceinline__ float fcomp(const float *f, int a) { return a == 0 ? f[0] : (a == 1 ? f[1] : f[2]); }

// box_inside on p = x - t of a kKeyBox volume d (the same answer, by its keys).
// In the surface band of axis a the sign of p_a is known (the side of the band),
// so p_a v_a >= 0 reduces to a sign test; only a subnormal v_a needs the product.
__device__ __forceinline__ bool keybox_inside(const DGeom &G, int d, const WPos &W) {
  const DKeyBox &K = G.kbox[d];
  int near = 0;  // bit a: axis a in the band; bit a + 3: on its high side
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long k = W.k[a];
    if (k <= K.k[a][0] || k >= K.k[a][3]) return false;
    if (k <= K.k[a][1]) near |= 1 << a;
    else if (k >= K.k[a][2]) near |= 9 << a;
  }
  if (!near) return true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(near & (1 << a))) continue;
    const double va = comp(W.u, a);
    const long long vb = __double_as_longlong(va);
    const long long mag = vb & 0x7FFFFFFFFFFFFFFFll;
    if (mag == 0) return false;                      // p_a v_a = 0
    if (mag < 0x0010000000000000ll) {                // subnormal v_a: the product decides
      const DWorld &w = G.wxf[d];
      const double pa = comp(W.x, a) - (a == 0 ? w.tx : (a == 1 ? w.ty : w.tz));
      if (pa * va >= 0.0) return false;
    } else if ((vb < 0) != ((near >> (a + 3)) & 1)) {
      return false;                                  // v_a points outward
    }
  }
  return true;
}

// vox_lookup for a keyed header tree (world-aligned mother), from the world point.
__device__ __forceinline__ int vox_lookup_keys(const DGeom &G, int h, const WPos &W) {
#pragma unroll 1
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    const DVoxHdr H = G.hdr[h];
    const int n = H.nslices;
    const long long kx = kcomp(W.k, H.axis);
    const long long *S = reinterpret_cast<const long long *>(G.skey) + H.slice_base;
    int k = __float2int_rd((fcomp(W.f, H.axis) - H.lo_wf) * H.inv_wf);
    k = max(0, min(k, n - 1));
#pragma unroll 1
    while (k > 0 && kx < __ldg(&S[k])) --k;
#pragma unroll 1
    while (k + 1 < n && kx >= __ldg(&S[k + 1])) ++k;
    const DVoxSlice Sl = G.slice[H.slice_base + k];
    if (Sl.child >= 0) return Sl.child;
    h = -Sl.child - 1;
  }
  return 0;
}

// Warp-collective navigation.  Every lane of the warp must call these functions
// together (they synchronise with __syncwarp / __any_sync over the full warp);
// lanes with `active` false only take part in the synchronisation.  The point is
// SIMT efficiency: each round every searching lane first scans its candidate list
// in cheap FP32/integer code to the next candidate that needs FP64 work, then the
// warp meets and all those lanes run the FP64 test together.
constexpr unsigned kFull = 0xffffffffu;

// Descend from volume m into the first daughter, in id order, that contains the
// point; repeat.  (p, v) is the point in m's frame when have_p is set; otherwise it
// is derived from the world point when an FP64 test needs it.  kKeyBox daughters
// and keyed voxel trees are answered from the world point's keys.  `blocked` is a
// daughter of m already known not to contain the point (the volume just left).
// Returns the deepest volume.
template <bool COUNT>
__device__ __forceinline__ int descend_body(const DGeom &G, bool active, int m, V3 p, V3 v, bool have_p,
                                            const WPos &W, int blocked, Counters &cnt) {
#pragma unroll 1
  for (int lev = 0; lev < kDMax; ++lev) {
    const bool want = active && G.vol[m].vox >= 0;
    if (!__any_sync(kFull, want)) break;
    DCandList L{0, 0};
    if (want) {
      const int h = G.vol[m].vox;
      if (G.hdr[h].keyed) {
        L = G.clist[vox_lookup_keys(G, h, W)];
      } else {
        if (!have_p) {
          world_to_local(G.wxf[m], G.vol[m].flags & kWorldAligned, W.x, W.u, p, v);
          have_p = true;
        }
        L = G.clist[vox_lookup(G, h, p)];
      }
    }
    float px = 0.f, py = 0.f, pz = 0.f;
    bool have_pf = false;
    int i = 0, found = -1;
    bool searching = want, via_fp64 = false;
    V3 fp = p, fv = v;
#pragma unroll 1
    while (__any_sync(kFull, searching)) {
      int d = -1;
      if (searching) {
#pragma unroll 1
        while (i < L.count) {
          const int c = __ldg(&G.cand[L.offset + i]);
          ++i;
          if (c == blocked) continue;
          const DBox32 &B = G.box[c];
          if (B.keyed) {
            diag<COUNT>(cnt, G4N_C_KEY_INSIDE);
            if (keybox_inside(G, c, W)) {
              found = c;
              searching = false;
              break;
            }
            continue;
          }
          if (!have_p) {
            world_to_local(G.wxf[m], G.vol[m].flags & kWorldAligned, W.x, W.u, p, v);
            have_p = true;
          }
          if (!have_pf) {
            px = (float)p.x;
            py = (float)p.y;
            pz = (float)p.z;
            have_pf = true;
          }
          if (box32_contains(B, px, py, pz) && !(iso_lb32(G.v32[c], px, py, pz) > (float)(2.0 * G.half))) {
            d = c;
            break;
          }
        }
        if (d < 0) searching = false;
      }
      __syncwarp();
      if (d >= 0) {
        const DVol &D = G.vol[d];
        V3 dp, dv;
        to_local(D, p, v, dp, dv);
        diag_test<COUNT>(cnt, G4N_C_INSIDE, G4N_C_INSIDE_CURVED, D.kind);
        if (vol_inside(D, dp, dv, G.half)) {
          found = d;
          fp = dp;
          fv = dv;
          via_fp64 = true;
          searching = false;
        }
      }
    }
    if (want && found >= 0) {
      m = found;
      have_p = via_fp64;
      p = fp;
      v = fv;
      blocked = -1;
    } else {
      active = false;
    }
  }
  return m;
}

// The descent out of line: one copy of its code serves every call site of a kernel.  The
// FP32 modes use it (their kernels are larger and stall on instruction fetch, which the
// shared copy relieves: measured 8 % on the barrel scene); the FP64 navigator inlines it
// (measured 2 % faster on the calorimeter, whose relocations are mostly face records).
// Counters are passed by pointer (null without diagnostics) so that they stay in registers.
template <bool COUNT>
__device__ __noinline__ int descend_ool(const DGeom &G, bool active, int m, V3 p, V3 v, bool have_p, const WPos &W,
                                        int blocked, Counters *cntp) {
  Counters none;
  return descend_body<COUNT>(G, active, m, p, v, have_p, W, blocked, COUNT ? *cntp : none);
}

template <bool COUNT, bool OOL>
__device__ __forceinline__ int descend_warp(const DGeom &G, bool active, int m, V3 p, V3 v, bool have_p,
                                            const WPos &W, int blocked, Counters &cnt) {
  if (OOL) return descend_ool<COUNT>(G, active, m, p, v, have_p, W, blocked, COUNT ? &cnt : nullptr);
  return descend_body<COUNT>(G, active, m, p, v, have_p, W, blocked, cnt);
}

// Locate from the world (warp-collective): the leaf, or -1 outside the world.
template <bool COUNT, bool OOL = false>
__device__ __forceinline__ int locate_world_warp(const DGeom &G, bool active, const V3 &x, const V3 &u, Counters &cnt) {
  V3 p{0, 0, 0}, v{0, 0, 1};
  bool in = false, have_p = false;
  const WPos W = make_wpos(x, u);
  if (active) {
    if (G.vol[0].flags & kKeyBox) {
      diag<COUNT>(cnt, G4N_C_KEY_INSIDE);
      in = keybox_inside(G, 0, W);
    } else {
      world_to_local(G.wxf[0], G.vol[0].flags & kWorldAligned, x, u, p, v);
      have_p = true;
      diag_test<COUNT>(cnt, G4N_C_INSIDE, G4N_C_INSIDE_CURVED, G.vol[0].kind);
      in = vol_inside(G.vol[0], p, v, G.half);
    }
  }
  const int leaf = descend_warp<COUNT, OOL>(G, in, 0, p, v, have_p, W, -1, cnt);
  return in ? leaf : -1;
}

// After a move (warp-collective): leave every volume that no longer contains the
// point, then descend.  A step that ended on the leaf's own exit surface (limiter
// mother, positive length) leaves the leaf for certain: the point is on that
// surface moving outward, so the leaf's Inside test is false and is skipped.  A
// volume left on the way up is blocked in the descent below its mother (its
// Inside is already known to be false).  Returns the new leaf or -1 (left the world).
template <int MODE, bool COUNT>
__device__ __forceinline__ int relocate_warp(const DGeom &G, bool active, int leaf, const V3 &x, const V3 &u,
                                             bool left_leaf, Counters &cnt) {
  if (!__any_sync(kFull, active)) return -1;  // no lane relocates: skip the warp's whole search
  int blocked = -1;
  if (active && left_leaf) {
    blocked = leaf;
    leaf = G.vol[leaf].mother;
  }
  bool up = active && leaf >= 0;
  bool in = false, have_p = false;
  V3 p{0, 0, 0}, v{0, 0, 1};
  const WPos W = make_wpos(x, u);
#pragma unroll 1
  while (__any_sync(kFull, up)) {
    if (up) {
      const DVol &L = G.vol[leaf];
      bool ok = false;
      if (L.flags & kKeyBox) {
        diag<COUNT>(cnt, G4N_C_KEY_INSIDE);
        ok = keybox_inside(G, leaf, W);
        have_p = false;
      } else {
        world_to_local(G.wxf[leaf], L.flags & kWorldAligned, x, u, p, v);
        have_p = true;
        if (MODE != kFP64) ok = certainly_inside32(L, make_ray32(p, v), (float)(4.0 * G.half) + 1e-30f);
        if (!ok) {
          diag_test<COUNT>(cnt, G4N_C_INSIDE, G4N_C_INSIDE_CURVED, L.kind);
          ok = vol_inside(L, p, v, G.half);
        }
      }
      if (ok) {
        in = true;
        up = false;
      } else {
        blocked = leaf;
        leaf = L.mother;
        if (leaf < 0) up = false;
      }
    }
  }
  const int out = descend_warp<COUNT, MODE != kFP64>(G, in, in ? leaf : 0, p, v, have_p, W, blocked, cnt);
  return in ? out : -1;
}

// Relocation after a step that left kKeyBox volume `leaf` through `face` (limiter mother,
// positive length), from the volume's precomputed face record: true, and the new leaf
// (-1: left the world) in *out, when x lies in the record's region and the direction's
// normal component is not subnormal; the answer is then the one relocate_warp gives.
__device__ __forceinline__ bool face_relocate(const DGeom &G, int leaf, int face, const V3 &x, const V3 &u, int *out) {
  const int base = G.vol[leaf].face;
  if (base < 0 || face < 0) return false;
  const DFace &F = G.face[base + face];
  if (!F.ok) return false;
  if ((__double_as_longlong(comp(u, face >> 1)) & 0x7FF0000000000000ll) == 0) return false;
  const long long kx = dkey(x.x), ky = dkey(x.y), kz = dkey(x.z);
  if (kx < F.k[0][0] || kx > F.k[0][1] || ky < F.k[1][0] || ky > F.k[1][1] || kz < F.k[2][0] || kz > F.k[2][1])
    return false;
  *out = F.leaf;
  return true;
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

// One node step of the plain FP64 voxel walk: the exit texit of the current node along the
// ray (the first level whose slab the ray leaves), the end test texit >= bound, the
// neighbouring node across that face and the lookup of its deeper levels at p + texit v.
// Returns 0: the walk ends; 1: ch holds the next node.  With `saf` the distances from the
// point to the node's slab faces lower *saf.
__device__ __forceinline__ int walk_step64(const DGeom &G, Chain &ch, const V3 &p, const V3 &v, const Inv3 &iv,
                                           double bound, bool saf, double *saf64, int *it, int cap, bool *timeout) {
  double texit = kInf;
  int lstar = -1;
#pragma unroll 1
  for (int l = 0; l < ch.nlev; ++l) {
    const DVoxHdr H = G.hdr[ch.h[l]];
    const double pa = comp(p, H.axis), va = comp(v, H.axis);
    const double blo = H.lo + ch.k0[l] * H.width, bhi = H.lo + (ch.k1[l] + 1) * H.width;
    if (saf) *saf64 = fmin(*saf64, fmax(fmin(pa - blo, bhi - pa), 0.0));
    double t = kInf;
    if (va > 0.0) t = (bhi - pa) * icomp(iv, H.axis);
    else if (va < 0.0) t = (blo - pa) * icomp(iv, H.axis);
    if (t < texit) {
      texit = t;
      lstar = l;
    }
  }
  if (!(texit < bound)) return 0;
  const DVoxHdr H = G.hdr[ch.h[lstar]];
  const int nk = comp(v, H.axis) > 0.0 ? ch.k1[lstar] + 1 : ch.k0[lstar] - 1;
  if (nk < 0 || nk >= H.nslices || ++*it >= cap) {
    if (*it >= cap) *timeout = true;
    return 0;
  }
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
  return 1;
}

// The same, out of line: the FP32 modes take it only when their intervals do not decide.
__device__ __noinline__ int walk_step64_ool(const DGeom &G, Chain &ch, const V3 &p, const V3 &v, const Inv3 &iv,
                                            double bound, bool saf, double *saf64, int *it, int cap, bool *timeout) {
  return walk_step64(G, ch, p, v, iv, bound, saf, saf64, it, cap, timeout);
}

// chain_fill from the root header h0 for every FP64 point in the ray's enclosure (FP32
// modes); false if a level's slice index is undecided (the caller then fills in FP64).
__device__ __forceinline__ bool chain_fill32(const DGeom &G, Chain &ch, int h, const Ray32 &r) {
#pragma unroll 1
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    const DVoxHdr32 H = G.hdr32[h];
    const int a = H.n_axis & 3;
    const int k = slice_of32(H, sel3(r.plo[0], r.plo[1], r.plo[2], a), sel3(r.phi[0], r.phi[1], r.phi[2], a));
    if (k < 0) return false;
    const DVoxSlice S = G.slice[H.slice_base + k];
    ch.h[lev] = h;
    ch.k0[lev] = S.k0;
    ch.k1[lev] = S.k1;
    if (S.child >= 0) {
      ch.nlev = lev + 1;
      ch.list = S.child;
      return true;
    }
    h = -S.child - 1;
  }
  ch.nlev = kMaxLevels;
  ch.list = 0;
  return true;
}

// Lower / upper bound of num / |v_a| for a runtime axis a.
__device__ __forceinline__ float div_lo_a(float n, const Ray32 &r, int a) {
  return n >= 0.f ? __fmul_rd(n, sel3(r.ilo[0], r.ilo[1], r.ilo[2], a)) : __fmul_rd(n, sel3(r.ihi[0], r.ihi[1], r.ihi[2], a));
}
__device__ __forceinline__ float div_hi_a(float n, const Ray32 &r, int a) {
  return n >= 0.f ? __fmul_ru(n, sel3(r.ihi[0], r.ihi[1], r.ihi[2], a)) : __fmul_ru(n, sel3(r.ilo[0], r.ilo[1], r.ilo[2], a));
}

// One node step of the voxel walk in FP32 interval arithmetic (FP32 modes): the exit of
// the current node along the ray (the level whose slab the ray leaves first), the end
// test against bound_f (an upper bound of the FP64 walk's bound min(best, stop)), the
// neighbouring node and the lookup of its deeper levels at the entry point.  Returns 0:
// the walk ends; 1: ch holds the next node; 2: undecided (ch unchanged), the FP64 code
// takes this node step.  With `saf` the distances from the point to the node's slab
// faces lower the isotropic safety *saf_f.
__device__ __forceinline__ int walk_step32(const DGeom &G, Chain &ch, const Ray32 &r, const V3 &v, float bound_f,
                                           bool saf, float *saf_f, int *it, int cap, bool *timeout) {
  float tl[kMaxLevels], th[kMaxLevels];
  const int nlev = ch.nlev;
  int lstar = -1;
  float ts_lo = kInfF, ts_hi = kInfF;
  bool tiny = false;
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    tl[l] = th[l] = kInfF;
    if (l < nlev) {
      const DVoxHdr32 H = G.hdr32[ch.h[l]];
      const int a = H.n_axis & 3;
      float blo_dn, blo_up, bhi_dn, bhi_up;
      slab32(H, ch.k0[l], ch.k1[l], blo_dn, blo_up, bhi_dn, bhi_up);
      const float plo = sel3(r.plo[0], r.plo[1], r.plo[2], a), phi = sel3(r.phi[0], r.phi[1], r.phi[2], a);
      if (saf) *saf_f = fminf(*saf_f, fmaxf(fminf(__fsub_rd(plo, blo_up), __fsub_rd(bhi_dn, phi)), 0.f));
      const int sg = sel3i(r.sgn[0], r.sgn[1], r.sgn[2], a);
      if (sg > 0) {
        tl[l] = div_lo_a(__fsub_rd(bhi_dn, phi), r, a);
        th[l] = div_hi_a(__fsub_ru(bhi_up, plo), r, a);
      } else if (sg < 0) {
        tl[l] = div_lo_a(__fsub_rd(plo, blo_up), r, a);
        th[l] = div_hi_a(__fsub_ru(phi, blo_dn), r, a);
      } else {
        tiny |= nonzero_bits(comp(v, a));  // a direction component too small for the enclosure
      }
      if (th[l] < ts_hi) {
        ts_hi = th[l];
        ts_lo = tl[l];
        lstar = l;
      }
    }
  }
  if (tiny) return 2;
  if (lstar < 0) return 0;  // the ray leaves no slab: the FP64 exit is +inf
  // the FP64 minimum is taken by lstar alone (the first level attaining it wins ties)
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l)
    if (l != lstar && !(tl[l] > ts_hi)) return 2;
  if (ts_lo >= bound_f) return 0;  // texit >= bound_f >= min(best, stop)
  const DVoxHdr32 H = G.hdr32[ch.h[lstar]];
  const int nk = sel3i(r.sgn[0], r.sgn[1], r.sgn[2], H.n_axis & 3) > 0 ? ch.k1[lstar] + 1 : ch.k0[lstar] - 1;
  if (nk < 0 || nk >= (H.n_axis >> 2) || ++*it >= cap) {
    if (*it >= cap) *timeout = true;
    return 0;
  }
  const DVoxSlice S = G.slice[H.slice_base + nk];
  int list = S.child;
  int dh[kMaxLevels - 1], dk0[kMaxLevels - 1], dk1[kMaxLevels - 1];
  int nd = 0;
  if (list < 0) {
    // deeper levels: slices of the entry point p + texit v, texit in [ts_lo, ts_hi]
    int hh = -S.child - 1;
#pragma unroll
    for (int j = 0; j < kMaxLevels - 1; ++j) {
      if (list < 0 && lstar + 1 + j < kMaxLevels) {
        const DVoxHdr32 D = G.hdr32[hh];
        float qlo, qhi;
        if (!advance32(r, v, D.n_axis & 3, ts_lo, ts_hi, qlo, qhi)) return 2;
        const int k = slice_of32(D, qlo, qhi);
        if (k < 0) return 2;
        const DVoxSlice Sd = G.slice[D.slice_base + k];
        dh[j] = hh;
        dk0[j] = Sd.k0;
        dk1[j] = Sd.k1;
        nd = j + 1;
        if (Sd.child >= 0) list = Sd.child;
        else hh = -Sd.child - 1;
      }
    }
  }
  ch.k0[lstar] = S.k0;
  ch.k1[lstar] = S.k1;
#pragma unroll
  for (int j = 0; j < kMaxLevels - 1; ++j) {
    if (j < nd) {
      ch.h[lstar + 1 + j] = dh[j];
      ch.k0[lstar + 1 + j] = dk0[j];
      ch.k1[lstar + 1 + j] = dk1[j];
    }
  }
  if (list >= 0) {
    ch.nlev = lstar + 1 + nd;
    ch.list = list;
  } else {
    ch.nlev = kMaxLevels;
    ch.list = 0;
  }
  return 1;
}

// Training-sample log written by the plain navigator (features, label = list slot of the
// daughter entered, candidate count); `count` may exceed `capacity` (extra samples dropped).
struct MlpLog {
  float *feat;
  int32_t *label;
  int32_t *ncand;
  unsigned long long *count;
  int64_t capacity;
};

// What geom_step needs for the proposal: the weights and this warp's scratch (learned
// mode), the sample log (plain mode, optional) and the track's log-energy feature.
struct MlpCtx {
  const mlp::SmemWeights *w;
  mlp::SmemWarp *scratch;
  const MlpLog *log;
  float loge;
};

// Proposal features of the node holding p (leaf frame): the point in the node's own
// coordinates (axes the node does not slice use the leaf's half extent), the direction,
// log E, n / 32 and 1.
__device__ __forceinline__ void node_features(const DGeom &G, const DVol &V, const Chain &ch, const V3 &p, const V3 &v,
                                              float loge, int n, float *f) {
  double c[3] = {0.0, 0.0, 0.0};
  double h[3];
  if (V.kind == kBox) {
    h[0] = V.p[0];
    h[1] = V.p[1];
    h[2] = V.p[2];
  } else if (V.kind == kOrb) {
    h[0] = h[1] = h[2] = V.p[0];
  } else if (V.kind == kCone) {
    h[0] = h[1] = fmax(V.p[3] - V.p[2] * V.p[4], V.p[3] + V.p[2] * V.p[4]);
    h[2] = V.p[4];
  } else {
    h[0] = h[1] = V.p[1];
    h[2] = V.p[2];
  }
  for (int l = 0; l < ch.nlev; ++l) {
    const DVoxHdr H = G.hdr[ch.h[l]];
    const double lo = H.lo + ch.k0[l] * H.width, hi = H.lo + (ch.k1[l] + 1) * H.width;
    c[H.axis] = 0.5 * (lo + hi);
    h[H.axis] = 0.5 * (hi - lo);
  }
  f[0] = fminf(fmaxf((float)((p.x - c[0]) / h[0]), -2.f), 2.f);
  f[1] = fminf(fmaxf((float)((p.y - c[1]) / h[1]), -2.f), 2.f);
  f[2] = fminf(fmaxf((float)((p.z - c[2]) / h[2]), -2.f), 2.f);
  f[3] = (float)v.x;
  f[4] = (float)v.y;
  f[5] = (float)v.z;
  f[6] = loge;
  f[7] = (float)n * (1.0f / 32.0f);
  f[8] = 1.0f;
}

// A boundary search that yields after walking its budget of voxel nodes is continued in a
// later round at the node it had stepped into (its Chain, kept by the caller), with the best
// daughter found so far and the safety bound of its first round.
struct WalkResume {
  double best;    // best DistanceToIn found so far (+inf: none)
  double safety;  // isotropic safety bound of the first round
  int bl;         // the daughter of `best` (G4N_LIM_MOTHER: none)
  int it;         // voxel nodes walked so far (the walk's iteration cap)
};

struct StepResult {
  double step;    // geometric step (exact when it is <= the limit)
  double safety;  // isotropic lower bound
  int lim;        // daughter id or G4N_LIM_MOTHER
  int face;       // limiter mother and a box leaf: the exit face (2 axis + (v_axis > 0)), else -1
  bool physics;   // FP32 mode: proven that the limit comes first (no FP64 geometry done)
  bool yielded;   // the search used its node budget: continue it from `resume`
  WalkResume resume;
};

// iv: the reciprocal of v; the FP32 modes read it only when the leaf is a box (its exit).
//
// Geometric step inside `leaf` from local point p along v (Sec. 3.2, problem 2),
// warp-collective: DistanceToOut of the leaf, then DistanceToIn of the daughters
// listed in the voxel nodes the ray crosses, stopping once the node exit lies
// beyond the best distance or `limit`.  FP64 mode: every candidate in FP64.  FP32
// mode: a candidate is evaluated in FP64 only if its FP32 entry bound does not
// exceed the best exact distance so far, and no FP64 geometry at all is done when
// the bounds prove that `limit` comes first.  Both return the FP64 result.
//
// walk_cap: the voxel nodes a search may walk in all (its rounds together); a search that reaches it
// stops there and sets *timeout (the caller reports G4N_ERR_TIMEOUT).
//
// Budget (budget > 0): after `budget` node steps a lane's search yields (R.yielded, with the
// state to continue from in R.resume and in `ch`, which then holds the node stepped into);
// `resume` continues such a search from there.  The result of a search is the same whether
// or not it yields.  `ch` is the caller's voxel chain (per-lane local memory).
template <int MODE, bool COUNT>
__device__ __forceinline__ StepResult geom_step_warp(const DGeom &G, bool active, int leaf, const V3 &p, const V3 &v,
                                                     const Inv3 &iv, double limit, bool want_safety, Counters &cnt,
                                                     bool *timeout, int walk_cap, const MlpCtx &mc, Chain &ch,
                                                     bool resume = false,
                                                     const WalkResume &from = WalkResume{kInf, 0.0, -1, 0},
                                                     int budget = 0) {
  const double half = G.half;
  StepResult R{kInf, 0.0, G4N_LIM_MOTHER, -1, false, false, WalkResume{kInf, 0.0, -1, 0}};
  int nodes = 0;          // node steps taken in this call (the budget)
  double best = kInf, stop = 0.0, tout = kInf;
  int oface = -1;
  float out_lo = 0.f;
  float bound_f = kInfF;  // FP32 modes: float >= min(best, stop), the FP32 walk's bound
  float saf_f = 0.f;      // FP32 modes: the isotropic safety bound
  Ray32 r;
  bool walking = false, first = true;
  int i = 0, it = 0, bl = G4N_LIM_MOTHER;
  DCandList L{0, 0}, L0{0, 0};
  int prop_done = -1;
  float feat[mlp::kIn];
  bool have_feat = false;
  if (active) {
    const DVol &V = G.vol[leaf];
    if (MODE != kFP64) {
      r = make_ray32(p, v);
      float out_hi, saf32;
      exit_bounds32(V, r, p, &out_lo, &out_hi, &saf32);
      saf_f = resume ? (float)from.safety : saf32;
      stop = fmin(limit, (double)out_hi);
    } else {
      diag_test<COUNT>(cnt, G4N_C_DIST_OUT, G4N_C_DIST_OUT_CURVED, V.kind);
      tout = vol_dist_out(V, p, v, iv, half, &oface);
      R.safety = resume ? from.safety : (want_safety ? vol_safety_out(V, p) : 0.0);
      stop = fmin(limit, tout);
    }
    if (resume) {
      best = from.best;
      bl = from.bl;
      it = from.it;
      first = false;
    }
    if (MODE != kFP64) bound_f = __double2float_ru(fmin(best, stop));
    if (V.vox >= 0) {
      if (!resume && (MODE == kFP64 || !chain_fill32(G, ch, V.vox, r))) chain_fill(G, ch, 0, V.vox, p);
      L = G.clist[ch.list];
      L0 = L;
      walking = true;
      diag<COUNT>(cnt, G4N_C_VOX_NODES);
      if (!resume && (MODE == kLearned || mc.log) && L.count >= 2 && L.count <= mlp::kOut) {
        // learned mode: a proposal can only save work when two or more of the node's candidates pass
        // the FP32 bounds (with one or none the bounds alone leave a single FP64 evaluation at most)
        int open = 2;
        if (MODE == kLearned) {
          open = 0;
#pragma unroll 1
          for (int k = 0; k < L.count && open < 2; ++k) {
            const int c = __ldg(&G.cand[L.offset + k]);
            const DBox32 B = G.box[c];
            const float iso = iso_lb32(G.v32[c], r.plo[0], r.plo[1], r.plo[2]) - (float)(2.0 * G.half);
            if (fmaxf(box_entry_lb(B.lo, B.hi, r, nullptr), iso) <= bound_f) ++open;
          }
        }
        if (open >= 2) {
          node_features(G, V, ch, p, v, mc.loge, L.count, feat);
          have_feat = true;
        }
      }
    }
  }
  // learned mode: the network proposes which first-node candidate is entered first; it is
  // evaluated before the others so that its exact distance prunes them (warp-collective)
  int prop = -1;
  if (MODE == kLearned && __any_sync(kFull, have_feat)) {
    float f0[mlp::kIn];
#pragma unroll
    for (int k = 0; k < mlp::kIn; ++k) f0[k] = have_feat ? feat[k] : 0.f;
    mlp::put_features(*mc.scratch, f0);
    mlp::forward_warp(*mc.w, *mc.scratch);
    if (have_feat) {
      prop = mlp::argmax_row(*mc.scratch, L.count);
      diag<COUNT>(cnt, G4N_C_PROPOSALS);
    }
    __syncwarp();
  }
#pragma unroll 1
  while (__any_sync(kFull, walking)) {
    int d = -1;
    bool from_first = false;
    if (walking) {
      // scan to the next candidate that needs FP64 work, walking nodes as lists run out
#pragma unroll 1
      for (;;) {
        if (MODE == kLearned && prop >= 0) {
          // the proposal goes first if its bound still allows it to matter
          const int c = __ldg(&G.cand[L0.offset + prop]);
          const DBox32 B = G.box[c];
          const float iso = iso_lb32(G.v32[c], r.plo[0], r.plo[1], r.plo[2]) - (float)(2.0 * G.half);
          const float lb = fmaxf(box_entry_lb(B.lo, B.hi, r, nullptr), iso);
          if (lb <= bound_f) {
            d = c;
            from_first = true;
            break;
          }
          prop = -1;  // not worth it: the scan treats the slot like any other
        }
        if (i < L.count) {
          const int c = __ldg(&G.cand[L.offset + i]);
          ++i;
          if (MODE != kFP64) {
            const DBox32 B = G.box[c];
            const float iso = iso_lb32(G.v32[c], r.plo[0], r.plo[1], r.plo[2]) - (float)(2.0 * G.half);
            if (first && want_safety) saf_f = fminf(saf_f, fmaxf(box_gap_lb(B.lo, B.hi, r), iso));
            if (MODE == kLearned && first && i - 1 == prop_done) continue;  // already evaluated exactly
            const float lb = fmaxf(box_entry_lb(B.lo, B.hi, r, nullptr), iso);
            if (!(lb <= bound_f)) {
              if (MODE == kLearned) diag<COUNT>(cnt, G4N_C_PRUNED);
              continue;
            }
            diag<COUNT>(cnt, G4N_C_RECHECKS);
          }
          d = c;
          from_first = first;
          break;
        }
        // list done: exit of the current node along the ray; its slab boundaries bound the safety
        int w = 2;
        if (MODE != kFP64) w = walk_step32(G, ch, r, v, bound_f, first && want_safety, &saf_f, &it, walk_cap, timeout);
        if (w == 2) {
          // FP64 node step (the FP32 modes come here only when the intervals do not decide)
          if (MODE == kFP64) {
            w = walk_step64(G, ch, p, v, iv, fmin(best, stop), first && want_safety, &R.safety, &it, walk_cap, timeout);
          } else {
            double s64 = kInf;
            w = walk_step64_ool(G, ch, p, v, inv_dir(v), fmin(best, stop), first && want_safety, &s64, &it, walk_cap,
                                timeout);
            saf_f = fminf(saf_f, __double2float_rd(s64));
          }
        }
        first = false;
        if (w == 0) {
          walking = false;
          break;
        }
        if (budget > 0 && ++nodes >= budget) {
          // yield: ch holds the node stepped into; the search continues there in a later round
          walking = false;
          R.yielded = true;
          diag<COUNT>(cnt, G4N_C_WALK_YIELDS);
          break;
        }
        L = G.clist[ch.list];
        i = 0;
        diag<COUNT>(cnt, G4N_C_VOX_NODES);
      }
    }
    __syncwarp();
    if (MODE == kLearned && prop >= 0 && d >= 0) {
      prop_done = prop;  // the proposed slot is skipped when the first node is scanned
      prop = -1;
      diag<COUNT>(cnt, G4N_C_RECHECKS);
    }
    if (d >= 0) {
      const DVol &D = G.vol[d];
      V3 dp, dv;
      to_local(D, p, v, dp, dv);
      diag_kind<COUNT>(cnt, D.kind);
      const double t = vol_dist_in(D, dp, dv, half);
      if (t < kInf && (t < best || (t == best && (bl < 0 || d < bl)))) {
        best = t;
        bl = d;
        if (MODE != kFP64) bound_f = __double2float_ru(fmin(best, stop));
      }
      if (MODE == kFP64 && from_first && want_safety) R.safety = fmin(R.safety, vol_safety_in(D, dp));
    }
  }
  if (MODE != kFP64) R.safety = saf_f;
  if (!active) return R;
  if (R.yielded) {
    R.resume = WalkResume{best, R.safety, bl, it};
    return R;
  }
  if (MODE == kFP64 && mc.log && have_feat && bl >= 0 && best <= tout) {
    // training sample: the daughter entered, if it is listed in the first node
    int slot = -1;
    for (int k = 0; k < L0.count; ++k)
      if (__ldg(&G.cand[L0.offset + k]) == bl) {
        slot = k;
        break;
      }
    if (slot >= 0) {
      const unsigned long long at = atomicAdd(mc.log->count, 1ull);
      if ((int64_t)at < mc.log->capacity) {
        for (int k = 0; k < mlp::kIn; ++k) mc.log->feat[at * mlp::kIn + k] = feat[k];
        mc.log->label[at] = slot;
        mc.log->ncand[at] = L0.count;
      }
    }
  }
  if (MODE != kFP64) {
    // the FP32 bounds prove the limit comes first: no FP64 geometry needed
    if (best > limit && (double)out_lo > limit) {
      R.physics = true;
      return R;
    }
    diag_test<COUNT>(cnt, G4N_C_DIST_OUT, G4N_C_DIST_OUT_CURVED, G.vol[leaf].kind);
    tout = vol_dist_out(G.vol[leaf], p, v, iv, half, &oface);
  }
  // a daughter wins a tie with the mother; `best` already holds the lowest id among tied daughters
  if (bl >= 0 && best <= tout) {
    R.step = best;
    R.lim = bl;
  } else {
    R.step = tout;
    R.lim = G4N_LIM_MOTHER;
    R.face = oface;
  }
  return R;
}

// ---------------------------------------------------------------- attenuation table

// Bin k with E_k <= E < E_{k+1} and its interpolation fraction; clamped ends give
// (0, 0) below the table and (n-2, 1) above.
__device__ __forceinline__ void energy_bin(const double *Eg, int n, double E, int &k, double &f) {
  if (E <= Eg[0]) {
    k = 0;
    f = 0.0;
  } else if (E >= Eg[n - 1]) {
    k = n - 2;
    f = 1.0;
  } else {
    int lo = 0, hi = n - 1;
    const long long eb = __double_as_longlong(E);  // E and the grid are positive: bit order = value order
#pragma unroll 1
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__double_as_longlong(Eg[mid]) <= eb) lo = mid;
      else hi = mid;
    }
    k = lo;
    f = (E - Eg[lo]) / (Eg[lo + 1] - Eg[lo]);
  }
}

// Lin-lin interpolation of both coefficients at a known bin.  At the clamped ends
// the table value is returned exactly.
__device__ __forceinline__ void mu_at(const DGeom &G, int mat, int k, double f, double &mu_tot, double &mu_pe) {
  const int off = G.mat_off[mat];
  const double *C = G.matC + off, *P = G.matP + off;
  double mc, mp;
  const long long fb = __double_as_longlong(f);
  if (fb == 0) {                                   // f == +0 (f is never -0 or negative)
    mc = C[k];
    mp = P[k];
  } else if (fb == 0x3FF0000000000000ll) {         // f == 1
    mc = C[k + 1];
    mp = P[k + 1];
  } else {
    mc = C[k] + f * (C[k + 1] - C[k]);
    mp = P[k] + f * (P[k + 1] - P[k]);
  }
  mu_tot = mc + mp;
  mu_pe = mp;
}

// Binary search for E_k <= E < E_{k+1}, lin-lin interpolation, clamped at the ends.
__device__ __forceinline__ void mu_lookup(const DGeom &G, int mat, double E, double &mu_tot, double &mu_pe) {
  const int off = G.mat_off[mat], n = G.mat_n[mat];
  int k;
  double f;
  energy_bin(G.matE + off, n, E, k, f);
  mu_at(G, mat, k, f, mu_tot, mu_pe);
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

// The two 53-bit integers of one Philox block (counter (draw, id lo, id hi, stream)): the
// uniforms in (0, 1] are a 2^-53 (from x1:x0) and b 2^-53 (from x3:x2).  A draw site takes
// whole blocks; a single uniform uses a.  Out of line: its ~100 instructions would otherwise
// be repeated at each of the draw sites of the transport kernel.
struct M53x2 {
  uint64_t a, b;
};

__device__ __noinline__ M53x2 philox_m53_pair(uint64_t seed, int64_t tid, uint32_t stream, uint32_t &draw) {
  const uint4 x = philox4x32_10(make_uint4(draw++, (uint32_t)(uint64_t)tid, (uint32_t)((uint64_t)tid >> 32), stream),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint64_t wa = ((uint64_t)x.y << 32) | x.x, wb = ((uint64_t)x.w << 32) | x.z;
  return M53x2{(wa >> 11) + 1, (wb >> 11) + 1};
}

__device__ __forceinline__ uint64_t philox_m53(uint64_t seed, int64_t tid, uint32_t stream, uint32_t &draw) {
  return philox_m53_pair(seed, tid, stream, draw).a;
}

__device__ __forceinline__ double m53_double(uint64_t m) { return (double)m * 0x1.0p-53; }

// m 2^-53 as a float, truncated to 24 bits (relative error < 2^-23), with integer
// instructions only (m in [1, 2^53]).
__device__ __forceinline__ float m53_float(uint64_t m) {
  const int lz = __clzll((long long)m);                 // 11 .. 63
  const int sh = 40 - lz;                               // keep the leading one and 23 bits below it
  const uint32_t mant = sh >= 0 ? (uint32_t)(m >> sh) : (uint32_t)(m << (-sh));
  return __uint_as_float(((uint32_t)(63 - lz - 53 + 127) << 23) | (mant & 0x7FFFFFu));
}

// Uniform in (0, 1] from one Philox block.
__device__ __forceinline__ double philox_uniform(uint64_t seed, int64_t tid, uint32_t stream, uint32_t &draw) {
  return m53_double(philox_m53(seed, tid, stream, draw));
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
