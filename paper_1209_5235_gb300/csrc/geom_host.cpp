// geom_host.cpp -- context, geometry construction, validation, smart voxels and
// upload for libg4nav (host code, C++17).
//
// The geometry model is Geant4's (Sec. 3.2): a hierarchy of placed solids; each
// placement here is a distinct volume.  Navigation needs, per mother volume, a
// way to find the few daughters worth testing; like Geant4's smart voxels this
// slices the mother's extent along one axis, lists the daughters overlapping
// each slice, merges equal neighbouring slices into one node and refines crowded
// nodes along a further axis.  The lists are conservative (daughter extents are
// padded), so every navigation result equals the brute-force one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <map>
#include <random>

#include "g4n_internal.h"

using namespace g4n;

int g4n_fail(g4n_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define G4N_CUDA_TRY(call, what)                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return g4n_fail(ctx, e_ == cudaErrorMemoryAllocation ? G4N_ERR_OOM : G4N_ERR_CUDA,   \
                      std::string(what) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

namespace {

constexpr int kMaxGeoms = 4096;
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct Box3 {
  double lo[3], hi[3];
};

// Tight extent of a solid in its own frame, rotated by (c, s) about z and shifted by t.
Box3 solid_extent(const HSolid &so, double c, double s, const double *t) {
  Box3 b;
  if (so.kind == kBox) {
    double ex = std::fabs(c) * so.a + std::fabs(s) * so.b;
    double ey = std::fabs(s) * so.a + std::fabs(c) * so.b;
    b = {{-ex, -ey, -so.c}, {ex, ey, so.c}};
  } else if (so.kind == kOrb) {
    b = {{-so.a, -so.a, -so.a}, {so.a, so.a, so.a}};
  } else if (so.kind == kCone) {
    const double rmax = std::max(so.b, so.e);
    b = {{-rmax, -rmax, -so.c}, {rmax, rmax, so.c}};
  } else {
    double rmin = so.a, rmax = so.b;
    if (so.dphi >= kTwoPi - 1e-12) {
      b = {{-rmax, -rmax, -so.c}, {rmax, rmax, so.c}};
    } else {
      // phi range in the mother frame, starting in [0, 2 pi) so that axis angles 0 .. 4 pi cover it
      double th = std::atan2(s, c);
      double a0 = std::fmod(so.sphi + th, kTwoPi);
      if (a0 < 0.0) a0 += kTwoPi;
      const double a1 = a0 + so.dphi;
      double xs[16], ys[16];
      int n = 0;
      double ang[2] = {a0, a1};
      for (double a : ang) {
        xs[n] = rmax * std::cos(a); ys[n++] = rmax * std::sin(a);
        xs[n] = rmin * std::cos(a); ys[n++] = rmin * std::sin(a);
      }
      // axis directions inside the range (a0 < 2 pi, a1 < 4 pi)
      for (int k = 0; k <= 8; ++k) {
        const double a = k * (kTwoPi / 4.0);
        if (a > a0 && a < a1) { xs[n] = rmax * std::cos(a); ys[n++] = rmax * std::sin(a); }
      }
      b.lo[0] = b.hi[0] = xs[0];
      b.lo[1] = b.hi[1] = ys[0];
      for (int i = 1; i < n; ++i) {
        b.lo[0] = std::min(b.lo[0], xs[i]); b.hi[0] = std::max(b.hi[0], xs[i]);
        b.lo[1] = std::min(b.lo[1], ys[i]); b.hi[1] = std::max(b.hi[1], ys[i]);
      }
      if (rmin == 0.0) {
        b.lo[0] = std::min(b.lo[0], 0.0); b.hi[0] = std::max(b.hi[0], 0.0);
        b.lo[1] = std::min(b.lo[1], 0.0); b.hi[1] = std::max(b.hi[1], 0.0);
      }
      b.lo[2] = -so.c;
      b.hi[2] = so.c;
    }
  }
  for (int i = 0; i < 3; ++i) { b.lo[i] += t[i]; b.hi[i] += t[i]; }
  return b;
}

// Signed outside-ness (> 0 outside, < 0 inside) of a local point; used only for validation.
double solid_outside(const HSolid &so, const double *p) {
  if (so.kind == kBox) {
    return std::max({std::fabs(p[0]) - so.a, std::fabs(p[1]) - so.b, std::fabs(p[2]) - so.c});
  }
  if (so.kind == kOrb) return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]) - so.a;
  if (so.kind == kCone) {
    const double r = std::hypot(p[0], p[1]), f = (p[2] + so.c) / (2.0 * so.c);
    double m = std::max(std::fabs(p[2]) - so.c, r - (so.b + (so.e - so.b) * f));
    if (so.a > 0.0) m = std::max(m, so.a + (so.d - so.a) * f - r);
    return m;
  }
  double r = std::hypot(p[0], p[1]);
  double m = std::max(r - so.b, std::fabs(p[2]) - so.c);
  if (so.a > 0.0) m = std::max(m, so.a - r);
  if (so.dphi < kTwoPi - 1e-12) {
    double cs = std::cos(so.sphi), ss = std::sin(so.sphi);
    double ce = std::cos(so.sphi + so.dphi), se = std::sin(so.sphi + so.dphi);
    double a = -(cs * p[1] - ss * p[0]), bb = -(se * p[0] - ce * p[1]);
    m = std::max(m, so.dphi > M_PI ? std::min(a, bb) : std::max(a, bb));
  }
  return m;
}

// Points on the surface of a solid (local frame), for the containment check.
void surface_samples(const HSolid &so, std::mt19937_64 &rng, int n, std::vector<double> &out) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  out.clear();
  for (int i = 0; i < n; ++i) {
    double p[3];
    if (so.kind == kBox) {
      double h[3] = {so.a, so.b, so.c};
      int f = i % 6;
      for (int k = 0; k < 3; ++k) p[k] = (2.0 * U(rng) - 1.0) * h[k];
      p[f / 2] = (f % 2 ? -1.0 : 1.0) * h[f / 2];
    } else if (so.kind == kOrb) {
      double z = 2.0 * U(rng) - 1.0, ph = kTwoPi * U(rng), st = std::sqrt(std::max(0.0, 1.0 - z * z));
      p[0] = so.a * st * std::cos(ph); p[1] = so.a * st * std::sin(ph); p[2] = so.a * z;
    } else if (so.kind == kCone) {
      // outer surface, inner surface, end faces
      const int f = i % 4;
      const double ph = kTwoPi * U(rng);
      double z = (2.0 * U(rng) - 1.0) * so.c;
      if (f == 2) z = (i % 8 < 4) ? so.c : -so.c;
      const double fr = (z + so.c) / (2.0 * so.c);
      const double ro = so.b + (so.e - so.b) * fr, ri = so.a + (so.d - so.a) * fr;
      const double r = f == 0 ? ro : (f == 1 ? ri : ri + (ro - ri) * U(rng));
      p[0] = r * std::cos(ph); p[1] = r * std::sin(ph); p[2] = z;
    } else {
      int f = i % 4;
      double ph = so.sphi + so.dphi * (f == 3 ? (i % 8 < 4 ? 0.0 : 1.0) : U(rng));
      double r = f == 0 ? so.b : (f == 1 ? so.a : so.a + (so.b - so.a) * U(rng));
      double z = f == 2 ? ((i % 8 < 4) ? so.c : -so.c) : (2.0 * U(rng) - 1.0) * so.c;
      p[0] = r * std::cos(ph); p[1] = r * std::sin(ph); p[2] = z;
    }
    out.insert(out.end(), p, p + 3);
  }
}

void interior_samples(const HSolid &so, std::mt19937_64 &rng, int n, double margin, std::vector<double> &out) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double t0[3] = {0, 0, 0};
  Box3 e = solid_extent(so, 1.0, 0.0, t0);
  out.clear();
  for (int tries = 0; tries < 64 * n && (int)out.size() < 3 * n; ++tries) {
    double p[3];
    for (int k = 0; k < 3; ++k) p[k] = e.lo[k] + (e.hi[k] - e.lo[k]) * U(rng);
    if (solid_outside(so, p) < -margin) out.insert(out.end(), p, p + 3);
  }
}

// local -> mother
void to_mother(const HPlace &pl, const double *l, double *m) {
  m[0] = pl.c * l[0] - pl.s * l[1] + pl.t[0];
  m[1] = pl.s * l[0] + pl.c * l[1] + pl.t[1];
  m[2] = l[2] + pl.t[2];
}

// mother -> local
void to_local(const HPlace &pl, const double *m, double *l) {
  double dx = m[0] - pl.t[0], dy = m[1] - pl.t[1];
  l[0] = pl.c * dx + pl.s * dy;
  l[1] = -pl.s * dx + pl.c * dy;
  l[2] = m[2] - pl.t[2];
}

// The floats nearest below and above x (both x when x is a float).
void float_enclose(double x, float &lo, float &hi) {
  const float f = (float)x;
  lo = (double)f > x ? std::nextafter(f, -HUGE_VALF) : f;
  hi = (double)f < x ? std::nextafter(f, HUGE_VALF) : f;
}

int smart_levels(const g4n_voxel_params &P) { return P.n_levels > 0 ? std::min(P.n_levels, kMaxLevels) : kMaxLevels; }

// Distance from the origin to the convex quadrilateral with corners (x[i], y[i]) in order (0 inside).
double origin_to_quad(const double *x, const double *y) {
  bool pos = true, neg = true;
  double d = HUGE_VAL;
  for (int i = 0; i < 4; ++i) {
    const int j = (i + 1) & 3;
    const double ex = x[j] - x[i], ey = y[j] - y[i];
    const double cr = ex * (-y[i]) - ey * (-x[i]);  // edge x (origin - corner)
    pos = pos && cr >= 0.0;
    neg = neg && cr <= 0.0;
    const double l2 = ex * ex + ey * ey;
    double t = l2 > 0.0 ? -(x[i] * ex + y[i] * ey) / l2 : 0.0;
    t = std::min(1.0, std::max(0.0, t));
    d = std::min(d, std::hypot(x[i] + t * ex, y[i] + t * ey));
  }
  return (pos || neg) ? 0.0 : d;
}

// Can the solid of placement pl, grown by m, reach into box R (the mother frame)?  False only when it
// certainly cannot.  A voxel node lists the daughters whose padded extent overlaps its slab; this test
// drops those whose extent box overlaps the slab but whose solid does not: concentric shells around a
// node away from their annulus, phi segments whose wedge misses the node, rotated boxes.  The lists
// stay conservative (every daughter within m of the node's region is kept).
bool may_overlap(const HSolid &so, const HPlace &pl, const Box3 &R, double m) {
  const double zh = so.kind == kOrb ? so.a : so.c;
  if (R.lo[2] - pl.t[2] > zh + m || R.hi[2] - pl.t[2] < -zh - m) return false;
  if (so.kind == kOrb) {
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double dd = std::max({R.lo[k] - pl.t[k], 0.0, pl.t[k] - R.hi[k]});
      d2 += dd * dd;
    }
    return d2 <= (so.a + m) * (so.a + m);
  }
  // the region's rectangle in the solid's frame
  double x[4], y[4];
  const double cxs[4] = {R.lo[0], R.hi[0], R.hi[0], R.lo[0]}, cys[4] = {R.lo[1], R.lo[1], R.hi[1], R.hi[1]};
  for (int i = 0; i < 4; ++i) {
    const double mm[3] = {cxs[i], cys[i], 0.0};
    double l[3];
    to_local(pl, mm, l);
    x[i] = l[0];
    y[i] = l[1];
  }
  if (so.kind == kBox) {
    const double xl = std::min({x[0], x[1], x[2], x[3]}), xh = std::max({x[0], x[1], x[2], x[3]});
    const double yl = std::min({y[0], y[1], y[2], y[3]}), yh = std::max({y[0], y[1], y[2], y[3]});
    return !(xl > so.a + m || xh < -so.a - m || yl > so.b + m || yh < -so.b - m);
  }
  const double rin = so.kind == kCone ? std::min(so.a, so.d) : so.a;
  const double rout = so.kind == kCone ? std::max(so.b, so.e) : so.b;
  double dmax = 0.0;
  for (int i = 0; i < 4; ++i) dmax = std::max(dmax, std::hypot(x[i], y[i]));
  if (origin_to_quad(x, y) > rout + m) return false;
  if (rin > 0.0 && dmax < rin - m) return false;
  if (so.kind == kTube && so.dphi < kTwoPi - 1e-12) {
    // signed distances to the lines of the phi planes, positive on the solid's side (a linear function
    // takes its maximum over the rectangle at a corner)
    const double cs = std::cos(so.sphi), ss = std::sin(so.sphi);
    const double ce = std::cos(so.sphi + so.dphi), se = std::sin(so.sphi + so.dphi);
    double ps = -HUGE_VAL, pe = -HUGE_VAL;
    for (int i = 0; i < 4; ++i) {
      ps = std::max(ps, cs * y[i] - ss * x[i]);
      pe = std::max(pe, se * x[i] - ce * y[i]);
    }
    if (so.dphi > M_PI ? (ps < -m && pe < -m) : (ps < -m || pe < -m)) return false;
  }
  return true;
}

struct VoxBuilder {
  HGeom &g;
  const g4n_voxel_params &P;
  const std::vector<Box3> &dbox;  // padded daughter extents in the mother frame
  const std::vector<HSolid> &solids;
  const std::vector<HPlace> &places;
  double margin;                  // the lists' padding plus rounding slack (may_overlap)
  std::map<std::vector<int32_t>, int32_t> list_ids;

  // The daughters of lst that may reach into region R.
  std::vector<int32_t> filter(const std::vector<int32_t> &lst, const Box3 &R) const {
    std::vector<int32_t> out;
    out.reserve(lst.size());
    for (int32_t d : lst)
      if (may_overlap(solids[places[d].solid], places[d], R, margin)) out.push_back(d);
    return out;
  }

  int32_t list_id(const std::vector<int32_t> &lst) {
    auto it = list_ids.find(lst);
    if (it != list_ids.end()) return it->second;
    int32_t id = (int32_t)g.clist.size();
    g.clist.push_back({(int32_t)g.cand.size(), (int32_t)lst.size()});
    g.cand.insert(g.cand.end(), lst.begin(), lst.end());
    list_ids.emplace(lst, id);
    return id;
  }

  static void slice_range(const Box3 &b, int axis, double lo, double w, int n, int &k0, int &k1) {
    k0 = (int)std::floor((b.lo[axis] - lo) / w);
    k1 = (int)std::floor((b.hi[axis] - lo) / w);
    k0 = std::max(0, std::min(n - 1, k0));
    k1 = std::max(0, std::min(n - 1, k1));
  }

  // region: the node's extent (slicing); freg: the same grown by the margin, where the node's points lie
  int32_t build(const Box3 &region, const Box3 &freg, const std::vector<int32_t> &D, int level, int used) {
    int axis = -1, n = 1;
    if (P.mode == 1) {
      axis = P.axes[level];
      n = std::max(1, P.slices[level]);
    } else if (P.mode == 2) {
      axis = 0;
      n = 1;
    } else {
      double best = 1e300;
      int nn = (int)std::max(1.0, std::min((double)P.max_slices, std::floor(P.smartless * (double)D.size())));
      for (int a = 0; a < 3; ++a) {
        if (used & (1 << a)) continue;
        double w = (region.hi[a] - region.lo[a]) / nn;
        if (!(w > 0.0)) continue;
        double tot = 0.0;
        for (int32_t d : D) {
          int k0, k1;
          slice_range(dbox[d], a, region.lo[a], w, nn, k0, k1);
          tot += k1 - k0 + 1;
        }
        if (tot / nn < best) { best = tot / nn; axis = a; n = nn; }
      }
      if (axis < 0) { axis = 0; n = 1; }
    }
    double w = (region.hi[axis] - region.lo[axis]) / n;
    if (!(w > 0.0)) { w = 1.0; n = 1; }
    int32_t h = (int32_t)g.hdr.size();
    int32_t base = (int32_t)g.slice.size();
    g.hdr.push_back({region.lo[axis], w, 1.0 / w, axis, n, base, 0, 0.f, 0.f});
    g.slice.resize(g.slice.size() + n);
    std::vector<std::vector<int32_t>> lists(n);
    for (int32_t d : D) {
      int k0, k1;
      slice_range(dbox[d], axis, region.lo[axis], w, n, k0, k1);
      for (int k = k0; k <= k1; ++k) lists[k].push_back(d);
    }
    // the slab of slice k (grown by the margin; the end slices keep the node's own bounds)
    auto slab = [&](int k0, int k1) {
      Box3 b = freg;
      if (k0 > 0) b.lo[axis] = region.lo[axis] + k0 * w - margin;
      if (k1 < n - 1) b.hi[axis] = region.lo[axis] + (k1 + 1) * w + margin;
      return b;
    };
    for (int k = 0; k < n; ++k) lists[k] = filter(lists[k], slab(k, k));
    int k = 0;
    while (k < n) {
      int k1 = k;
      while (k1 + 1 < n && lists[k1 + 1] == lists[k]) ++k1;
      const std::vector<int32_t> &lst = lists[k];
      bool refine = false;
      if (level + 1 < kMaxLevels && !lst.empty()) {
        if (P.mode == 1) refine = level + 1 < P.n_levels;
        else if (P.mode == 0) refine = (int)lst.size() > P.refine_above && level + 1 < smart_levels(P);
      }
      int used2 = used | (1 << axis);
      if (refine && P.mode == 0 && used2 == 7) refine = false;
      int32_t child;
      if (refine) {
        Box3 sub = region;
        sub.lo[axis] = region.lo[axis] + k * w;
        sub.hi[axis] = region.lo[axis] + (k1 + 1) * w;
        child = -(build(sub, slab(k, k1), lst, level + 1, used2) + 1);
      } else {
        child = list_id(lst);
      }
      for (int q = k; q <= k1; ++q) g.slice[base + q] = {child, (int16_t)k, (int16_t)k1};
      k = k1 + 1;
    }
    return h;
  }
};

// ---------------------------------------------------------------- exact coordinate keys
// key(x): the bit pattern of a double as a signed integer with the negative half
// reflected, so that x < y <=> key(x) < key(y) for all non-NaN doubles (-0 < +0).
// A predicate of a coordinate that is monotone in it is then answered exactly by
// one integer comparison against the key of its first true (or last true) point,
// found here by bisection over keys with the very IEEE operations the FP64 device
// code performs.
int64_t dkey(double x) {
  int64_t b;
  std::memcpy(&b, &x, 8);
  return b ^ ((b >> 63) & INT64_C(0x7FFFFFFFFFFFFFFF));
}

double dunkey(int64_t k) {
  const int64_t b = k ^ ((k >> 63) & INT64_C(0x7FFFFFFFFFFFFFFF));
  double x;
  std::memcpy(&x, &b, 8);
  return x;
}

// Smallest key in [lo, hi] where pred (false ... true over the keys) holds; hi + 1 if none.
template <class F>
int64_t first_true(int64_t lo, int64_t hi, F pred) {
  if (!pred(dunkey(hi))) return hi + 1;
  while (lo < hi) {
    const int64_t mid = (int64_t)((uint64_t)lo + (((uint64_t)hi - (uint64_t)lo) >> 1));
    if (pred(dunkey(mid))) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

const int64_t kKeyMin = dkey(-DBL_MAX), kKeyMax = dkey(DBL_MAX);

// The thresholds of a world-aligned box (centre t, half-lengths h) for the band half.
DKeyBox key_box(const double *t, const double *h, double half) {
  DKeyBox K;
  for (int a = 0; a < 3; ++a) {
    const double c = t[a], ha = h[a];
    auto g = [c, ha](double x) { return std::fabs(x - c) - ha; };
    const int64_t kc = dkey(c);
    // low side: last key <= key(c) where the predicate holds (it holds below a threshold)
    K.k[a][0] = first_true(kKeyMin, kc, [&](double x) { return !(g(x) > half); }) - 1;
    K.k[a][1] = first_true(kKeyMin, kc, [&](double x) { return !(g(x) >= -half); }) - 1;
    K.k[a][2] = first_true(kc, kKeyMax, [&](double x) { return g(x) >= -half; });
    K.k[a][3] = first_true(kc, kKeyMax, [&](double x) { return g(x) > half; });
  }
  return K;
}

// Slice keys of the header tree rooted at h, for a mother whose world translation is wt.
void key_headers(HGeom &g, int32_t h0, const double *wt) {
  std::vector<int32_t> todo{h0};
  std::vector<char> seen(g.hdr.size(), 0);
  while (!todo.empty()) {
    const int32_t h = todo.back();
    todo.pop_back();
    if (seen[h]) continue;
    seen[h] = 1;
    DVoxHdr &H = g.hdr[h];
    const double t = wt[H.axis], lo = H.lo, iw = H.inv_width;
    const int n = H.nslices;
    auto slice_at = [t, lo, iw, n](double x) {
      const double p = x - t;
      double f = std::floor((p - lo) * iw);
      f = std::fmin(std::fmax(f, 0.0), (double)(n - 1));
      return (int)f;
    };
    H.keyed = 1;
    H.lo_wf = (float)(t + lo);
    H.inv_wf = (float)iw;
    g.skey[H.slice_base] = INT64_MIN;
    for (int k = 1; k < n; ++k)
      g.skey[H.slice_base + k] = first_true(kKeyMin, kKeyMax, [&](double x) { return slice_at(x) >= k; });
    for (int k = 0; k < n; ++k)
      if (g.slice[H.slice_base + k].child < 0) todo.push_back(-g.slice[H.slice_base + k].child - 1);
  }
}

// ---------------------------------------------------------------- face relocation records
// Inside test of volume V for a whole region R (key intervals per axis) and every
// direction whose component on axis a has sign s (tangential components free):
// 1 / 0 when the device's test gives that answer at every point, -1 when it is not
// decided (the region straddles a threshold, a tangential band, or V is not a kKeyBox).
int region_inside(const HGeom &g, int V, const int64_t R[3][2], int a, int s) {
  if (!(g.vol[V].flags & kKeyBox)) return -1;
  const DKeyBox &K = g.kbox[V];
  for (int b = 0; b < 3; ++b)
    if (R[b][1] <= K.k[b][0] || R[b][0] >= K.k[b][3]) return 0;   // outside by more than the band on axis b
  int near = 0, high = 0;
  for (int b = 0; b < 3; ++b) {
    const int64_t lo = R[b][0], hi = R[b][1];
    if (lo > K.k[b][1] && hi < K.k[b][2]) continue;                 // inside by more than the band
    if (lo > K.k[b][0] && hi <= K.k[b][1]) { near |= 1 << b; continue; }
    if (lo >= K.k[b][2] && hi < K.k[b][3]) { near |= 1 << b; high |= 1 << b; continue; }
    return -1;
  }
  if (!near) return 1;
  for (int b = 0; b < 3; ++b) {
    if (!(near & (1 << b))) continue;
    if (b != a) return -1;                                           // depends on a free direction component
    if (((high >> b) & 1) == (s > 0)) return 0;                      // p_a v_a > 0: leaving V
  }
  return 1;
}

// Candidate lists of the voxel nodes of the tree at header h that overlap [lo, hi] (mother frame).
void vox_collect(const HGeom &g, int32_t h, const double *lo, const double *hi, std::vector<int32_t> &lists) {
  const DVoxHdr &H = g.hdr[h];
  const int n = H.nslices;
  long k0 = (long)std::floor((lo[H.axis] - H.lo) * H.inv_width) - 1;
  long k1 = (long)std::floor((hi[H.axis] - H.lo) * H.inv_width) + 1;
  k0 = std::max(0L, std::min((long)n - 1, k0));
  k1 = std::max(0L, std::min((long)n - 1, k1));
  for (long k = k0; k <= k1; ++k) {
    const int32_t c = g.slice[H.slice_base + k].child;
    if (c >= 0) lists.push_back(c);
    else vox_collect(g, -c - 1, lo, hi, lists);
  }
}

// The relocation after leaving kKeyBox volume L outward through face (a, s) for every point of
// region R, evaluated as the device does it (up through the mothers from L's, the left volume
// blocked; down through the daughters in id order); false if some test is not decided.
bool eval_face(const HGeom &g, const std::vector<Box3> &ext, int L, int a, int s, const int64_t R[3][2], int &out) {
  int blocked = L, V = g.vol[L].mother;
  while (V >= 0) {
    const int r = region_inside(g, V, R, a, s);
    if (r < 0) return false;
    if (r == 1) break;
    blocked = V;
    V = g.vol[V].mother;
  }
  if (V < 0) {
    out = -1;
    return true;
  }
  double rlo[3], rhi[3];
  for (int b = 0; b < 3; ++b) {
    rlo[b] = dunkey(R[b][0]);
    rhi[b] = dunkey(R[b][1]);
  }
  int cur = V;
  for (int lev = 0; lev < kDMax; ++lev) {
    const DVol &C = g.vol[cur];
    if (C.vox < 0) break;
    if (!(C.flags & kWorldAligned)) return false;
    const DWorld &w = g.wxf[cur];
    const double wt[3] = {w.tx, w.ty, w.tz};
    double lo[3], hi[3];
    for (int b = 0; b < 3; ++b) {
      const double sl = 1e-9 * (1.0 + std::fabs(rlo[b]) + std::fabs(wt[b]));
      lo[b] = rlo[b] - wt[b] - sl;
      hi[b] = rhi[b] - wt[b] + sl;
    }
    std::vector<int32_t> lists, cands;
    vox_collect(g, C.vox, lo, hi, lists);
    for (int32_t l : lists) {
      const DCandList &cl = g.clist[l];
      for (int32_t q = 0; q < cl.count; ++q) {
        const int32_t d = g.cand[cl.offset + q];
        bool hit = d != blocked;
        for (int b = 0; b < 3 && hit; ++b) hit = ext[d].hi[b] >= lo[b] && ext[d].lo[b] <= hi[b];
        if (hit) cands.push_back(d);
      }
    }
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    int found = -1;
    for (int32_t d : cands) {
      const int r = region_inside(g, d, R, a, s);
      if (r < 0) return false;
      if (r == 1) {
        found = d;
        break;
      }
    }
    if (found < 0) break;
    cur = found;
    blocked = -1;
  }
  out = cur;
  return true;
}

}  // namespace

extern "C" {

int g4n_create(g4n_ctx **ctx_out, int device) {
  if (!ctx_out) return G4N_ERR_ARG;
  *ctx_out = nullptr;
  g4n_ctx *ctx = new (std::nothrow) g4n_ctx();
  if (!ctx) return G4N_ERR_OOM;
  if (device == -1) {  // host-only context: builds and validates tables, never touches a GPU
    ctx->device = -1;
    *ctx_out = ctx;
    return G4N_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    delete ctx;
    return G4N_ERR_CUDA;
  }
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return G4N_ERR_CUDA; }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc((void **)&ctx->d_geoms, kMaxGeoms * sizeof(DGeom)) != cudaSuccess) { delete ctx; return G4N_ERR_OOM; }
  ctx->d_geoms_cap = kMaxGeoms;
  *ctx_out = ctx;
  return G4N_OK;
}

int g4n_destroy(g4n_ctx *ctx) {
  if (!ctx) return G4N_OK;
  if (ctx->device < 0) {
    for (HGeom *g : ctx->geoms) delete g;
    delete ctx;
    return G4N_OK;
  }
  cudaSetDevice(ctx->device);
  g4n_mlp_free(ctx);
  for (HGeom *g : ctx->geoms) {
    if (g) { cudaFree(g->blob); delete g; }
  }
  cudaFree(ctx->d_geoms);
  cudaFree(ctx->ws);
  cudaFree(ctx->items);
  cudaFree(ctx->d_stage);
  cudaFree(ctx->stage_q);
  for (void *p : ctx->retired) cudaFree(p);
  cudaFreeHost(ctx->h_stage);
  cudaFreeHost(ctx->stage_flag);
  for (void *e : ctx->stage_ev)
    if (e) cudaEventDestroy((cudaEvent_t)e);
  delete ctx;
  return G4N_OK;
}

const char *g4n_last_error(const g4n_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int g4n_set_tolerance_scale(g4n_ctx *ctx, double scale) {
  if (!ctx) return G4N_ERR_ARG;
  if (!(scale > 0.0 && std::isfinite(scale))) return g4n_fail(ctx, G4N_ERR_ARG, "tolerance scale must be positive");
  if (!ctx->b.solids.empty() || !ctx->geoms.empty())
    return g4n_fail(ctx, G4N_ERR_STATE, "tolerance scale must be set before the first solid");
  ctx->scale = scale;
  ctx->tol = 1e-9 * scale;
  ctx->half = 0.5 * ctx->tol;
  return G4N_OK;
}

int g4n_material_add(g4n_ctx *ctx, double density, int32_t n_e, const double *E, const double *mu_c, const double *mu_p,
                     int32_t *out_mat) {
  if (!ctx || !E || !mu_c || !mu_p || !out_mat) return g4n_fail(ctx, G4N_ERR_ARG, "material: null argument");
  if (n_e < 2 || n_e > 4096) return g4n_fail(ctx, G4N_ERR_ARG, "material: need 2..4096 table points");
  HMat m;
  m.rho = density;
  for (int i = 0; i < n_e; ++i) {
    if (!(std::isfinite(E[i]) && E[i] > 0.0 && std::isfinite(mu_c[i]) && mu_c[i] >= 0.0 && std::isfinite(mu_p[i]) &&
          mu_p[i] >= 0.0))
      return g4n_fail(ctx, G4N_ERR_ARG, "material: energies must be positive and coefficients finite, >= 0");
    if (i > 0 && !(E[i] > E[i - 1])) return g4n_fail(ctx, G4N_ERR_ARG, "material: energies must increase strictly");
  }
  m.E.assign(E, E + n_e);
  m.muC.assign(mu_c, mu_c + n_e);
  m.muP.assign(mu_p, mu_p + n_e);
  ctx->b.mats.push_back(std::move(m));
  *out_mat = (int32_t)ctx->b.mats.size() - 1;
  return G4N_OK;
}

static int add_solid(g4n_ctx *ctx, const HSolid &s, int32_t *out) {
  if (!out) return g4n_fail(ctx, G4N_ERR_ARG, "solid: null output");
  ctx->b.solids.push_back(s);
  *out = (int32_t)ctx->b.solids.size() - 1;
  return G4N_OK;
}

int g4n_solid_box(g4n_ctx *ctx, double hx, double hy, double hz, int32_t *out) {
  if (!ctx) return G4N_ERR_ARG;
  if (!(hx > ctx->tol && hy > ctx->tol && hz > ctx->tol && std::isfinite(hx + hy + hz)))
    return g4n_fail(ctx, G4N_ERR_ARG, "box: half-lengths must exceed the tolerance");
  return add_solid(ctx, {kBox, hx, hy, hz, 0.0, 0.0}, out);
}

int g4n_solid_tube(g4n_ctx *ctx, double rmin, double rmax, double hz, double sphi, double dphi, int32_t *out) {
  if (!ctx) return G4N_ERR_ARG;
  if (!(rmin >= 0.0 && (rmin == 0.0 || rmin > ctx->tol) && rmax > rmin + ctx->tol && hz > ctx->tol &&
        std::isfinite(rmax + hz + sphi + dphi)))
    return g4n_fail(ctx, G4N_ERR_ARG, "tube: need 0 <= rmin < rmax, hz > tolerance");
  if (!(dphi > 0.0 && dphi <= kTwoPi + 1e-12)) return g4n_fail(ctx, G4N_ERR_ARG, "tube: need 0 < dphi <= 2 pi");
  return add_solid(ctx, {kTube, rmin, rmax, hz, sphi, dphi}, out);
}

int g4n_solid_cone(g4n_ctx *ctx, double rmin1, double rmax1, double rmin2, double rmax2, double hz, int32_t *out) {
  if (!ctx) return G4N_ERR_ARG;
  if (!(hz > ctx->tol && rmax1 > rmin1 + ctx->tol && rmax2 > rmin2 + ctx->tol && rmin1 >= 0.0 && rmin2 >= 0.0 &&
        std::isfinite(rmax1 + rmax2 + hz)))
    return g4n_fail(ctx, G4N_ERR_ARG, "cone: need 0 <= rmin < rmax at both ends, hz > tolerance");
  if (!((rmin1 == 0.0 && rmin2 == 0.0) || (rmin1 > ctx->tol && rmin2 > ctx->tol)))
    return g4n_fail(ctx, G4N_ERR_ARG, "cone: rmin1 and rmin2 both 0 or both above the tolerance");
  return add_solid(ctx, {kCone, rmin1, rmax1, hz, 0.0, kTwoPi, rmin2, rmax2}, out);
}

int g4n_solid_orb(g4n_ctx *ctx, double r, int32_t *out) {
  if (!ctx) return G4N_ERR_ARG;
  if (!(r > ctx->tol && std::isfinite(r))) return g4n_fail(ctx, G4N_ERR_ARG, "orb: radius must exceed the tolerance");
  return add_solid(ctx, {kOrb, r, 0.0, 0.0, 0.0, 0.0}, out);
}

int g4n_place(g4n_ctx *ctx, int32_t mother, int32_t solid, int32_t mat, const double *t, const double *rot,
              int32_t *out_vol) {
  if (!ctx || !t || !out_vol) return g4n_fail(ctx, G4N_ERR_ARG, "place: null argument");
  auto &B = ctx->b;
  if (solid < 0 || solid >= (int32_t)B.solids.size()) return g4n_fail(ctx, G4N_ERR_ARG, "place: bad solid id");
  if (mat < 0 || mat >= (int32_t)B.mats.size()) return g4n_fail(ctx, G4N_ERR_ARG, "place: bad material id");
  if (B.places.empty() ? mother != -1 : (mother < 0 || mother >= (int32_t)B.places.size()))
    return g4n_fail(ctx, G4N_ERR_ARG, "place: the first placement is the world (mother -1), later ones need a placed mother");
  HPlace p;
  p.mother = mother; p.solid = solid; p.mat = mat;
  for (int i = 0; i < 3; ++i) {
    if (!std::isfinite(t[i])) return g4n_fail(ctx, G4N_ERR_ARG, "place: non-finite translation");
    p.t[i] = t[i];
  }
  p.c = rot ? rot[0] : 1.0;
  p.s = rot ? rot[1] : 0.0;
  if (!(std::fabs(p.c * p.c + p.s * p.s - 1.0) <= 1e-12)) return g4n_fail(ctx, G4N_ERR_ARG, "place: rotation (cos, sin) not unit");
  B.places.push_back(p);
  B.touch_lv.push_back(-1);
  B.touch_copy.push_back(-1);
  *out_vol = (int32_t)B.places.size() - 1;
  return G4N_OK;
}

// ---------------------------------------------------------------- logical volumes (reuse)

static bool read_placement(g4n_ctx *ctx, const double *t, const double *rot, double *tt, double *c, double *s,
                           const char *who) {
  for (int i = 0; i < 3; ++i) {
    if (!std::isfinite(t[i])) {
      g4n_fail(ctx, G4N_ERR_ARG, std::string(who) + ": non-finite translation");
      return false;
    }
    tt[i] = t[i];
  }
  *c = rot ? rot[0] : 1.0;
  *s = rot ? rot[1] : 0.0;
  if (!(std::fabs(*c * *c + *s * *s - 1.0) <= 1e-12)) {
    g4n_fail(ctx, G4N_ERR_ARG, std::string(who) + ": rotation (cos, sin) not unit");
    return false;
  }
  return true;
}

int g4n_logical_create(g4n_ctx *ctx, int32_t solid, int32_t mat, int32_t *out_lv) {
  if (!ctx || !out_lv) return g4n_fail(ctx, G4N_ERR_ARG, "logical_create: null argument");
  auto &B = ctx->b;
  if (solid < 0 || solid >= (int32_t)B.solids.size()) return g4n_fail(ctx, G4N_ERR_ARG, "logical_create: bad solid id");
  if (mat < 0 || mat >= (int32_t)B.mats.size()) return g4n_fail(ctx, G4N_ERR_ARG, "logical_create: bad material id");
  B.lvs.push_back({solid, mat, {}});
  *out_lv = (int32_t)B.lvs.size() - 1;
  return G4N_OK;
}

// Does logical volume `from` contain `target` anywhere in its subtree (or is it)?
static bool lv_reaches(const std::vector<HLogical> &lvs, int32_t from, int32_t target) {
  if (from == target) return true;
  for (const HLogDaughter &d : lvs[from].dau)
    if (lv_reaches(lvs, d.lv, target)) return true;
  return false;
}

int g4n_logical_add_daughter(g4n_ctx *ctx, int32_t mother_lv, int32_t daughter_lv, const double *t, const double *rot,
                             int32_t *out_copy) {
  if (!ctx || !t || !out_copy) return g4n_fail(ctx, G4N_ERR_ARG, "logical_add_daughter: null argument");
  auto &B = ctx->b;
  const int32_t n = (int32_t)B.lvs.size();
  if (mother_lv < 0 || mother_lv >= n || daughter_lv < 0 || daughter_lv >= n)
    return g4n_fail(ctx, G4N_ERR_ARG, "logical_add_daughter: bad logical volume id");
  if (lv_reaches(B.lvs, daughter_lv, mother_lv))
    return g4n_fail(ctx, G4N_ERR_ARG, "logical_add_daughter: a logical volume cannot contain itself");
  HLogDaughter d;
  d.lv = daughter_lv;
  if (!read_placement(ctx, t, rot, d.t, &d.c, &d.s, "logical_add_daughter")) return G4N_ERR_ARG;
  B.lvs[mother_lv].dau.push_back(d);
  *out_copy = (int32_t)B.lvs[mother_lv].dau.size() - 1;
  return G4N_OK;
}

// Expand logical volume lv placed in physical volume `mother` (depth first: the volume, then each
// daughter's subtree in order); returns false after g4n_fail on a depth overflow.
static bool expand_logical(g4n_ctx *ctx, int32_t mother, int32_t lv, int32_t copy, const double *t, double c, double s,
                           int level) {
  auto &B = ctx->b;
  if (level >= kDMax) {
    g4n_fail(ctx, G4N_ERR_GEOM, "place_logical: expansion deeper than G4N_DMAX");
    return false;
  }
  HPlace p;
  p.mother = mother;
  p.solid = B.lvs[lv].solid;
  p.mat = B.lvs[lv].mat;
  for (int i = 0; i < 3; ++i) p.t[i] = t[i];
  p.c = c;
  p.s = s;
  B.places.push_back(p);
  B.touch_lv.push_back(lv);
  B.touch_copy.push_back(copy);
  const int32_t me = (int32_t)B.places.size() - 1;
  const std::vector<HLogDaughter> dau = B.lvs[lv].dau;  // copy: B.places grows below
  for (size_t k = 0; k < dau.size(); ++k)
    if (!expand_logical(ctx, me, dau[k].lv, (int32_t)k, dau[k].t, dau[k].c, dau[k].s, level + 1)) return false;
  return true;
}

int g4n_place_logical(g4n_ctx *ctx, int32_t mother, int32_t lv, const double *t, const double *rot,
                      int32_t *out_first_vol, int32_t *out_n_vols) {
  if (!ctx || !t || !out_first_vol || !out_n_vols) return g4n_fail(ctx, G4N_ERR_ARG, "place_logical: null argument");
  auto &B = ctx->b;
  if (lv < 0 || lv >= (int32_t)B.lvs.size()) return g4n_fail(ctx, G4N_ERR_ARG, "place_logical: bad logical volume id");
  if (B.places.empty() ? mother != -1 : (mother < 0 || mother >= (int32_t)B.places.size()))
    return g4n_fail(ctx, G4N_ERR_ARG, "place_logical: the first placement is the world (mother -1), later ones need a placed mother");
  double tt[3], c, s;
  if (!read_placement(ctx, t, rot, tt, &c, &s, "place_logical")) return G4N_ERR_ARG;
  const size_t first = B.places.size();
  if (!expand_logical(ctx, mother, lv, 0, tt, c, s, 0)) {
    B.places.resize(first);
    B.touch_lv.resize(first);
    B.touch_copy.resize(first);
    return G4N_ERR_GEOM;
  }
  *out_first_vol = (int32_t)first;
  *out_n_vols = (int32_t)(B.places.size() - first);
  return G4N_OK;
}

int g4n_touchable(g4n_ctx *ctx, int32_t geom, int32_t vol, int32_t cap, int32_t *out_lv, int32_t *out_copy,
                  int32_t *out_depth) {
  if (!ctx || !out_depth || (cap > 0 && (!out_lv || !out_copy)) || cap < 0)
    return g4n_fail(ctx, G4N_ERR_ARG, "touchable: bad arguments");
  if (geom < 0 || geom >= (int32_t)ctx->geoms.size()) return g4n_fail(ctx, G4N_ERR_ARG, "touchable: bad geometry id");
  const HGeom *g = ctx->geoms[geom];
  if (vol < 0 || vol >= (int32_t)g->vol.size()) return g4n_fail(ctx, G4N_ERR_ARG, "touchable: bad volume id");
  const int depth = g->vol[vol].depth;
  *out_depth = depth;
  // the chain from the world (level 0) down to vol
  for (int32_t v = vol, k = depth - 1; v >= 0; v = g->vol[v].mother, --k) {
    if (k < cap) {
      out_lv[k] = g->touch_lv[v];
      out_copy[k] = g->touch_copy[v];
    }
  }
  return G4N_OK;
}

int g4n_voxelize(g4n_ctx *ctx, const g4n_voxel_params *p) {
  if (!ctx || !p) return g4n_fail(ctx, G4N_ERR_ARG, "voxelize: null argument");
  if (p->mode < 0 || p->mode > 2) return g4n_fail(ctx, G4N_ERR_ARG, "voxelize: mode must be 0, 1 or 2");
  if (p->mode == 1) {
    if (p->n_levels < 1 || p->n_levels > kMaxLevels) return g4n_fail(ctx, G4N_ERR_ARG, "voxelize: 1..3 fixed levels");
    int used = 0;
    for (int l = 0; l < p->n_levels; ++l) {
      if (p->axes[l] < 0 || p->axes[l] > 2 || (used & (1 << p->axes[l])) || p->slices[l] < 1 || p->slices[l] > 30000)
        return g4n_fail(ctx, G4N_ERR_ARG, "voxelize: fixed levels need distinct axes and 1..30000 slices");
      used |= 1 << p->axes[l];
    }
  }
  if (p->mode == 0 && !(p->smartless > 0.0 && p->max_slices >= 1 && p->max_slices <= 30000))
    return g4n_fail(ctx, G4N_ERR_ARG, "voxelize: smartless > 0, 1 <= max_slices <= 30000");
  ctx->b.vox = *p;
  ctx->b.vox_set = true;
  return G4N_OK;
}

static int finalize_impl(g4n_ctx *ctx, int32_t *out_geom);

int g4n_geom_finalize(g4n_ctx *ctx, int32_t *out_geom) {
  if (!ctx || !out_geom) return g4n_fail(ctx, G4N_ERR_ARG, "finalize: null argument");
  auto &B = ctx->b;
  const int n = (int)B.places.size();
  if (n == 0) return g4n_fail(ctx, G4N_ERR_STATE, "finalize: no volumes placed");
  if ((int)ctx->geoms.size() >= kMaxGeoms) return g4n_fail(ctx, G4N_ERR_ARG, "finalize: too many geometries");
  const double tol = ctx->tol;
  int rc = finalize_impl(ctx, out_geom);
  if (rc != G4N_OK) B.clear();  // a rejected geometry is discarded; the next placement starts a new world
  return rc;
}

static int finalize_impl(g4n_ctx *ctx, int32_t *out_geom) {
  auto &B = ctx->b;
  const int n = (int)B.places.size();
  const double tol = ctx->tol;
  HGeom *g = new HGeom();
  // --- volume table, depth, daughter counts, composed world transforms
  g->vol.resize(n);
  g->wxf.resize(n);
  std::vector<std::vector<int32_t>> dau(n);
  for (int i = 0; i < n; ++i) {
    const HPlace &pl = B.places[i];
    const HSolid &so = B.solids[pl.solid];
    DVol &v = g->vol[i];
    std::memset(&v, 0, sizeof(v));
    v.tx = pl.t[0]; v.ty = pl.t[1]; v.tz = pl.t[2]; v.c = pl.c; v.s = pl.s;
    v.kind = so.kind;
    v.mother = pl.mother;
    v.mat = pl.mat;
    v.vox = -1;
    if (so.kind == kBox) { v.p[0] = so.a; v.p[1] = so.b; v.p[2] = so.c; }
    else if (so.kind == kOrb) { v.p[0] = so.a; }
    else if (so.kind == kCone) {
      // R(z) = k z + c of the inner and outer surfaces, hz, cos of the half-opening angles
      const double ko = (so.e - so.b) / (2.0 * so.c), co = 0.5 * (so.b + so.e);
      const double ki = (so.d - so.a) / (2.0 * so.c), ci = 0.5 * (so.a + so.d);
      v.p[0] = ki; v.p[1] = ci; v.p[2] = ko; v.p[3] = co; v.p[4] = so.c;
      v.p[5] = 1.0 / std::sqrt(1.0 + ki * ki);
      v.p[6] = 1.0 / std::sqrt(1.0 + ko * ko);
      v.flags = so.a > 0.0 ? kHasRmin : 0;
    } else {
      v.p[0] = so.a; v.p[1] = so.b; v.p[2] = so.c;
      v.p[3] = std::cos(so.sphi); v.p[4] = std::sin(so.sphi);
      v.p[5] = std::cos(so.sphi + so.dphi); v.p[6] = std::sin(so.sphi + so.dphi);
      bool seg = so.dphi < kTwoPi - 1e-12;
      v.flags = (seg ? kSeg : 0) | (seg && so.dphi > M_PI ? kWide : 0) | (so.a > 0.0 ? kHasRmin : 0);
    }
    DWorld &w = g->wxf[i];
    std::memset(&w, 0, sizeof(w));
    if (pl.mother < 0) {
      v.depth = 1;
      w.tx = pl.t[0]; w.ty = pl.t[1]; w.tz = pl.t[2]; w.c = pl.c; w.s = pl.s;
    } else {
      const DVol &m = g->vol[pl.mother];
      const DWorld &mw = g->wxf[pl.mother];
      v.depth = m.depth + 1;
      w.c = mw.c * pl.c - mw.s * pl.s;
      w.s = mw.s * pl.c + mw.c * pl.s;
      w.tx = mw.tx + mw.c * pl.t[0] - mw.s * pl.t[1];
      w.ty = mw.ty + mw.s * pl.t[0] + mw.c * pl.t[1];
      w.tz = mw.tz + pl.t[2];
      dau[pl.mother].push_back(i);
      g->vol[pl.mother].n_dau++;
    }
    if (w.c == 1.0 && w.s == 0.0) v.flags |= kWorldAligned;
    if (pl.c == 1.0 && pl.s == 0.0) v.flags |= kPlacedAligned;
    if (v.depth > kDMax) {
      delete g;
      return g4n_fail(ctx, G4N_ERR_GEOM, "finalize: hierarchy deeper than G4N_DMAX at volume " + std::to_string(i));
    }
    g->max_depth = std::max(g->max_depth, v.depth);
  }
  // --- padded daughter extents in their mother's frame
  const double pad = 4.0 * tol;
  std::vector<Box3> ext(n);
  std::vector<DBox32> &box = g->box;
  box.resize(n);
  for (int i = 0; i < n; ++i) {
    const HPlace &pl = B.places[i];
    Box3 e = solid_extent(B.solids[pl.solid], pl.c, pl.s, pl.t);
    for (int k = 0; k < 3; ++k) {
      double sl = 1e-12 * (std::fabs(e.lo[k]) + std::fabs(e.hi[k]));
      e.lo[k] -= pad + sl;
      e.hi[k] += pad + sl;
      box[i].lo[k] = std::nextafter((float)e.lo[k], -INFINITY);
      box[i].hi[k] = std::nextafter((float)e.hi[k], INFINITY);
      if ((double)box[i].lo[k] > e.lo[k]) box[i].lo[k] = std::nextafter(box[i].lo[k], -INFINITY);
      if ((double)box[i].hi[k] < e.hi[k]) box[i].hi[k] = std::nextafter(box[i].hi[k], INFINITY);
    }
    box[i].keyed = 0;
    box[i].pad = 0.f;
    ext[i] = e;
  }
  // --- FP32 copies for the conservative bounds
  g->v32.resize(n);
  for (int i = 0; i < n; ++i) {
    const DVol &v = g->vol[i];
    DVol32 &w = g->v32[i];
    std::memset(&w, 0, sizeof(w));
    w.tx = (float)v.tx; w.ty = (float)v.ty; w.tz = (float)v.tz; w.c = (float)v.c; w.s = (float)v.s;
    w.q0 = (float)v.p[0]; w.q1 = (float)v.p[1]; w.q2 = (float)v.p[2];
    w.kind = v.kind;
    w.flags = v.flags;
    if (v.kind == kCone) {
      // the bounding tube: the distance to it bounds the distance to the cone from below
      const HSolid &so = B.solids[B.places[i].solid];
      w.q0 = (float)std::min(so.a, so.d);
      w.q1 = (float)std::max(so.b, so.e);
      w.q2 = (float)so.c;
    }
    const double ext = v.kind == kOrb ? v.p[0]
                       : v.kind == kTube ? std::max(v.p[1], v.p[2])
                       : v.kind == kCone ? std::max({B.solids[B.places[i].solid].b, B.solids[B.places[i].solid].e, v.p[4]})
                                         : std::max({v.p[0], v.p[1], v.p[2]});
    w.scale = (float)(std::fabs(v.tx) + std::fabs(v.ty) + std::fabs(v.tz) + 2.0 * ext);
  }
  // --- validation: containment (surface samples) and sibling overlaps (interior samples)
  std::mt19937_64 rng(0x9E3779B97F4A7C15ull);
  std::vector<double> pts;
  const double slack = 10.0 * tol;
  for (int i = 1; i < n; ++i) {
    const HPlace &pl = B.places[i];
    const HPlace &mp = B.places[pl.mother];
    const HSolid &ms = B.solids[mp.solid];
    surface_samples(B.solids[pl.solid], rng, 48, pts);
    for (size_t q = 0; q < pts.size(); q += 3) {
      double m[3];
      to_mother(pl, &pts[q], m);
      double rel = 1e-12 * (std::fabs(m[0]) + std::fabs(m[1]) + std::fabs(m[2]));
      if (solid_outside(ms, m) > slack + rel) {
        delete g;
        return g4n_fail(ctx, G4N_ERR_GEOM, "finalize: volume " + std::to_string(i) + " sticks out of its mother " +
                                               std::to_string(pl.mother));
      }
    }
  }
  for (int m = 0; m < n; ++m) {
    std::vector<int32_t> &D = dau[m];
    if (D.size() < 2) continue;
    std::vector<int32_t> order(D);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return ext[a].lo[0] < ext[b].lo[0]; });
    for (size_t a = 0; a < order.size(); ++a) {
      int32_t da = order[a];
      for (size_t bq = a + 1; bq < order.size(); ++bq) {
        int32_t db = order[bq];
        if (ext[db].lo[0] >= ext[da].hi[0] - 2 * pad - slack) break;
        bool ov = true;
        for (int k = 0; k < 3; ++k)
          if (ext[da].hi[k] - ext[db].lo[k] <= 2 * pad + slack || ext[db].hi[k] - ext[da].lo[k] <= 2 * pad + slack) ov = false;
        if (!ov) continue;
        const HPlace &pa = B.places[da], &pb = B.places[db];
        interior_samples(B.solids[pa.solid], rng, 24, slack, pts);
        for (size_t q = 0; q < pts.size(); q += 3) {
          double mm[3], lb[3];
          to_mother(pa, &pts[q], mm);
          to_local(pb, mm, lb);
          if (solid_outside(B.solids[pb.solid], lb) < -slack) {
            delete g;
            return g4n_fail(ctx, G4N_ERR_GEOM, "finalize: volumes " + std::to_string(da) + " and " + std::to_string(db) +
                                                   " overlap");
          }
        }
      }
    }
  }
  // --- voxels
  g4n_voxel_params P = B.vox;
  if (!B.vox_set) { P.mode = 0; P.n_levels = 0; P.smartless = 2.0; P.max_slices = 1000; P.refine_above = 4; }
  for (int m = 0; m < n; ++m) {
    if (dau[m].empty()) continue;
    const HPlace &mp = B.places[m];
    double zero[3] = {0, 0, 0};
    Box3 region = solid_extent(B.solids[mp.solid], 1.0, 0.0, zero);
    double scale = 0.0;
    for (int k = 0; k < 3; ++k) scale = std::max({scale, std::fabs(region.lo[k]), std::fabs(region.hi[k])});
    const double margin = 2.0 * pad + 1e-10 * scale;
    Box3 freg = region;
    for (int k = 0; k < 3; ++k) {
      freg.lo[k] -= margin;
      freg.hi[k] += margin;
    }
    VoxBuilder vb{*g, P, ext, B.solids, B.places, margin, {}};
    g->vol[m].vox = vb.build(region, freg, vb.filter(dau[m], freg), 0, 0);
  }
  if (g->clist.empty()) g->clist.push_back({0, 0});
  if (g->cand.empty()) g->cand.push_back(-1);
  if (g->hdr.empty()) g->hdr.push_back({0, 1, 1, 0, 1, 0, 0, 0.f, 0.f});
  if (g->slice.empty()) g->slice.push_back({0, 0, 0});
  // --- materials
  for (const HMat &m : B.mats) {
    g->mat_off.push_back((int32_t)g->matE.size());
    g->mat_n.push_back((int32_t)m.E.size());
    g->matE.insert(g->matE.end(), m.E.begin(), m.E.end());
    g->matC.insert(g->matC.end(), m.muC.begin(), m.muC.end());
    g->matP.insert(g->matP.end(), m.muP.begin(), m.muP.end());
  }
  // --- exact coordinate keys: world-aligned boxes and the voxel slices of world-aligned mothers
  g->kbox.assign(n, DKeyBox{});
  g->skey.assign(g->slice.size(), INT64_MIN);
  const double half = 0.5 * tol;
  for (int i = 0; i < n; ++i) {
    DVol &v = g->vol[i];
    const DWorld &w = g->wxf[i];
    const double wt[3] = {w.tx, w.ty, w.tz};
    if (!(v.flags & kWorldAligned)) continue;
    if (v.kind == kBox && half >= 1e-15 && v.p[0] >= 4.0 * half && v.p[1] >= 4.0 * half && v.p[2] >= 4.0 * half) {
      g->kbox[i] = key_box(wt, v.p, half);
      v.flags |= kKeyBox;
      g->box[i].keyed = 1;
    }
    if (v.vox >= 0) key_headers(*g, v.vox, wt);
  }
  // --- face relocation records of kKeyBox volumes
  for (int i = 0; i < n; ++i) g->vol[i].face = -1;
  for (int i = 0; i < n; ++i) {
    DVol &v = g->vol[i];
    if (!(v.flags & kKeyBox) || v.mother < 0) continue;
    const DWorld &w = g->wxf[i];
    const double wt[3] = {w.tx, w.ty, w.tz};
    v.face = (int32_t)g->face.size();
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, s = (f & 1) ? 1 : -1;
      DFace F;
      std::memset(&F, 0, sizeof(F));
      F.leaf = -1;
      bool ok = true;
      for (int b = 0; b < 3; ++b) {
        if (b == a) {
          const double plane = wt[a] + s * v.p[a], d = 0.125 * tol;
          F.k[b][0] = dkey(plane - d);
          F.k[b][1] = dkey(plane + d);
        } else {
          const double m = 1e-6 + 1e-12 * (std::fabs(wt[b]) + v.p[b]);
          const double lo = wt[b] - v.p[b] + m, hi = wt[b] + v.p[b] - m;
          if (!(lo < hi)) ok = false;
          F.k[b][0] = dkey(lo);
          F.k[b][1] = dkey(hi);
        }
      }
      int leaf = -1;
      if (ok && eval_face(*g, ext, i, a, s, F.k, leaf)) {
        F.leaf = leaf;
        F.ok = 1;
      }
      g->face.push_back(F);
    }
  }
  if (g->face.empty()) g->face.push_back(DFace{});
  // --- touchables: the logical volume and copy number of every volume
  g->touch_lv = B.touch_lv;
  g->touch_copy = B.touch_copy;
  // --- FP32 copies of the voxel headers
  g->hdr32.resize(g->hdr.size());
  for (size_t h = 0; h < g->hdr.size(); ++h) {
    const DVoxHdr &H = g->hdr[h];
    DVoxHdr32 &F = g->hdr32[h];
    float_enclose(H.lo, F.lo_dn, F.lo_up);
    float_enclose(H.width, F.w_dn, F.w_up);
    float_enclose(H.inv_width, F.iw_dn, F.iw_up);
    F.slice_base = H.slice_base;
    F.n_axis = (H.nslices << 2) | H.axis;
  }
  // --- upload as one blob
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  constexpr int kTables = 17;
  size_t off[kTables], sz[kTables] = {g->vol.size() * sizeof(DVol), g->wxf.size() * sizeof(DWorld), g->box.size() * sizeof(DBox32),
                            g->hdr.size() * sizeof(DVoxHdr), g->slice.size() * sizeof(DVoxSlice),
                            g->clist.size() * sizeof(DCandList), g->cand.size() * sizeof(int32_t),
                            g->matE.size() * sizeof(double), g->matC.size() * sizeof(double), g->matP.size() * sizeof(double),
                            g->mat_off.size() * sizeof(int32_t), g->mat_n.size() * sizeof(int32_t),
                            g->v32.size() * sizeof(DVol32), g->kbox.size() * sizeof(DKeyBox),
                            g->skey.size() * sizeof(int64_t), g->face.size() * sizeof(DFace),
                            g->hdr32.size() * sizeof(DVoxHdr32)};
  const void *src[kTables] = {g->vol.data(), g->wxf.data(), g->box.data(), g->hdr.data(), g->slice.data(), g->clist.data(),
                         g->cand.data(), g->matE.data(), g->matC.data(), g->matP.data(), g->mat_off.data(), g->mat_n.data(),
                         g->v32.data(), g->kbox.data(), g->skey.data(), g->face.data(), g->hdr32.data()};
  size_t total = 0;
  for (int k = 0; k < kTables; ++k) { off[k] = total; total += al(std::max<size_t>(sz[k], 8)); }
  if (ctx->device < 0) {  // host-only context: keep the host tables
    g->blob_bytes = total;
    g->dview.n_vol = n;
    g->dview.n_mat = (int32_t)B.mats.size();
    g->dview.tol = tol;
    g->dview.half = 0.5 * tol;
    ctx->geoms.push_back(g);
    B.clear();
    *out_geom = (int32_t)ctx->geoms.size() - 1;
    return G4N_OK;
  }
  cudaSetDevice(ctx->device);
  if (cudaMalloc(&g->blob, total) != cudaSuccess) {
    delete g;
    return g4n_fail(ctx, G4N_ERR_OOM, "finalize: device allocation of the geometry tables failed");
  }
  g->blob_bytes = total;
  char *base = (char *)g->blob;
  for (int k = 0; k < kTables; ++k) {
    if (sz[k] && cudaMemcpy(base + off[k], src[k], sz[k], cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(g->blob);
      delete g;
      return g4n_fail(ctx, G4N_ERR_CUDA, "finalize: upload failed");
    }
  }
  DGeom &d = g->dview;
  d.vol = (const DVol *)(base + off[0]);
  d.wxf = (const DWorld *)(base + off[1]);
  d.box = (const DBox32 *)(base + off[2]);
  d.hdr = (const DVoxHdr *)(base + off[3]);
  d.hdr32 = (const DVoxHdr32 *)(base + off[16]);
  d.slice = (const DVoxSlice *)(base + off[4]);
  d.clist = (const DCandList *)(base + off[5]);
  d.cand = (const int32_t *)(base + off[6]);
  d.matE = (const double *)(base + off[7]);
  d.matC = (const double *)(base + off[8]);
  d.matP = (const double *)(base + off[9]);
  d.mat_off = (const int32_t *)(base + off[10]);
  d.mat_n = (const int32_t *)(base + off[11]);
  d.v32 = (const DVol32 *)(base + off[12]);
  d.kbox = (const DKeyBox *)(base + off[13]);
  d.skey = (const int64_t *)(base + off[14]);
  d.face = (const DFace *)(base + off[15]);
  d.n_vol = n;
  d.n_mat = (int32_t)B.mats.size();
  d.shared_grid = 1;
  for (const HMat &m : B.mats)
    if (m.E != B.mats[0].E) d.shared_grid = 0;
  d.tol = tol;
  d.half = 0.5 * tol;
  int32_t gid = (int32_t)ctx->geoms.size();
  if (cudaMemcpy(ctx->d_geoms + gid, &d, sizeof(DGeom), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(g->blob);
    delete g;
    return g4n_fail(ctx, G4N_ERR_CUDA, "finalize: directory upload failed");
  }
  ctx->geoms.push_back(g);
  B.clear();
  *out_geom = gid;
  return G4N_OK;
}

int g4n_geom_info(g4n_ctx *ctx, int32_t geom, int64_t *out8) {
  if (!ctx || !out8 || geom < 0 || geom >= (int32_t)ctx->geoms.size()) return g4n_fail(ctx, G4N_ERR_ARG, "geom_info: bad id");
  const HGeom *g = ctx->geoms[geom];
  out8[0] = (int64_t)g->vol.size();
  out8[1] = (int64_t)g->hdr.size();
  out8[2] = (int64_t)g->slice.size();
  out8[3] = (int64_t)g->clist.size();
  out8[4] = (int64_t)g->cand.size();
  out8[5] = (int64_t)g->blob_bytes;
  out8[6] = g->max_depth;
  out8[7] = (int64_t)g->mat_n.size();
  return G4N_OK;
}

}  // extern "C"
