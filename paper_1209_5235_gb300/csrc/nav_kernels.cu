// nav_kernels.cu -- sm_103a kernels and their C-ABI entry points: locate,
// compute_step and the persistent transport kernel (Algorithm 1 with Compton
// scattering, photoabsorption and energy deposits), plus g4n_sync.
//
// Transport design, two schedules over the same per-track device functions:
//  - persistent: one grid sized to fill every SM; each lane carries one track in
//    registers for its whole history.  A warp refills its idle lanes from one
//    global queue head with a single atomicAdd per refill (__ballot_sync/__popc),
//    so uneven history lengths and uneven geometries share one launch (the
//    periodic compaction/refill of Sec. 5, done per step in-warp).
//  - staged (transport_staged.cuh): the tracks in flight live in SoA queues in
//    HBM and advance in iterations of a step kernel and an interaction/source
//    kernel, each track queued by the solid kind of its leaf (the compaction of
//    Sec. 5 done every step, globally, by the queues themselves).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "g4n_internal.h"
#include "nav_device.cuh"

using namespace g4n;
using namespace g4n::dev;

namespace g4n {

// Device copy of one work item.
struct DItem {
  int32_t geom, pad;
  int64_t n, tid0, tally_off, start;
  double src[16];  // pos[3], sigma, has_z, z0, z1, iso, dir[3], e_kind, e0, e1, -
};

enum StatusBits : uint32_t { kStStepLimit = 1u, kStTimeout = 2u, kStRejection = 4u, kStBadInput = 8u };

struct Workspace {
  unsigned long long q_head;
  uint32_t status;
  uint32_t pad[13];
  dev::MlpLog log;        // training-sample log of g4n_mlp_log
  unsigned long long log_count;
  unsigned long long pad2[7];
};

}  // namespace g4n

namespace {

constexpr double kMeC2 = 0.51099895;
constexpr int kEvNone = 0, kEvPhoto = 1, kEvCompton = 2, kEvCutoff = 3, kEvEscape = 4, kEvPush = 5, kEvStepLimit = 6;
constexpr int kLimPush = -3, kLimStepLimit = -4;
constexpr uint64_t kFnvOffset = 0xcbf29ce484222325ull;

__device__ __forceinline__ bool bad_dir(const V3 &u) {
  const double n2 = u.x * u.x + u.y * u.y + u.z * u.z;
  return !(fabs(n2 - 1.0) <= 1e-6);
}

__device__ __forceinline__ void flag(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// Transport kernels with EV count once-per-track events (starts, ends, pushes, interactions) in
// shared memory, one array per block, so that the per-lane counter registers hold only the per-step
// counts (registers are what limits these kernels at 4 blocks per SM); the others count in registers.
__shared__ unsigned long long s_events[G4N_N_COUNTERS];
template <bool EV>
__device__ __forceinline__ void event(Counters &cnt, int k) {
  if (EV) atomicAdd(&s_events[k], 1ull);
  else cnt.c[k]++;
}

// ---------------------------------------------------------------- locate

// 8 blocks of 128 per SM (64 registers, a few hundred bytes of spills): the descent waits on its chain
// of dependent table loads, and more resident warps hide it (10^7 calorimeter queries: 6.3e9 -> 8.8e9 /s
// against 5 blocks at 96 registers; 10 to 16 blocks were slower again).
__global__ void __launch_bounds__(128, 8) k_locate(const DGeom *__restrict__ geoms, int gid, int64_t n,
                                                const double *__restrict__ pos, const double *__restrict__ dir,
                                                int32_t *__restrict__ out_depth, int32_t *__restrict__ out_path,
                                                uint32_t *status) {
  const DGeom &G = geoms[gid];
  Counters cnt;
  const int64_t lane = threadIdx.x & 31;
  // warp-uniform loop: the navigation below is warp-collective
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    V3 x{0, 0, 0}, u{0, 0, 1};
    bool ok = false;
    if (i < n) {
      x = V3{pos[i], pos[n + i], pos[2 * n + i]};
      u = V3{dir[i], dir[n + i], dir[2 * n + i]};
      ok = !bad_dir(u) && isfinite(x.x + x.y + x.z);
      if (!ok) flag(status, kStBadInput);
    }
    const int leaf = locate_world_warp<false>(G, ok, x, u, cnt);
    if (i < n) {
      const int depth = ok ? (leaf >= 0 ? G.vol[leaf].depth : 0) : -1;
      out_depth[i] = depth;
      int v = leaf;
      for (int k = kDMax - 1; k >= 0; --k) {
        if (k < depth) {
          out_path[k * n + i] = v;
          v = G.vol[v].mother;
        } else {
          out_path[k * n + i] = -1;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- compute_step

template <int MODE>
__global__ void __launch_bounds__(128) k_compute_step(const DGeom *__restrict__ geoms, int gid, int64_t n,
                                                      const double *__restrict__ pos, const double *__restrict__ dir,
                                                      const int32_t *__restrict__ depth, const int32_t *__restrict__ path,
                                                      const double *__restrict__ proposed, double *__restrict__ out_step,
                                                      double *__restrict__ out_safety, int32_t *__restrict__ out_lim,
                                                      uint32_t *status, const mlp::SmemWeights *__restrict__ mlp_w,
                                                      int walk_cap) {
  const DGeom &G = geoms[gid];
  Counters cnt;
  const int64_t lane = threadIdx.x & 31;
  MlpCtx mc{nullptr, nullptr, nullptr, 0.f};
  if (MODE == kLearned) {
    extern __shared__ __align__(16) unsigned char smem[];
    mlp::SmemWeights *sw = reinterpret_cast<mlp::SmemWeights *>(smem);
    mlp::load_weights(*sw, mlp_w);
    __syncthreads();
    mc.w = sw;
    mc.scratch = reinterpret_cast<mlp::SmemWarp *>(smem + sizeof(mlp::SmemWeights)) + (threadIdx.x >> 5);
    mc.loge = 0.46f;  // log-energy feature at 1 MeV: the query carries no energy
  }
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + lane;
    bool ok = false;
    int leaf = 0;
    double prop = kInf;
    V3 p{0, 0, 0}, v{0, 0, 1};
    if (i < n) {
      const V3 x{pos[i], pos[n + i], pos[2 * n + i]};
      const V3 u{dir[i], dir[n + i], dir[2 * n + i]};
      const int d = depth[i];
      leaf = (d >= 1 && d <= kDMax) ? path[(int64_t)(d - 1) * n + i] : -1;
      ok = !bad_dir(u) && leaf >= 0 && leaf < G.n_vol && G.vol[leaf].depth == d;
      if (!ok) {
        flag(status, kStBadInput);
        out_step[i] = nan("");
        out_safety[i] = nan("");
        out_lim[i] = INT32_MIN;
        leaf = 0;
      } else {
        prop = proposed ? proposed[i] : kInf;
        world_to_local(G.wxf[leaf], G.vol[leaf].flags & kWorldAligned, x, u, p, v);
      }
    }
    bool timeout = false;
    Chain ch;
    const StepResult R = geom_step_warp<MODE, false>(G, ok, leaf, p, v, inv_dir(v), prop, true, cnt, &timeout, walk_cap,
                                                     mc, ch);
    if (ok) {
      if (timeout) flag(status, kStTimeout);
      double s = R.step;
      int lim = R.lim;
      if (R.physics || prop < s) {
        s = prop;
        lim = G4N_LIM_PHYSICS;
      }
      out_step[i] = s;
      out_safety[i] = R.safety;
      out_lim[i] = lim;
    }
  }
}

// ---------------------------------------------------------------- transport

// Shared memory of the learned mode's weights and per-warp scratch (16-byte multiple).
__host__ __device__ __forceinline__ size_t mlp_block_bytes(unsigned block) {
  return (sizeof(mlp::SmemWeights) + (size_t)(block / 32) * sizeof(mlp::SmemWarp) + 15) & ~size_t(15);
}

enum Phase : int { kEmpty = 0, kStep = 1, kInteract = 2, kWalk = 3 };  // kWalk: a yielded boundary search

// Voxel nodes a boundary search walks per round before it yields (walk_budget = 0); budgets
// from kNeverYield on select the kernel without yielding.
constexpr int kDefaultWalkBudget = 16;
constexpr int kNeverYield = 1 << 16;

struct Track {
  V3 x, u;
  Inv3 iu;           // reciprocal of u (used in world-aligned volumes)
  double E, Y, len, safety, mu, mupe, efrac;
  uint64_t h;
  int64_t tid, gidx;
  int leaf, item, steps, nzero, ebin;
  uint32_t draw;
  WalkResume w;      // phase kWalk: the yielded boundary search of the current step
};

// The per-track history hash and path length are outputs: a launch that does not ask for
// them (out_hash / out_len null) does not compute them.
struct TParams {
  const DGeom *geoms;
  const DItem *items;
  int n_items;
  int64_t total;
  unsigned long long *q_head;
  uint32_t *status;
  uint64_t seed;
  double cutoff;
  int64_t max_steps;
  int nb;
  int64_t stride;
  double *edep;
  unsigned long long *counters;
  uint64_t *out_hash;
  double *out_len;
  int refill_min;    // refill a warp's idle lanes once at least this many are idle
  int interact_min;  // run the interaction phase once at least this many lanes wait for it
  int walk_budget;   // voxel nodes a boundary search walks per round before it yields
  int regroup;       // regrouping kernel: rounds between block-wide regroups of the tracks
  int walk_cap;      // voxel nodes a boundary search may walk (then G4N_ERR_TIMEOUT)
  int trial_cap;     // trials of a rejection sampler (then G4N_ERR_TIMEOUT)
  const mlp::SmemWeights *mlp_w;  // learned mode: weights (device image)
  const MlpLog *log;              // plain mode: training-sample log (null: none)
};

__device__ __forceinline__ int find_item(const DItem *items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].start <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Unit-disc rejection: (cos, sin) of a uniform azimuth, one Philox block per trial.  Points
// with a^2 + b^2 > 1 + 1e-5 in FP32 (from the Philox integers; error < 2e-6) are rejected
// without FP64 work; the others take the FP64 test and, if accepted, the FP64 evaluation.
__device__ __forceinline__ bool disc_azimuth(uint64_t seed, int64_t tid, uint32_t stream, uint32_t &draw, double &c,
                                             double &s, int trials) {
#pragma unroll 1
  for (int t = 0; t < trials; ++t) {
    const M53x2 ab = philox_m53_pair(seed, tid, stream, draw);
    const uint64_t ma = ab.a, mb = ab.b;
    const float af = 2.0f * m53_float(ma) - 1.0f, bf = 2.0f * m53_float(mb) - 1.0f;
    const float r2f = af * af + bf * bf;
    if (r2f > 1.0f + 1e-5f) continue;
    const double a = 2.0 * m53_double(ma) - 1.0;
    const double b = 2.0 * m53_double(mb) - 1.0;
    const double r2 = a * a + b * b;
    if (r2 > 0.0 && r2 <= 1.0) {
      const double inv = 1.0 / r2;
      c = (a * a - b * b) * inv;
      s = 2.0 * a * b * inv;
      return true;
    }
  }
  c = 1.0;
  s = 0.0;
  return false;
}

// Source of track tid (stream 0).
__device__ void make_source(const double *src, uint64_t seed, int64_t tid, V3 &x, V3 &u, double &E, uint32_t *status,
                            int trials) {
  uint32_t draw = 0;
  x = V3{src[0], src[1], src[2]};
  if (src[3] > 0.0) {
    bool ok = false;
#pragma unroll 1
    for (int t = 0; t < trials; ++t) {
      const M53x2 ab = philox_m53_pair(seed, tid, 0, draw);  // one block per trial
      const double a = 2.0 * m53_double(ab.a) - 1.0;
      const double b = 2.0 * m53_double(ab.b) - 1.0;
      const double s = a * a + b * b;
      if (s > 0.0 && s < 1.0) {
        const double f = sqrt(-2.0 * log(s) / s);
        x.x += src[3] * (a * f);
        x.y += src[3] * (b * f);
        ok = true;
        break;
      }
    }
    if (!ok) flag(status, kStRejection);
  }
  if (src[4] != 0.0) x.z = src[5] + (src[6] - src[5]) * philox_uniform(seed, tid, 0, draw);
  if (src[7] != 0.0) {
    const double ct = 2.0 * philox_uniform(seed, tid, 0, draw) - 1.0;
    double cph, sph;
    if (!disc_azimuth(seed, tid, 0, draw, cph, sph, trials)) flag(status, kStRejection);
    const double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
    u = V3{st * cph, st * sph, ct};
  } else {
    u = V3{src[8], src[9], src[10]};
  }
  const int ek = (int)src[11];
  if (ek == 0) E = src[12];
  else if (ek == 1) E = src[12] + (src[13] - src[12]) * philox_uniform(seed, tid, 0, draw);
  else E = src[12] * exp(philox_uniform(seed, tid, 0, draw) * log(src[13] / src[12]));
}

__device__ __forceinline__ void tally(const TParams &P, const Track &t, int col, double e) {
  const DItem &it = P.items[t.item];
  atomicAdd(&P.edep[(t.tid % P.nb) * P.stride + it.tally_off + col], e);
}

__device__ __forceinline__ void finish(const TParams &P, const Track &t) {
  if (P.out_hash) P.out_hash[t.gidx] = t.h;
  if (P.out_len) P.out_len[t.gidx] = t.len;
}

// Attenuation of the track's leaf at its energy (cached energy bin when all materials share a grid).
__device__ __forceinline__ void update_mu(const DGeom &G, Track &t) {
  if (G.shared_grid) mu_at(G, G.vol[t.leaf].mat, t.ebin, t.efrac, t.mu, t.mupe);
  else mu_lookup(G, G.vol[t.leaf].mat, t.E, t.mu, t.mupe);
}

__device__ __forceinline__ void set_energy(const DGeom &G, Track &t, double E) {
  t.E = E;
  if (G.shared_grid) energy_bin(G.matE, G.mat_n[0], E, t.ebin, t.efrac);
}

__device__ __forceinline__ void set_direction(Track &t, const V3 &u) {
  t.u = u;
  t.iu = inv_dir(u);
}

// Start track number g of the concatenated items on the lanes with `active` set
// (warp-collective: locate runs across the warp).  Returns the new phase of the
// lane: kStep, or kEmpty if the track ended at once (or the lane was not active).
template <int MODE, bool COUNT, bool EV>
__device__ int start_warp(const TParams &P, bool active, int64_t g, Track &t, Counters &cnt) {
  const DGeom *Gp = &P.geoms[P.items[0].geom];
  if (active) {
    t.gidx = g;
    t.item = find_item(P.items, P.n_items, g);
    const DItem &it = P.items[t.item];
    t.tid = it.tid0 + (g - it.start);
    Gp = &P.geoms[it.geom];
    V3 u;
    double E;
    make_source(it.src, P.seed, t.tid, t.x, u, E, P.status, P.trial_cap);
    set_direction(t, u);
    tally(P, t, Gp->n_vol + 1, E);
    event<EV>(cnt, G4N_C_TRACKS);
    t.h = kFnvOffset;
    t.len = 0.0;
    t.steps = 0;
    t.nzero = 0;
    t.safety = 0.0;
    t.E = E;
  }
  const DGeom &G = *Gp;
  const int leaf = locate_world_warp<COUNT, MODE != kFP64>(G, active, t.x, t.u, cnt);
  if (!active) return kEmpty;
  t.leaf = leaf;
  if (leaf < 0) {
    event<EV>(cnt, G4N_C_ESCAPED);
    tally(P, t, G.n_vol, t.E);
    if (P.out_hash) t.h = hash_step(t.h, -1, G4N_LIM_MOTHER, kEvEscape);
    finish(P, t);
    t.leaf = 0;
    return kEmpty;
  }
  t.draw = 0;
  t.Y = -log(philox_uniform(P.seed, t.tid, 1, t.draw));
  set_energy(G, t, t.E);
  update_mu(G, t);
  return kStep;
}

// Kahn's rejection method for the Klein-Nishina law of eta = E / E' (three uniforms per
// trial: r1, r2 from one Philox block, r3 from the next).  Each comparison of a uniform
// with its threshold is first made in FP32 and kept when they differ by more than 1e-5.  All three thresholds lie in [0, 1]; their FP32
// values (written without cancellation: 1 - (eta - 1) / alpha = 1 - 2 (1 - r2) / (1 + 2
// alpha r2)) and the uniforms' FP32 copies (built from the Philox integers, relative error
// < 2^-23) are within 2e-6 of the exact ones, so such a decision is the exact one; the
// others are taken on the FP64 thresholds of the plain formulas.  The accepted trial's eta
// and cos theta are computed in FP64.  FP64 work is left for the accepted trial and the
// rare close calls.
__device__ __forceinline__ bool kahn(double E, uint64_t seed, int64_t tid, uint32_t &draw, double &eta, double &cost,
                                     int trials) {
  constexpr float kMargin = 1e-5f;
  const double al = E / kMeC2;
  const float alf = (float)al;
  const float p1f = (1.0f + 2.0f * alf) / (9.0f + 2.0f * alf);
#pragma unroll 1
  for (int t = 0; t < trials; ++t) {
    const M53x2 b12 = philox_m53_pair(seed, tid, 1, draw);
    const uint64_t m1 = b12.a, m2 = b12.b;
    const uint64_t m3 = philox_m53(seed, tid, 1, draw);
    const float d1 = m53_float(m1) - p1f;
    const bool first = fabsf(d1) > kMargin ? d1 <= 0.f : m53_double(m1) <= (1.0 + 2.0 * al) / (9.0 + 2.0 * al);
    const float r2f = m53_float(m2), r3f = m53_float(m3);
    const float a2 = 2.0f * alf * r2f, den = 1.0f + a2;
    if (first) {
      const float d = r3f - 4.0f * a2 / (den * den);
      if (fabsf(d) > kMargin && d > 0.f) continue;
      eta = 1.0 + 2.0 * al * m53_double(m2);
      if (!(fabsf(d) > kMargin) && !(m53_double(m3) <= 4.0 * (1.0 / eta - 1.0 / (eta * eta)))) continue;
      cost = 1.0 - (eta - 1.0) / al;
    } else {
      const float cf = 1.0f - 2.0f * (1.0f - r2f) / den;
      const float d = r3f - 0.5f * (cf * cf + den / (1.0f + 2.0f * alf));
      if (fabsf(d) > kMargin && d > 0.f) continue;
      eta = (1.0 + 2.0 * al) / (1.0 + 2.0 * al * m53_double(m2));
      cost = 1.0 - (eta - 1.0) / al;
      if (!(fabsf(d) > kMargin) && !(m53_double(m3) <= 0.5 * (cost * cost + 1.0 / eta))) continue;
    }
    return true;
  }
  eta = 1.0;
  cost = 1.0;
  return false;
}

// New direction at polar cosine ct and azimuth (cph, sph) about u.
__device__ __forceinline__ V3 deflect(const V3 &u, double ct, double cph, double sph) {
  const double st = sqrt(fmax(0.0, (1.0 - ct) * (1.0 + ct)));
  const double dx = st * cph, dy = st * sph, dz = ct;
  const double perp2 = u.x * u.x + u.y * u.y;
  if (perp2 > 0.0) {
    const double perp = sqrt(perp2), ip = 1.0 / perp;
    const double nx = (u.x * u.z * dx - u.y * dy) * ip + u.x * dz;
    const double ny = (u.y * u.z * dx + u.x * dy) * ip + u.y * dz;
    const double nz = -perp * dx + u.z * dz;
    return V3{nx, ny, nz};
  }
  if (u.z >= 0.0) return V3{dx, dy, dz};
  return V3{dx, -dy, -dz};
}

// One transport step of Algorithm 1 on every lane in phase kStep
// (warp-collective): the free path (Eq. 7) races the geometric step; a boundary
// crossing relocates, a physics end point waits for the interaction phase.
// Returns the lane's next phase.
constexpr int kReloc = 4;  // staged schedule: the step is done, its relocation search is deferred (aux: limiter, left)

// The relocation after a geometric step (from the current leaf; `need`: the lanes that search, `leaf` the
// answer of the others), the push after ten zero steps, and the step record: the tail of step_warp, shared
// with the staged schedule's relocation kernel (update_nzero false there: the step kernel counted it).
template <int MODE, bool COUNT, bool EV>
__device__ __forceinline__ int reloc_tail(const TParams &P, const DGeom &G, Track &t, bool geo, bool need, int leaf,
                                          bool from_left, double s, int lim, bool update_nzero, Counters &cnt,
                                          int next) {
  bool pushing = false;
  int from = t.leaf;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int found = relocate_warp<MODE, COUNT>(G, need, need ? from : 0, t.x, t.u, from_left, cnt);
    if (need) leaf = found;
    need = false;
    if (pass == 0 && geo) {
      if (update_nzero) t.nzero = (dkey(s) <= dkey(G.half)) ? t.nzero + 1 : 0;
      if (leaf >= 0 && t.nzero >= 10) {
        const double push = 100.0 * G.tol;
        t.x.x += push * t.u.x;
        t.x.y += push * t.u.y;
        t.x.z += push * t.u.z;
        if (P.out_len) t.len += push;
        event<EV>(cnt, G4N_C_PUSHES);
        t.nzero = 0;
        pushing = need = true;
        from = leaf;
        from_left = false;
      }
    }
    if (!__any_sync(kFull, need)) break;
  }
  if (pushing && P.out_hash) t.h = hash_step(t.h, leaf, kLimPush, kEvPush);
  if (geo) {
    if (leaf < 0) {
      event<EV>(cnt, G4N_C_ESCAPED);
      tally(P, t, G.n_vol, t.E);
      if (P.out_hash) t.h = hash_step(t.h, -1, lim, kEvEscape);
      finish(P, t);
      next = kEmpty;
    } else {
      t.leaf = leaf;
      if (P.out_hash) t.h = hash_step(t.h, leaf, lim, kEvNone);
      update_mu(G, t);
      next = kStep;
    }
  }
  return next;
}

template <int MODE, bool COUNT, bool YIELD, bool EV, bool DEFER = false>
__device__ int step_warp(const TParams &P, Track &t, int phase, Counters &cnt, MlpCtx mc, Chain &wch,
                         int *aux = nullptr) {
  const bool resume = YIELD && phase == kWalk;  // continue the step's yielded boundary search
  bool act = phase == kStep || resume;
  const DGeom &G = P.geoms[P.items[act ? t.item : 0].geom];
  int next = phase;
  if (act && !resume && t.steps >= P.max_steps) {
    event<EV>(cnt, G4N_C_STEP_LIMIT);
    flag(P.status, kStStepLimit);
    if (P.out_hash) t.h = hash_step(t.h, t.leaf, kLimStepLimit, kEvStepLimit);
    finish(P, t);
    next = kEmpty;
    act = false;
  }
  // the free path s_phys = Y / mu (Eq. 7) races the geometric step; the division is only done
  // when its value is needed (physics wins, or a voxel walk / FP32 bound needs the limit)
  double sphys = kInf;
  bool need_geo = false;
  V3 p{0, 0, 0}, v{0, 0, 1};
  Inv3 iv{0, 0, 0};
  bool lazy = false;       // FP64 mode: sphys not computed, s * mu is compared with Y instead
  bool want_saf = true;    // FP64 mode, leaf without daughters: the safety is taken in the interaction phase
  double lim_geo = kInf;  // limit handed to the geometric step (an upper bound of sphys)
  if (act) {
    const DVol &L = G.vol[t.leaf];
    const bool mu_pos = nonzero_bits(t.mu);  // mu >= 0
    lazy = MODE == kFP64 && mu_pos && !mc.log;
    if (!lazy) sphys = mu_pos ? t.Y / t.mu : kInf;
    // a zero safety (after every boundary crossing) always needs the boundary search.  Lazy form: the
    // search is skipped only when Y - safety mu (one rounding, by the fma) lies below -2^-49 Y, so that
    // fl(Y / mu) < safety holds as well (the comparison the oracle makes)
    need_geo = resume || !nonzero_bits(t.safety) ||
               (lazy ? !(fma(-t.safety, t.mu, t.Y) < -0x1p-49 * t.Y) : !(sphys < t.safety));
    want_saf = !(MODE == kFP64 && L.vox < 0);
    if (!need_geo) {
      diag<COUNT>(cnt, G4N_C_SAFETY_SKIPS);
      if (lazy) sphys = t.Y / t.mu;
    } else {
      const bool aligned = L.flags & kWorldAligned;
      world_to_local(G.wxf[t.leaf], aligned, t.x, t.u, p, v);
      // the reciprocal direction serves the FP64 voxel walk and a box's exit; the FP32 modes walk in
      // FP32 (their rare FP64 node step forms it itself) and need it only in box leaves
      iv = aligned ? t.iu : ((MODE == kFP64 || L.kind == kBox) ? inv_dir(v) : Inv3{0.0, 0.0, 0.0});
      // the voxel walk may stop at any bound >= sphys: candidates found beyond sphys lose
      // to the physics step all the same
      lim_geo = !lazy ? sphys
                : L.vox < 0 ? kInf
                            : (double)__fdiv_ru(__double2float_ru(t.Y), __double2float_rd(t.mu));
    }
  }
  bool timeout = false;
  if (MODE == kLearned || mc.log) mc.loge = act ? (logf((float)t.E) + 4.6f) * 0.1f : 0.f;
  // the learned proposal and the sample log look at the first node only: no yielding there
  const int budget = (!YIELD || MODE == kLearned || mc.log) ? 0 : P.walk_budget;
  const StepResult R = geom_step_warp<MODE, COUNT>(G, need_geo, need_geo ? t.leaf : 0, p, v, iv, lim_geo, want_saf,
                                                   cnt, &timeout, P.walk_cap, mc, wch, resume, t.w, budget);
  if (act && R.yielded) {
    // the search used its node budget: the step continues in a later round
    t.w = R.resume;
    next = kWalk;
    act = false;
  }
  bool geo = false;
  double s = sphys;
  int lim = G4N_LIM_PHYSICS;
  if (act) {
    if (timeout) flag(P.status, kStTimeout);
    if (need_geo) {
      t.safety = R.safety;
      // geometry wins iff step <= fl(Y / mu).  Lazy form: Y - step mu (one rounding, by the fma) decides
      // when it lies outside +-2^-49 Y, a margin far above the rounding of either form; a near-tie takes
      // the division itself
      bool geo_first;
      if (!lazy) {
        geo_first = R.step <= sphys;
      } else {
        const double d = fma(-R.step, t.mu, t.Y), m = 0x1p-49 * t.Y;
        geo_first = d > m || (!(d < -m) && R.step <= t.Y / t.mu);
      }
      if (!R.physics && geo_first) {
        geo = true;
        s = R.step;
        lim = R.lim;
      } else if (lazy) {
        s = sphys = t.Y / t.mu;
      }
    }
    ++t.steps;
    if (!EV) cnt.c[G4N_C_STEPS]++;  // EV: the sum of the geometry- and physics-limited counts
    t.x.x += s * t.u.x;
    t.x.y += s * t.u.y;
    t.x.z += s * t.u.z;
    if (P.out_len) t.len += s;
    if (!geo) {
      // free path ends inside the volume: the interaction is done in the interaction phase
      t.safety = fmax(t.safety - s, 0.0);
      t.nzero = 0;
      cnt.c[G4N_C_PHYS_STEPS]++;
      next = kInteract;
    } else {
      if (nonzero_bits(t.mu)) t.Y = fmax(t.Y - s * t.mu, 0.0);
      cnt.c[G4N_C_GEOM_STEPS]++;
      t.safety = 0.0;
    }
  }
  // leaving a box through a face whose relocation is tabulated needs no search
  int leaf = -1;
  const bool left = geo && lim == G4N_LIM_MOTHER && s > 0.0;
  const bool fast = left && face_relocate(G, t.leaf, R.face, t.x, t.u, &leaf);
  if (fast) diag<COUNT>(cnt, G4N_C_FACE_RELOC);
  // relocation search, then (after 10 zero steps) the push and its relocation: one copy of
  // the relocation code serves both passes.  DEFER: a lane that needs the search stops here (its
  // zero-step count updated) and goes to the relocation queue with its limiter and exit flag.
  bool defer = false;
  if (DEFER && geo && !fast) {
    defer = true;
    t.nzero = (dkey(s) <= dkey(G.half)) ? t.nzero + 1 : 0;
    *aux = (lim << 1) | (left ? 1 : 0);
  }
  next = reloc_tail<MODE, COUNT, EV>(P, G, t, geo && !defer, !DEFER && geo && !fast, leaf, left, s, lim, true, cnt,
                                     next);
  return defer ? kReloc : next;
}

// The interaction at the end of a free path: photoabsorption if U mu_tot < mu_photo,
// else a Compton scatter (Kahn), the cutoff, and a new Y = -log W.
template <int MODE, bool EV>
__device__ int interact(const TParams &P, Track &t, Counters &cnt) {
  const DItem &it = P.items[t.item];
  const DGeom &G = P.geoms[it.geom];
  // one block per interaction: U chooses the process, W gives the next free path
  const M53x2 uw = philox_m53_pair(P.seed, t.tid, 1, t.draw);
  const double U = m53_double(uw.a);
  if (U * t.mu < t.mupe) {
    event<EV>(cnt, G4N_C_PHOTO);
    tally(P, t, t.leaf, t.E);
    if (P.out_hash) t.h = hash_step(t.h, t.leaf, G4N_LIM_PHYSICS, kEvPhoto);
    finish(P, t);
    return kEmpty;
  }
  event<EV>(cnt, G4N_C_COMPTON);
  double eta, cost, cph, sph;
  bool ok = kahn(t.E, P.seed, t.tid, t.draw, eta, cost, P.trial_cap);
  ok &= disc_azimuth(P.seed, t.tid, 1, t.draw, cph, sph, P.trial_cap);
  if (!ok) flag(P.status, kStRejection);
  set_direction(t, deflect(t.u, cost, cph, sph));
  const double E1 = t.E / eta;
  if (E1 < P.cutoff) {
    event<EV>(cnt, G4N_C_CUTOFF);
    tally(P, t, t.leaf, t.E);
    if (P.out_hash) t.h = hash_step(t.h, t.leaf, G4N_LIM_PHYSICS, kEvCutoff);
    finish(P, t);
    return kEmpty;
  }
  tally(P, t, t.leaf, t.E - E1);
  set_energy(G, t, E1);
  t.Y = -log(m53_double(uw.b));
  if (P.out_hash) t.h = hash_step(t.h, t.leaf, G4N_LIM_PHYSICS, kEvCompton);
  update_mu(G, t);
  // FP64 mode: the isotropic safety of a leaf without daughters, at the interaction point
  // (the step phase does not compute it there; a safety only lets the next step skip a
  // boundary search whose answer could not win).  The FP32 modes keep their FP32 bound.
  const DVol &L = G.vol[t.leaf];
  if (MODE == kFP64 && L.vox < 0) {
    V3 p, v;
    world_to_local(G.wxf[t.leaf], L.flags & kWorldAligned, t.x, t.u, p, v);
    t.safety = fmax(t.safety, vol_safety_out(L, p));
  }
  return kStep;
}

// ---------------------------------------------------------------- regrouping between rounds
// The alternative divergence cure: every P.regroup rounds the block's tracks are sorted by
// (phase, solid kind of the leaf) and dealt out again, so that each warp holds tracks that
// run the same code (the interaction phase, boxes, tubes, orbs, yielded searches; idle lanes
// together, which then refill a whole warp at once).  A track's state moves through shared
// memory as 32-bit words, one array per word (consecutive slots: no bank conflicts on the
// way back).  Histories do not depend on which lane carries them.

constexpr int kTrackWords = 62;  // Track (50 words), phase (1), voxel chain (11)

__device__ __forceinline__ int regroup_key(const TParams &P, const Track &t, int phase) {
  if (phase == kEmpty) return 0;
  const int kind = P.geoms[P.items[t.item].geom].vol[t.leaf].kind;  // box, tube, orb, cone
  return phase == kStep ? 1 + kind : (phase == kWalk ? 5 + kind : 9 + kind);
}
constexpr int kRegroupKeys = 13;

struct WordIO {
  uint32_t *S;
  int stride, slot, k;
  __device__ __forceinline__ void put(uint32_t w) { S[(k++) * stride + slot] = w; }
  __device__ __forceinline__ uint32_t get() { return S[(k++) * stride + slot]; }
  __device__ __forceinline__ void putd(double d) {
    put((uint32_t)__double2loint(d));
    put((uint32_t)__double2hiint(d));
  }
  __device__ __forceinline__ double getd() {
    const uint32_t lo = get(), hi = get();
    return __hiloint2double((int)hi, (int)lo);
  }
  __device__ __forceinline__ void putl(uint64_t l) {
    put((uint32_t)l);
    put((uint32_t)(l >> 32));
  }
  __device__ __forceinline__ uint64_t getl() {
    const uint64_t lo = get(), hi = get();
    return lo | (hi << 32);
  }
};

__device__ __forceinline__ void put_track(WordIO &io, const Track &t, int phase, const Chain &ch) {
  io.putd(t.x.x); io.putd(t.x.y); io.putd(t.x.z);
  io.putd(t.u.x); io.putd(t.u.y); io.putd(t.u.z);
  io.putd(t.iu.x); io.putd(t.iu.y); io.putd(t.iu.z);
  io.putd(t.E); io.putd(t.Y); io.putd(t.len); io.putd(t.safety); io.putd(t.mu); io.putd(t.mupe); io.putd(t.efrac);
  io.putd(t.w.best); io.putd(t.w.safety);
  io.putl(t.h); io.putl((uint64_t)t.tid); io.putl((uint64_t)t.gidx);
  io.put(t.leaf); io.put(t.item); io.put(t.steps); io.put(t.nzero); io.put(t.ebin); io.put(t.draw);
  io.put(t.w.bl); io.put(t.w.it);
  io.put(phase);
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    io.put(ch.h[l]);
    io.put(ch.k0[l]);
    io.put(ch.k1[l]);
  }
  io.put(ch.nlev);
  io.put(ch.list);
}

__device__ __forceinline__ void get_track(WordIO &io, Track &t, int &phase, Chain &ch) {
  t.x.x = io.getd(); t.x.y = io.getd(); t.x.z = io.getd();
  t.u.x = io.getd(); t.u.y = io.getd(); t.u.z = io.getd();
  t.iu.x = io.getd(); t.iu.y = io.getd(); t.iu.z = io.getd();
  t.E = io.getd(); t.Y = io.getd(); t.len = io.getd(); t.safety = io.getd(); t.mu = io.getd(); t.mupe = io.getd();
  t.efrac = io.getd();
  t.w.best = io.getd(); t.w.safety = io.getd();
  t.h = io.getl(); t.tid = (int64_t)io.getl(); t.gidx = (int64_t)io.getl();
  t.leaf = (int)io.get(); t.item = (int)io.get(); t.steps = (int)io.get(); t.nzero = (int)io.get();
  t.ebin = (int)io.get(); t.draw = io.get();
  t.w.bl = (int)io.get(); t.w.it = (int)io.get();
  phase = (int)io.get();
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    ch.h[l] = (int)io.get();
    ch.k0[l] = (int)io.get();
    ch.k1[l] = (int)io.get();
  }
  ch.nlev = (int)io.get();
  ch.list = (int)io.get();
}

// Block-wide regroup (every thread of the block calls it).  S: kTrackWords x blockDim.x words.
__device__ __forceinline__ void regroup_block(const TParams &P, Track &t, int &phase, Chain &ch, uint32_t *S) {
  __shared__ int count[kRegroupKeys], base[kRegroupKeys];
  const int tid = threadIdx.x;
  if (tid < kRegroupKeys) count[tid] = 0;
  __syncthreads();
  const int key = regroup_key(P, t, phase);
  const int rank = atomicAdd(&count[key], 1);
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
#pragma unroll
    for (int k = 0; k < kRegroupKeys; ++k) {
      base[k] = acc;
      acc += count[k];
    }
  }
  __syncthreads();
  WordIO out{S, (int)blockDim.x, base[key] + rank, 0};
  put_track(out, t, phase, ch);
  __syncthreads();
  WordIO in{S, (int)blockDim.x, tid, 0};
  get_track(in, t, phase, ch);
  __syncthreads();
}

// Persistent transport: every lane carries one track in registers.  Each round a
// warp (1) refills its idle lanes from the device queue when enough are idle (one
// atomic per refill), (2) runs the interaction phase when enough lanes wait for
// it, (3) advances every stepping lane by one step.  Deferring the long
// interaction and start-up code until many lanes need it keeps the warp's lanes
// on the same code; the order of operations inside each history is unchanged.
//
// YIELD: boundary searches yield after P.walk_budget voxel nodes (phase kWalk) and go on in a
// later round.  The kernel without it has none of that code: the workloads whose searches are
// short run faster without it (smaller code; measured 5 % on the calorimeter).
//
// REGROUP: every P.regroup rounds the block's tracks are regrouped (regroup_block); the rounds
// are then block-synchronous and the block ends when none of its lanes has work left.
//
// Occupancy: the kernel is latency bound, so 4 blocks of 128 per SM (128 registers, a few
// hundred bytes of spills to L1) beat 3 blocks without spills by 4 % on the calorimeter and the
// barrel.  The FP32 kernel with yielding searches spills most at 128 registers and keeps 3.
template <int MODE, bool COUNT, bool YIELD, bool REGROUP>
__global__ void __launch_bounds__(128, (MODE == kFP32 && YIELD) ? 3 : 4) k_transport(const TParams P) {
  constexpr bool kEv = !REGROUP;  // the regrouping kernels keep every count in registers
  Counters cnt;
#pragma unroll
  for (int k = 0; k < G4N_N_COUNTERS; ++k) cnt.c[k] = 0;
  if (kEv) {
    for (int k = threadIdx.x; k < G4N_N_COUNTERS; k += blockDim.x) s_events[k] = 0;
    __syncthreads();
  }
  const unsigned lane = threadIdx.x & 31u;
  MlpCtx mc{nullptr, nullptr, P.log, 0.f};
  if (MODE == kLearned) {
    extern __shared__ __align__(16) unsigned char smem[];
    mlp::SmemWeights *sw = reinterpret_cast<mlp::SmemWeights *>(smem);
    mlp::load_weights(*sw, P.mlp_w);
    __syncthreads();
    mc.w = sw;
    mc.scratch = reinterpret_cast<mlp::SmemWarp *>(smem + sizeof(mlp::SmemWeights)) + (threadIdx.x >> 5);
  }
  Track t;
  t.item = 0;
  t.leaf = 0;
  Chain wch;  // voxel chain of the lane's boundary search (kept while the search yields)
  int phase = kEmpty;
  bool drained = false;
  int round = 0;
#pragma unroll 1
  for (;;) {
    if (REGROUP) {
      if (round > 0 && round % P.regroup == 0) {
        if (!__syncthreads_or(phase != kEmpty || !drained)) break;
        extern __shared__ __align__(16) unsigned char smem_rg[];
        // the learned mode keeps its weights and per-warp scratch first; the regroup buffer follows them
        const size_t off = MODE == kLearned ? mlp_block_bytes(blockDim.x) : 0;
        regroup_block(P, t, phase, wch, reinterpret_cast<uint32_t *>(smem_rg + off));
      }
      ++round;
    }
    const unsigned idle = __ballot_sync(0xffffffffu, phase == kEmpty);
    const unsigned busy = ~idle;
    const long long c0 = COUNT ? clock64() : 0;
    if (idle && !drained && (__popc(idle) >= P.refill_min || busy == 0)) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(P.q_head, (unsigned long long)__popc(idle));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (base + __popc(idle) >= (unsigned long long)P.total) drained = true;
      const int64_t g = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
      const bool take = phase == kEmpty && g < P.total;
      const int started = start_warp<MODE, COUNT, kEv>(P, take, g, t, cnt);
      if (take) phase = started;
    }
    const unsigned waiting = __ballot_sync(0xffffffffu, phase == kInteract);
    const unsigned stepping = __ballot_sync(0xffffffffu, phase == kStep || phase == kWalk);
    const long long c1 = COUNT ? clock64() : 0;
    if (waiting && (__popc(waiting) >= P.interact_min || stepping == 0)) {
      if (phase == kInteract) phase = interact<MODE, kEv>(P, t, cnt);
    }
    __syncwarp();
    const long long c2 = COUNT ? clock64() : 0;
    const unsigned stepping2 = __ballot_sync(0xffffffffu, phase == kStep || phase == kWalk);
    if (!REGROUP || stepping2) phase = step_warp<MODE, COUNT, YIELD, kEv>(P, t, phase, cnt, mc, wch);
    if (COUNT) {
      __syncwarp();
      const long long c3 = clock64();
      if (lane == 0) {
        cnt.c[G4N_C_CYC_REFILL] += (uint32_t)((c1 - c0) >> 4);
        cnt.c[G4N_C_CYC_INTERACT] += (uint32_t)((c2 - c1) >> 4);
        cnt.c[G4N_C_CYC_STEP] += (uint32_t)((c3 - c2) >> 4);
        if (stepping2) {
          cnt.c[G4N_C_STEP_LANES] += __popc(stepping2);
          cnt.c[G4N_C_STEP_PHASES] += 1;
        }
      }
    }
    if (!REGROUP && drained && __ballot_sync(0xffffffffu, phase != kEmpty) == 0) break;
  }
  // flush counters: the block's event counts, then a warp reduction of the lanes' counts, one atomic
  // per counter per warp
  if (kEv) {
    cnt.c[G4N_C_STEPS] = cnt.c[G4N_C_GEOM_STEPS] + cnt.c[G4N_C_PHYS_STEPS];
    __syncthreads();
    for (int k = threadIdx.x; k < G4N_N_COUNTERS; k += blockDim.x)
      if (s_events[k]) atomicAdd(&P.counters[k], s_events[k]);
  }
#pragma unroll
  for (int k = 0; k < G4N_N_COUNTERS; ++k) {
    unsigned long long v = cnt.c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v) atomicAdd(&P.counters[k], v);
  }
}

// ---------------------------------------------------------------- free path (Algorithm 1)

struct FParams {
  const DGeom *geoms;
  int gid;
  int64_t n;
  const double *pos, *dir, *Y;
  double energy;
  double *out_T;
  int32_t *out_steps;
  unsigned long long *counters;
  unsigned long long *q_head;
  uint32_t *status;
  int64_t max_steps;
  int walk_cap;
  const mlp::SmemWeights *mlp_w;
};

// One ray per lane: the segment loop of Algorithm 1 with the optical depth S
// accumulated per segment.  Idle lanes take the next rays from the device
// queue (one atomic per warp); navigation is warp-collective as in transport.
template <int MODE, bool COUNT>
__global__ void __launch_bounds__(128, 3) k_free_path(const FParams P) {
  const DGeom &G = P.geoms[P.gid];
  Counters cnt;
#pragma unroll
  for (int k = 0; k < G4N_N_COUNTERS; ++k) cnt.c[k] = 0;
  const unsigned lane = threadIdx.x & 31u;
  MlpCtx mc{nullptr, nullptr, nullptr, 0.f};
  if (MODE == kLearned) {
    extern __shared__ __align__(16) unsigned char smem[];
    mlp::SmemWeights *sw = reinterpret_cast<mlp::SmemWeights *>(smem);
    mlp::load_weights(*sw, P.mlp_w);
    __syncthreads();
    mc.w = sw;
    mc.scratch = reinterpret_cast<mlp::SmemWarp *>(smem + sizeof(mlp::SmemWeights)) + (threadIdx.x >> 5);
    mc.loge = (logf((float)P.energy) + 4.6f) * 0.1f;
  }
  int64_t ray = -1, steps = 0;
  V3 x0{0, 0, 0}, u{0, 0, 1}, x{0, 0, 0};
  Inv3 iu{0, 0, 0};
  double t = 0.0, S = 0.0, Y = 0.0, mu = 0.0;
  int leaf = 0;
  bool active = false, drained = false;
#pragma unroll 1
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, !active);
    if (idle && !drained) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(P.q_head, (unsigned long long)__popc(idle));
      base = __shfl_sync(kFull, base, leader);
      if (base + __popc(idle) >= (unsigned long long)P.n) drained = true;
      const int64_t g = (int64_t)base + __popc(idle & ((1u << lane) - 1u));
      bool take = !active && g < P.n;
      if (take) {
        ray = g;
        x0 = V3{P.pos[g], P.pos[P.n + g], P.pos[2 * P.n + g]};
        u = V3{P.dir[g], P.dir[P.n + g], P.dir[2 * P.n + g]};
        Y = P.Y[g];
        steps = 0;
        if (bad_dir(u) || !isfinite(x0.x + x0.y + x0.z)) {
          flag(P.status, kStBadInput);
          P.out_T[g] = nan("");
          if (P.out_steps) P.out_steps[g] = 0;
          take = false;
        } else {
          cnt.c[G4N_C_TRACKS]++;
        }
      }
      const int l0 = locate_world_warp<COUNT>(G, take, x0, u, cnt);
      if (take) {
        if (!(Y > 0.0) || l0 < 0) {
          // Y <= 0: the interaction is at the start point; outside the world: no segment at all
          P.out_T[ray] = !(Y > 0.0) ? 0.0 : kInf;
          if (P.out_steps) P.out_steps[ray] = 0;
          if (Y > 0.0) cnt.c[G4N_C_ESCAPED]++;
        } else {
          leaf = l0;
          x = x0;
          iu = inv_dir(u);
          t = 0.0;
          S = 0.0;
          double mupe;
          mu_lookup(G, G.vol[leaf].mat, P.energy, mu, mupe);
          active = true;
        }
      }
    }
    if (drained && !__any_sync(kFull, active)) break;
    // one segment: the geometric step from x inside `leaf`
    V3 p{0, 0, 0}, v{0, 0, 1};
    Inv3 iv{0, 0, 0};
    if (active) {
      const bool aligned = G.vol[leaf].flags & kWorldAligned;
      world_to_local(G.wxf[leaf], aligned, x, u, p, v);
      iv = aligned ? iu : ((MODE == kFP64 || G.vol[leaf].kind == kBox) ? inv_dir(v) : Inv3{0.0, 0.0, 0.0});
    }
    bool timeout = false;
    Chain ch;
    const StepResult R = geom_step_warp<MODE, COUNT>(G, active, active ? leaf : 0, p, v, iv, kInf, false, cnt, &timeout,
                                                     P.walk_cap, mc, ch);
    bool cross = false;
    double s = 0.0;
    if (active) {
      if (timeout) flag(P.status, kStTimeout);
      s = R.step;
      ++steps;
      cnt.c[G4N_C_STEPS]++;
      if (mu > 0.0 && S + s * mu >= Y) {
        P.out_T[ray] = t + (Y - S) / mu;
        if (P.out_steps) P.out_steps[ray] = (int32_t)steps;
        cnt.c[G4N_C_PHYS_STEPS]++;
        active = false;
      } else if (steps >= P.max_steps) {
        flag(P.status, kStStepLimit);
        cnt.c[G4N_C_STEP_LIMIT]++;
        P.out_T[ray] = nan("");
        if (P.out_steps) P.out_steps[ray] = (int32_t)steps;
        active = false;
      } else {
        S += s * mu;
        t += s;
        x = V3{x0.x + t * u.x, x0.y + t * u.y, x0.z + t * u.z};
        cnt.c[G4N_C_GEOM_STEPS]++;
        cross = true;
      }
    }
    const bool left = cross && R.lim == G4N_LIM_MOTHER && s > 0.0;
    int nl = -1;
    const bool fast = left && face_relocate(G, leaf, R.face, x, u, &nl);
    if (fast) diag<COUNT>(cnt, G4N_C_FACE_RELOC);
    const int searched = relocate_warp<MODE, COUNT>(G, cross && !fast, cross && !fast ? leaf : 0, x, u, left, cnt);
    if (!fast) nl = searched;
    if (cross) {
      if (nl < 0) {
        P.out_T[ray] = kInf;
        if (P.out_steps) P.out_steps[ray] = (int32_t)steps;
        cnt.c[G4N_C_ESCAPED]++;
        active = false;
      } else {
        leaf = nl;
        double mupe;
        mu_lookup(G, G.vol[leaf].mat, P.energy, mu, mupe);
      }
    }
  }
  if (P.counters) {
#pragma unroll
    for (int k = 0; k < G4N_N_COUNTERS; ++k) {
      unsigned long long c = cnt.c[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
      if (lane == 0 && c) atomicAdd(&P.counters[k], c);
    }
  }
}

using FreePathKernel = void (*)(const FParams);

FreePathKernel free_path_kernel(int mode, bool count) {
  if (mode == G4N_MODE_FP64) return count ? k_free_path<kFP64, true> : k_free_path<kFP64, false>;
  if (mode == G4N_MODE_FP32_RECHECK) return count ? k_free_path<kFP32, true> : k_free_path<kFP32, false>;
  return count ? k_free_path<kLearned, true> : k_free_path<kLearned, false>;
}

using TransportKernel = void (*)(const TParams);

// The diagnostics kernel always has the yield code (its counters then also count yields); the
// learned mode never yields.
// The regrouping variants exist for the FP64 and FP32 modes without diagnostics.
template <int MODE>
TransportKernel plain_kernel(bool yield, bool regroup) {
  if (regroup) return yield ? k_transport<MODE, false, true, true> : k_transport<MODE, false, false, true>;
  return yield ? k_transport<MODE, false, true, false> : k_transport<MODE, false, false, false>;
}

TransportKernel transport_kernel(int mode, bool count, bool yield, bool regroup) {
  if (mode == G4N_MODE_FP64) return count ? k_transport<kFP64, true, true, false> : plain_kernel<kFP64>(yield, regroup);
  if (mode == G4N_MODE_FP32_RECHECK)
    return count ? k_transport<kFP32, true, true, false> : plain_kernel<kFP32>(yield, regroup);
  if (count) return k_transport<kLearned, true, false, false>;
  return regroup ? k_transport<kLearned, false, false, true> : k_transport<kLearned, false, false, false>;
}

// Dynamic shared memory of a launch: the MLP weights and one scratch tile per warp (learned mode).
// Dynamic shared memory of a transport launch: the MLP weights (learned mode) or the
// regroup buffer (regrouping kernels).
size_t transport_smem_bytes(int mode, int block, int regroup);

size_t mlp_smem_bytes(int mode, int block) { return mode == G4N_MODE_LEARNED ? mlp_block_bytes(block) : 0; }

size_t transport_smem_bytes(int mode, int block, int regroup) {
  return mlp_smem_bytes(mode, block) + (regroup > 0 ? (size_t)kTrackWords * block * sizeof(uint32_t) : 0);
}

// ---------------------------------------------------------------- host helpers

int check_geom(g4n_ctx *ctx, int32_t geom) {
  if (!ctx) return G4N_ERR_ARG;
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device queries");
  if (geom < 0 || geom >= (int32_t)ctx->geoms.size()) return g4n_fail(ctx, G4N_ERR_ARG, "unknown geometry id");
  return G4N_OK;
}

// The workspace header (queue head, status word, sample log) is allocated once and never moves;
// the item table grows by doubling.  An outgrown table may still be read by work in flight on
// some stream, so it is retired (freed by g4n_destroy) rather than freed: growing never
// synchronizes the device.
int ensure_ws(g4n_ctx *ctx, size_t item_bytes) {
  if (!ctx->ws) {
    if (cudaMalloc(&ctx->ws, sizeof(Workspace)) != cudaSuccess) {
      ctx->ws = nullptr;
      return g4n_fail(ctx, G4N_ERR_OOM, "workspace allocation failed");
    }
    if (cudaMemset(ctx->ws, 0, sizeof(Workspace)) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, "workspace init failed");
  }
  if (item_bytes <= ctx->items_bytes) return G4N_OK;
  const size_t bytes = std::max<size_t>({item_bytes, 2 * ctx->items_bytes, size_t(1) << 16});
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_OOM, "item table allocation failed");
  if (ctx->items) ctx->retired.push_back(ctx->items);
  ctx->items = p;
  ctx->items_bytes = bytes;
  return G4N_OK;
}

int launch_error(g4n_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return G4N_OK;
}

// Launch shape of a transport batch (validated); 0 fields take the defaults.
int transport_shape(g4n_ctx *ctx, const g4n_batch_desc *b, int *block, int *refill, int *inter, int *budget,
                    int *regroup) {
  *block = b->block_size > 0 ? b->block_size : 128;
  if (b->regroup_period < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport: regroup_period must be >= 0");
  *regroup = std::min(b->regroup_period, 1 << 20);
  if (b->walk_budget < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport: walk_budget must be >= 0");
  *budget = b->walk_budget > 0 ? std::min(b->walk_budget, 1 << 20) : kDefaultWalkBudget;
  if (*block % 32 || *block > 128) return g4n_fail(ctx, G4N_ERR_ARG, "transport: block_size must be a multiple of 32, <= 128");
  *refill = b->refill_min > 0 ? b->refill_min : 8;
  *inter = b->interact_min > 0 ? b->interact_min : 8;
  if (*refill > 32 || *inter > 32) return g4n_fail(ctx, G4N_ERR_ARG, "transport: refill_min/interact_min must be 1..32");
  if (b->mode != G4N_MODE_FP64 && b->mode != G4N_MODE_FP32_RECHECK && b->mode != G4N_MODE_LEARNED)
    return g4n_fail(ctx, G4N_ERR_ARG, "transport: unknown mode");
  if (b->schedule != G4N_SCHEDULE_PERSISTENT && b->schedule != G4N_SCHEDULE_STAGED)
    return g4n_fail(ctx, G4N_ERR_ARG, "transport: unknown schedule");
  if (b->pool_tracks < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport: pool_tracks must be >= 0");
  if (b->staged_flags & ~G4N_STAGED_RELOCATION_KERNEL) return g4n_fail(ctx, G4N_ERR_ARG, "transport: unknown staged_flags");
  if (b->mode == G4N_MODE_LEARNED && !g4n_mlp_image(ctx))
    return g4n_fail(ctx, G4N_ERR_STATE, "transport: learned mode needs MLP weights (g4n_mlp_load / g4n_mlp_train)");
  return G4N_OK;
}

// Validate the work items of a batch and build their device records.
int build_items(g4n_ctx *ctx, const g4n_batch_desc *b, std::vector<DItem> &items, int64_t &total) {
  items.assign(b->n_items, DItem{});
  total = 0;
  for (int i = 0; i < b->n_items; ++i) {
    const g4n_work_item &w = b->items[i];
    int rc = check_geom(ctx, w.geom);
    if (rc) return rc;
    const int64_t nv = ctx->geoms[w.geom]->dview.n_vol;
    if (w.n_tracks < 0 || w.track_id0 < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport: negative track count or id");
    if (w.tally_offset < 0 || w.tally_offset + nv + 2 > b->tally_stride)
      return g4n_fail(ctx, G4N_ERR_ARG, "transport: tally columns out of range");
    const g4n_source &s = w.source;
    if (!s.isotropic) {
      const double n2 = s.dir[0] * s.dir[0] + s.dir[1] * s.dir[1] + s.dir[2] * s.dir[2];
      if (!(std::fabs(n2 - 1.0) <= 1e-12)) return g4n_fail(ctx, G4N_ERR_ARG, "transport: source direction not unit");
    }
    if (s.e_kind < 0 || s.e_kind > 2 || !(s.e0 > 0.0) || (s.e_kind > 0 && !(s.e1 >= s.e0)))
      return g4n_fail(ctx, G4N_ERR_ARG, "transport: bad source energy");
    if (!(s.spot_sigma >= 0.0)) return g4n_fail(ctx, G4N_ERR_ARG, "transport: negative spot sigma");
    DItem &d = items[i];
    std::memset(&d, 0, sizeof(d));
    d.geom = w.geom;
    d.n = w.n_tracks;
    d.tid0 = w.track_id0;
    d.tally_off = w.tally_offset;
    d.start = total;
    double src[16] = {s.pos[0], s.pos[1], s.pos[2], s.spot_sigma, (double)(s.has_z != 0), s.z0, s.z1,
                      (double)(s.isotropic != 0), s.dir[0], s.dir[1], s.dir[2], (double)s.e_kind, s.e0, s.e1, 0.0, 0.0};
    std::memcpy(d.src, src, sizeof(src));
    total += w.n_tracks;
  }
  return G4N_OK;
}

// Launch the persistent transport kernel of mode b->mode with parameters P on `st`.
int launch_transport(g4n_ctx *ctx, const g4n_batch_desc *b, TParams &P, int block, cudaStream_t st) {
  const TransportKernel kern = transport_kernel(b->mode, b->flags & G4N_FLAG_DIAGNOSTICS, P.walk_budget < kNeverYield, P.regroup > 0);
  const size_t smem = transport_smem_bytes(b->mode, block, (b->flags & G4N_FLAG_DIAGNOSTICS) ? 0 : P.regroup);
  P.mlp_w = g4n_mlp_image(ctx);
  if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = b->blocks_per_sm;
  if (per_sm <= 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    per_sm = std::max(per_sm, 1);
  }
  int64_t grid = (int64_t)ctx->sm_count * per_sm;
  const int64_t need = (P.total + block - 1) / block;
  grid = std::max<int64_t>(1, std::min(grid, need));
  kern<<<(int)grid, block, smem, st>>>(P);
  ++ctx->launches;
  return launch_error(ctx, "transport launch");
}

int grid_for(g4n_ctx *ctx, int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  int64_t cap = (int64_t)ctx->sm_count * 16;
  return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

#include "transport_staged.cuh"

extern "C" {

int g4n_locate(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir, int32_t *out_depth,
               int32_t *out_path, g4n_stream stream) {
  int rc = check_geom(ctx, geom);
  if (rc) return rc;
  if (n < 0) return g4n_fail(ctx, G4N_ERR_ARG, "locate: n < 0");
  if (n == 0) return G4N_OK;
  if (!pos || !dir || !out_depth || !out_path) return g4n_fail(ctx, G4N_ERR_ARG, "locate: null array");
  if ((rc = ensure_ws(ctx, 0))) return rc;
  cudaSetDevice(ctx->device);
  Workspace *ws = (Workspace *)ctx->ws;
  ++ctx->launches;
  k_locate<<<grid_for(ctx, n, 128), 128, 0, (cudaStream_t)stream>>>(ctx->d_geoms, geom, n, pos, dir, out_depth,
                                                                     out_path, &ws->status);
  return launch_error(ctx, "locate launch");
}

int g4n_compute_step(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir, const int32_t *depth,
                     const int32_t *path, const double *proposed, double *out_step, double *out_safety,
                     int32_t *out_limiter, int32_t mode, g4n_stream stream) {
  int rc = check_geom(ctx, geom);
  if (rc) return rc;
  if (n < 0) return g4n_fail(ctx, G4N_ERR_ARG, "compute_step: n < 0");
  if (mode != G4N_MODE_FP64 && mode != G4N_MODE_FP32_RECHECK && mode != G4N_MODE_LEARNED)
    return g4n_fail(ctx, G4N_ERR_ARG, "compute_step: unknown mode");
  if (mode == G4N_MODE_LEARNED && !g4n_mlp_image(ctx))
    return g4n_fail(ctx, G4N_ERR_STATE, "compute_step: learned mode needs MLP weights");
  if (n == 0) return G4N_OK;
  if (!pos || !dir || !depth || !path || !out_step || !out_safety || !out_limiter)
    return g4n_fail(ctx, G4N_ERR_ARG, "compute_step: null array");
  if ((rc = ensure_ws(ctx, 0))) return rc;
  cudaSetDevice(ctx->device);
  Workspace *ws = (Workspace *)ctx->ws;
  auto kern = mode == G4N_MODE_FP64 ? k_compute_step<kFP64>
                                    : (mode == G4N_MODE_FP32_RECHECK ? k_compute_step<kFP32> : k_compute_step<kLearned>);
  const size_t smem = mlp_smem_bytes(mode, 128);
  if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ++ctx->launches;
  kern<<<grid_for(ctx, n, 128), 128, smem, (cudaStream_t)stream>>>(ctx->d_geoms, geom, n, pos, dir, depth, path,
                                                                    proposed, out_step, out_safety, out_limiter,
                                                                    &ws->status, g4n_mlp_image(ctx), ctx->walk_cap);
  return launch_error(ctx, "compute_step launch");
}

static int transport_impl(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep, uint64_t *out_counters,
                          uint64_t *out_track_hash, double *out_track_len, g4n_stream stream, bool logging);

int g4n_transport_batch(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep, uint64_t *out_counters,
                        uint64_t *out_track_hash, double *out_track_len, g4n_stream stream) {
  return transport_impl(ctx, b, out_edep, out_counters, out_track_hash, out_track_len, stream, false);
}

static int transport_impl(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep, uint64_t *out_counters,
                          uint64_t *out_track_hash, double *out_track_len, g4n_stream stream, bool logging) {
  if (!ctx || !b) return g4n_fail(ctx, G4N_ERR_ARG, "transport: null argument");
  if (b->n_items < 1 || !b->items) return g4n_fail(ctx, G4N_ERR_ARG, "transport: no work items");
  if (!out_edep || !out_counters) return g4n_fail(ctx, G4N_ERR_ARG, "transport: null output");
  int block, refill, inter, budget, regroup;
  if (int rc0 = transport_shape(ctx, b, &block, &refill, &inter, &budget, &regroup)) return rc0;
  if (b->n_tally_batches < 1) return g4n_fail(ctx, G4N_ERR_ARG, "transport: n_tally_batches < 1");
  if (!(b->cutoff >= 0.0)) return g4n_fail(ctx, G4N_ERR_ARG, "transport: cutoff must be >= 0");
  std::vector<DItem> items;
  int64_t total = 0;
  if (int rc1 = build_items(ctx, b, items, total)) return rc1;
  if (total == 0) return G4N_OK;
  int rc = ensure_ws(ctx, items.size() * sizeof(DItem));
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *ws = (Workspace *)ctx->ws;
  DItem *d_items = (DItem *)ctx->items;
  if (cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(DItem), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(&ws->q_head, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "transport: item upload failed");
  TParams P;
  P.geoms = ctx->d_geoms;
  P.items = d_items;
  P.n_items = b->n_items;
  P.total = total;
  P.q_head = &ws->q_head;
  P.status = &ws->status;
  P.seed = b->seed;
  P.cutoff = b->cutoff;
  P.max_steps = b->max_steps > 0 ? b->max_steps : 1000000;
  P.nb = b->n_tally_batches;
  P.stride = b->tally_stride;
  P.edep = out_edep;
  P.counters = (unsigned long long *)out_counters;
  P.out_hash = out_track_hash;
  P.out_len = out_track_len;
  P.refill_min = refill;
  P.interact_min = inter;
  P.walk_budget = budget;
  P.regroup = regroup;
  P.walk_cap = ctx->walk_cap;
  P.trial_cap = ctx->trial_cap;
  P.log = logging ? &ws->log : nullptr;
  if (b->schedule == G4N_SCHEDULE_STAGED && !logging && !(b->flags & G4N_FLAG_DIAGNOSTICS))
    return staged_transport(ctx, b, P, st);
  return launch_transport(ctx, b, P, block, st);
}

int g4n_transport_batch_host(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep, uint64_t *out_counters,
                             uint64_t *out_track_hash, double *out_track_len, g4n_stream stream) {
  if (!ctx || !b || !out_edep || !out_counters) return g4n_fail(ctx, G4N_ERR_ARG, "transport_host: null argument");
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device queries");
  int64_t total = 0;
  for (int i = 0; i < b->n_items && b->items; ++i) total += std::max<int64_t>(0, b->items[i].n_tracks);
  const size_t e_bytes = (size_t)b->n_tally_batches * (size_t)std::max<int64_t>(b->tally_stride, 0) * sizeof(double);
  const size_t c_bytes = G4N_N_COUNTERS * sizeof(uint64_t);
  const size_t h_bytes = out_track_hash ? (size_t)total * sizeof(uint64_t) : 0;
  const size_t l_bytes = out_track_len ? (size_t)total * sizeof(double) : 0;
  const size_t need = e_bytes + c_bytes + h_bytes + l_bytes + 4 * 256;
  cudaSetDevice(ctx->device);
  if (ctx->d_stage_bytes < need) {
    // grow by doubling; the outgrown buffer is retired, not freed (no device-wide synchronization)
    const size_t bytes = std::max(need, 2 * ctx->d_stage_bytes);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_OOM, "transport_host: staging allocation failed");
    if (ctx->d_stage) ctx->retired.push_back(ctx->d_stage);
    ctx->d_stage = p;
    ctx->d_stage_bytes = bytes;
  }
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  char *base = (char *)ctx->d_stage;
  double *d_e = (double *)base;
  uint64_t *d_c = (uint64_t *)(base + al(e_bytes));
  uint64_t *d_h = out_track_hash ? (uint64_t *)(base + al(e_bytes) + al(c_bytes)) : nullptr;
  double *d_l = out_track_len ? (double *)(base + al(e_bytes) + al(c_bytes) + al(h_bytes)) : nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_e, 0, e_bytes, st) != cudaSuccess || cudaMemsetAsync(d_c, 0, c_bytes, st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "transport_host: clear failed");
  int rc = g4n_transport_batch(ctx, b, d_e, d_c, d_h, d_l, stream);
  if (rc) return rc;
  if (cudaMemcpyAsync(out_edep, d_e, e_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(out_counters, d_c, c_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (d_h && cudaMemcpyAsync(out_track_hash, d_h, h_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      (d_l && cudaMemcpyAsync(out_track_len, d_l, l_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess))
    return g4n_fail(ctx, G4N_ERR_CUDA, "transport_host: copy back failed");
  return g4n_sync(ctx, stream);
}

int g4n_mlp_log(g4n_ctx *ctx, const g4n_batch_desc *b, float *feat, int32_t *label, int32_t *ncand, int64_t capacity,
                int64_t *out_count, g4n_stream stream) {
  if (!ctx || !b || !out_count) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_log: null argument");
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device queries");
  if (capacity < 0 || (capacity > 0 && (!feat || !label || !ncand))) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_log: bad buffers");
  if (b->mode != G4N_MODE_FP64) return g4n_fail(ctx, G4N_ERR_ARG, "mlp_log: samples are logged by the plain FP64 navigator");
  int rc = ensure_ws(ctx, (size_t)std::max(b->n_items, 1) * sizeof(DItem));
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *ws = (Workspace *)ctx->ws;
  dev::MlpLog L{feat, label, ncand, &ws->log_count, capacity};
  if (cudaMemcpyAsync(&ws->log, &L, sizeof(L), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(&ws->log_count, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "mlp_log: setup failed");
  // scratch outputs of the logging run (tallies and counters are not returned)
  int64_t stride = b->tally_stride;
  double *edep = nullptr;
  unsigned long long *cnt = nullptr;
  if (cudaMalloc(&edep, (size_t)b->n_tally_batches * stride * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&cnt, G4N_N_COUNTERS * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(edep);
    return g4n_fail(ctx, G4N_ERR_OOM, "mlp_log: allocation failed");
  }
  cudaMemsetAsync(edep, 0, (size_t)b->n_tally_batches * stride * sizeof(double), st);
  cudaMemsetAsync(cnt, 0, G4N_N_COUNTERS * sizeof(unsigned long long), st);
  rc = transport_impl(ctx, b, edep, (uint64_t *)cnt, nullptr, nullptr, stream, true);
  unsigned long long c = 0;
  if (rc == G4N_OK) {
    cudaMemcpyAsync(&c, &ws->log_count, sizeof(c), cudaMemcpyDeviceToHost, st);
    rc = g4n_sync(ctx, stream);
  }
  cudaFree(edep);
  cudaFree(cnt);
  if (rc) return rc;
  *out_count = (int64_t)std::min<unsigned long long>(c, (unsigned long long)capacity);
  return G4N_OK;
}

int g4n_free_path(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir, const double *Y,
                  double energy, double *out_T, int32_t *out_steps, uint64_t *out_counters, int32_t mode,
                  int64_t max_steps, int32_t flags, g4n_stream stream) {
  int rc = check_geom(ctx, geom);
  if (rc) return rc;
  if (n < 0) return g4n_fail(ctx, G4N_ERR_ARG, "free_path: n < 0");
  if (mode != G4N_MODE_FP64 && mode != G4N_MODE_FP32_RECHECK && mode != G4N_MODE_LEARNED)
    return g4n_fail(ctx, G4N_ERR_ARG, "free_path: unknown mode");
  if (mode == G4N_MODE_LEARNED && !g4n_mlp_image(ctx))
    return g4n_fail(ctx, G4N_ERR_STATE, "free_path: learned mode needs MLP weights");
  if (!(energy > 0.0) || !std::isfinite(energy)) return g4n_fail(ctx, G4N_ERR_ARG, "free_path: energy must be > 0");
  if (max_steps < 0) return g4n_fail(ctx, G4N_ERR_ARG, "free_path: max_steps < 0");
  if (n == 0) return G4N_OK;
  if (!pos || !dir || !Y || !out_T) return g4n_fail(ctx, G4N_ERR_ARG, "free_path: null array");
  if ((rc = ensure_ws(ctx, 0))) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *ws = (Workspace *)ctx->ws;
  if (cudaMemsetAsync(&ws->q_head, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "free_path: queue reset failed");
  FParams P;
  P.geoms = ctx->d_geoms;
  P.gid = geom;
  P.n = n;
  P.pos = pos;
  P.dir = dir;
  P.Y = Y;
  P.energy = energy;
  P.out_T = out_T;
  P.out_steps = out_steps;
  P.counters = reinterpret_cast<unsigned long long *>(out_counters);
  P.q_head = &ws->q_head;
  P.status = &ws->status;
  P.max_steps = max_steps > 0 ? max_steps : 1000000;
  P.walk_cap = ctx->walk_cap;
  P.mlp_w = g4n_mlp_image(ctx);
  const FreePathKernel kern = free_path_kernel(mode, (flags & G4N_FLAG_DIAGNOSTICS) && out_counters);
  const int block = 128;
  const size_t smem = mlp_smem_bytes(mode, block);
  if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
  int64_t grid = (int64_t)ctx->sm_count * std::max(per_sm, 1);
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, (n + block - 1) / block));
  kern<<<(int)grid, block, smem, st>>>(P);
  ++ctx->launches;
  return launch_error(ctx, "free_path launch");
}

int g4n_set_loop_caps(g4n_ctx *ctx, int32_t max_walk_nodes, int32_t max_sampler_trials) {
  if (!ctx) return G4N_ERR_ARG;
  if (max_walk_nodes < 0 || max_sampler_trials < 0) return g4n_fail(ctx, G4N_ERR_ARG, "loop caps must be >= 0");
  ctx->walk_cap = max_walk_nodes > 0 ? max_walk_nodes : kDefaultWalkCap;
  ctx->trial_cap = max_sampler_trials > 0 ? max_sampler_trials : kDefaultTrialCap;
  return G4N_OK;
}

int64_t g4n_kernel_launches(const g4n_ctx *ctx) { return ctx ? ctx->launches : -1; }

int g4n_sync(g4n_ctx *ctx, g4n_stream stream) {
  if (!ctx) return G4N_ERR_ARG;
  if (ctx->device < 0) return G4N_OK;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  if (!ctx->ws) return G4N_OK;
  uint32_t st = 0;
  Workspace *ws = (Workspace *)ctx->ws;
  if (cudaMemcpy(&st, &ws->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "sync: status read failed");
  if (st == 0) return G4N_OK;
  cudaMemset(&ws->status, 0, sizeof(uint32_t));
  if (st & kStBadInput) return g4n_fail(ctx, G4N_ERR_ARG, "device: non-unit/non-finite direction or bad path/depth input");
  if (st & kStTimeout) return g4n_fail(ctx, G4N_ERR_TIMEOUT, "device: a voxel walk reached its iteration cap");
  if (st & kStRejection) return g4n_fail(ctx, G4N_ERR_TIMEOUT, "device: a rejection sampler reached its trial cap");
  if (st & kStStepLimit) return g4n_fail(ctx, G4N_ERR_STEP_LIMIT, "device: a track reached the per-track step cap");
  return g4n_fail(ctx, G4N_ERR_STATE, "device: unknown status");
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free transport
//
// g4n_transport_batch keeps its queue head, status word and work-item table in
// a workspace that the context allocates with cudaMalloc on first use.  Some
// callers cannot allow that: a process whose own allocator has reserved the
// device memory up front, or a latency-critical loop that forbids device
// allocation (and the device-wide synchronization cudaFree implies) once it is
// running.  g4n_transport_batch_noalloc runs the same transport kernel with that
// scratch held in the fixed device array below instead, and calls no allocating
// CUDA or library routine.

namespace {

constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)G4N_NOALLOC_MAX_ITEMS * sizeof(DItem);

// Shared by every call in the process; every GPU that loads this library keeps it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current), looked up once per device.
int noalloc_scratch(g4n_ctx *ctx, int device, unsigned char **out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return g4n_fail(ctx, G4N_ERR_CUDA, std::string("transport_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    g_noalloc_addr[device] = p;
  }
  *out = (unsigned char *)g_noalloc_addr[device];
  return G4N_OK;
}

}  // namespace

extern "C" int g4n_transport_batch_noalloc(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep,
                                           uint64_t *out_counters, uint64_t *out_track_hash, double *out_track_len,
                                           g4n_stream stream) {
  if (!ctx || !b) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: null argument");
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device queries");
  if (b->n_items < 1 || !b->items) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: no work items");
  if (b->n_items > G4N_NOALLOC_MAX_ITEMS)
    return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: more than G4N_NOALLOC_MAX_ITEMS (" +
                                          std::to_string(G4N_NOALLOC_MAX_ITEMS) + ") work items; use g4n_transport_batch");
  if (!out_edep || !out_counters) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: null output");
  int block, refill, inter, budget, regroup;
  if (int rc0 = transport_shape(ctx, b, &block, &refill, &inter, &budget, &regroup)) return rc0;
  if (b->n_tally_batches < 1) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: n_tally_batches < 1");
  if (!(b->cutoff >= 0.0)) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: cutoff must be >= 0");
  DItem items[G4N_NOALLOC_MAX_ITEMS];  // host staging on the stack: no heap either
  int64_t total = 0;
  for (int i = 0; i < b->n_items; ++i) {
    const g4n_work_item &w = b->items[i];
    int rc = check_geom(ctx, w.geom);
    if (rc) return rc;
    const int64_t nv = ctx->geoms[w.geom]->dview.n_vol;
    if (w.n_tracks < 0 || w.track_id0 < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: negative track count or id");
    if (w.tally_offset < 0 || w.tally_offset + nv + 2 > b->tally_stride)
      return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: tally columns out of range");
    const g4n_source &s = w.source;
    if (!s.isotropic) {
      const double n2 = s.dir[0] * s.dir[0] + s.dir[1] * s.dir[1] + s.dir[2] * s.dir[2];
      if (!(std::fabs(n2 - 1.0) <= 1e-12)) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: source direction not unit");
    }
    if (s.e_kind < 0 || s.e_kind > 2 || !(s.e0 > 0.0) || (s.e_kind > 0 && !(s.e1 >= s.e0)))
      return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: bad source energy");
    if (!(s.spot_sigma >= 0.0)) return g4n_fail(ctx, G4N_ERR_ARG, "transport_noalloc: negative spot sigma");
    DItem &d = items[i];
    std::memset(&d, 0, sizeof(d));
    d.geom = w.geom;
    d.n = w.n_tracks;
    d.tid0 = w.track_id0;
    d.tally_off = w.tally_offset;
    d.start = total;
    const double src[16] = {s.pos[0], s.pos[1], s.pos[2], s.spot_sigma, (double)(s.has_z != 0), s.z0, s.z1,
                            (double)(s.isotropic != 0), s.dir[0], s.dir[1], s.dir[2], (double)s.e_kind, s.e0, s.e1,
                            0.0, 0.0};
    std::memcpy(d.src, src, sizeof(src));
    total += w.n_tracks;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, "transport_noalloc: cudaSetDevice failed");
  unsigned char *scratch = nullptr;
  int rc = noalloc_scratch(ctx, ctx->device, &scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // queue head and status start at zero on every call; the item table is rewritten
  if (cudaMemsetAsync(scratch, 0, 16, st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "transport_noalloc: scratch clear failed");
  if (total > 0) {
    if (cudaMemcpyAsync(scratch + kNoAllocHeader, items, (size_t)b->n_items * sizeof(DItem), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return g4n_fail(ctx, G4N_ERR_CUDA, "transport_noalloc: item upload failed");
    TParams P;
    P.geoms = ctx->d_geoms;
    P.items = (const DItem *)(scratch + kNoAllocHeader);
    P.n_items = b->n_items;
    P.total = total;
    P.q_head = (unsigned long long *)scratch;
    P.status = (uint32_t *)(scratch + 8);
    P.seed = b->seed;
    P.cutoff = b->cutoff;
    P.max_steps = b->max_steps > 0 ? b->max_steps : 1000000;
    P.nb = b->n_tally_batches;
    P.stride = b->tally_stride;
    P.edep = out_edep;
    P.counters = (unsigned long long *)out_counters;
    P.out_hash = out_track_hash;
    P.out_len = out_track_len;
    P.refill_min = refill;
    P.interact_min = inter;
    P.walk_budget = budget;
    P.regroup = regroup;
    P.walk_cap = ctx->walk_cap;
    P.trial_cap = ctx->trial_cap;
    P.log = nullptr;
    rc = launch_transport(ctx, b, P, block, st);
    if (rc) return rc;
  }
  // report this call's device status bits in the last counter slot
  if (cudaMemcpyAsync(out_counters + G4N_NOALLOC_STATUS_SLOT, scratch + 8, sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return g4n_fail(ctx, G4N_ERR_CUDA, "transport_noalloc: status copy failed");
  return G4N_OK;
}

// ---------------------------------------------------------------- CUDA graphs of a transport batch
//
// A batch that is launched again and again (the same geometry, items and outputs, a new seed)
// is recorded once as a CUDA graph: a node that resets the graph's own queue head, then the
// persistent kernel.  Replays change only the seed in the kernel node, so a replay costs one
// cudaGraphLaunch instead of an item upload, a memset and a kernel launch.

struct g4n_graph {
  g4n_ctx *ctx = nullptr;
  void *scratch = nullptr;  // queue head (first 256 B) and the device item table
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
  cudaKernelNodeParams kp{};
  TParams P{};
  void *args[1] = {nullptr};
};

extern "C" {

int g4n_graph_create(g4n_ctx *ctx, const g4n_batch_desc *b, double *out_edep, uint64_t *out_counters,
                     uint64_t *out_track_hash, double *out_track_len, g4n_graph **out) {
  if (!ctx || !b || !out) return g4n_fail(ctx, G4N_ERR_ARG, "graph_create: null argument");
  *out = nullptr;
  if (ctx->device < 0) return g4n_fail(ctx, G4N_ERR_STATE, "host-only context: no device queries");
  if (b->n_items < 1 || !b->items || !out_edep || !out_counters) return g4n_fail(ctx, G4N_ERR_ARG, "graph_create: no items or outputs");
  int block, refill, inter, budget, regroup;
  if (int rc0 = transport_shape(ctx, b, &block, &refill, &inter, &budget, &regroup)) return rc0;
  if (b->n_tally_batches < 1 || !(b->cutoff >= 0.0)) return g4n_fail(ctx, G4N_ERR_ARG, "graph_create: bad tallies or cutoff");
  std::vector<DItem> items;
  int64_t total = 0;
  if (int rc1 = build_items(ctx, b, items, total)) return rc1;
  if (total == 0) return g4n_fail(ctx, G4N_ERR_ARG, "graph_create: no tracks");
  if (int rc2 = ensure_ws(ctx, 0)) return rc2;
  cudaSetDevice(ctx->device);
  g4n_graph *g = new g4n_graph();
  g->ctx = ctx;
  const size_t bytes = 256 + items.size() * sizeof(DItem);
  if (cudaMalloc(&g->scratch, bytes) != cudaSuccess) {
    delete g;
    return g4n_fail(ctx, G4N_ERR_OOM, "graph_create: allocation failed");
  }
  DItem *d_items = (DItem *)((char *)g->scratch + 256);
  if (cudaMemcpy(d_items, items.data(), items.size() * sizeof(DItem), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(g->scratch);
    delete g;
    return g4n_fail(ctx, G4N_ERR_CUDA, "graph_create: item upload failed");
  }
  Workspace *ws = (Workspace *)ctx->ws;
  TParams &P = g->P;
  P.geoms = ctx->d_geoms;
  P.items = d_items;
  P.n_items = b->n_items;
  P.total = total;
  P.q_head = (unsigned long long *)g->scratch;
  P.status = &ws->status;
  P.seed = b->seed;
  P.cutoff = b->cutoff;
  P.max_steps = b->max_steps > 0 ? b->max_steps : 1000000;
  P.nb = b->n_tally_batches;
  P.stride = b->tally_stride;
  P.edep = out_edep;
  P.counters = (unsigned long long *)out_counters;
  P.out_hash = out_track_hash;
  P.out_len = out_track_len;
  P.refill_min = refill;
  P.interact_min = inter;
  P.walk_budget = budget;
  P.regroup = regroup;
  P.walk_cap = ctx->walk_cap;
  P.trial_cap = ctx->trial_cap;
  P.log = nullptr;
  P.mlp_w = g4n_mlp_image(ctx);
  const TransportKernel kern = transport_kernel(b->mode, b->flags & G4N_FLAG_DIAGNOSTICS, P.walk_budget < kNeverYield, P.regroup > 0);
  const size_t smem = transport_smem_bytes(b->mode, block, (b->flags & G4N_FLAG_DIAGNOSTICS) ? 0 : P.regroup);
  if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = b->blocks_per_sm;
  if (per_sm <= 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    per_sm = std::max(per_sm, 1);
  }
  int64_t grid = (int64_t)ctx->sm_count * per_sm;
  grid = std::max<int64_t>(1, std::min(grid, (total + block - 1) / block));
  bool ok = cudaGraphCreate(&g->graph, 0) == cudaSuccess;
  cudaGraphNode_t reset = nullptr;
  if (ok) {
    cudaMemsetParams mp{};
    mp.dst = g->scratch;
    mp.value = 0;
    mp.elementSize = 1;
    mp.width = 16;
    mp.height = 1;
    mp.pitch = 0;
    ok = cudaGraphAddMemsetNode(&reset, g->graph, nullptr, 0, &mp) == cudaSuccess;
  }
  if (ok) {
    g->args[0] = &g->P;
    g->kp.func = (void *)kern;
    g->kp.gridDim = dim3((unsigned)grid);
    g->kp.blockDim = dim3((unsigned)block);
    g->kp.sharedMemBytes = (unsigned)smem;
    g->kp.kernelParams = g->args;
    g->kp.extra = nullptr;
    ok = cudaGraphAddKernelNode(&g->kernel_node, g->graph, &reset, 1, &g->kp) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&g->exec, g->graph, 0) == cudaSuccess;
  if (!ok) {
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->scratch);
    delete g;
    return g4n_fail(ctx, G4N_ERR_CUDA, "graph_create: graph construction failed");
  }
  *out = g;
  return G4N_OK;
}

int g4n_graph_launch(g4n_graph *g, uint64_t seed, g4n_stream stream) {
  if (!g) return G4N_ERR_ARG;
  cudaSetDevice(g->ctx->device);
  g->P.seed = seed;
  if (cudaGraphExecKernelNodeSetParams(g->exec, g->kernel_node, &g->kp) != cudaSuccess ||
      cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess)
    return g4n_fail(g->ctx, G4N_ERR_CUDA, "graph_launch failed");
  ++g->ctx->launches;
  return G4N_OK;
}

int g4n_graph_destroy(g4n_graph *g) {
  if (!g) return G4N_OK;
  cudaSetDevice(g->ctx->device);
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  cudaFree(g->scratch);
  delete g;
  return G4N_OK;
}

}  // extern "C"
