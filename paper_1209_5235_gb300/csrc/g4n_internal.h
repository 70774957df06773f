// g4n_internal.h -- device table layout and context of libg4nav (product code).
//
// Geometry lives in HBM as one blob per finalized geometry:
//   DVol[n]      128 B per placed volume: placement (mother -> local), solid
//                parameters, kind/flags, mother, material, voxel root, depth
//   DWorld[n]    64 B: composed world -> local transform of each volume
//   DBox32[n]    32 B: FP32 bounding box of each volume in its mother's frame,
//                rounded outward and padded (conservative prefilter for Inside)
//   DVoxHdr[]    smart-voxel headers (one per slicing level and node)
//   DVoxHdr32[]  their FP32 enclosures (the FP32 voxel walk)
//   DVoxSlice[]  per slice: child (candidate list or sub-header) and the
//                slice range [k0, k1] of the merged node it belongs to
//   DCandList[]  (offset, count) into cand[]: daughter ids in increasing id
//   materials    per material: energy grid, mu_compton, mu_photo (1/mm)
//   DKeyBox[n]   world-aligned boxes: exact world-coordinate thresholds of
//                their Inside test, as ordered integer keys of doubles
//   skey[]       per slice of a world-aligned mother: the smallest world
//                coordinate (as a key) that falls in that slice or above
//   DFace[]      6 per kKeyBox volume: relocation results across its faces
// All tables are small (a few MB at most) and stay L2-resident.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "g4nav.h"

namespace g4n {

constexpr int kDMax = G4N_DMAX;
constexpr int kMaxLevels = 3;
constexpr int kDefaultWalkCap = 1 << 16;   // voxel nodes one boundary search may walk
constexpr int kDefaultTrialCap = 1000;     // trials of one rejection sampler

enum SolidKind : int32_t { kBox = 0, kTube = 1, kOrb = 2, kCone = 3 };
// tube bits; world rotation is identity; placement rotation (mother -> local) is identity
// kKeyBox: a world-aligned box whose Inside test is answered by its DKeyBox thresholds
enum VolFlags : int32_t { kSeg = 1, kWide = 2, kHasRmin = 4, kWorldAligned = 8, kPlacedAligned = 16, kKeyBox = 32 };

struct alignas(128) DVol {
  double tx, ty, tz, c, s;  // placement: local = R(theta)^T (mother - t)
  double p[7];              // box: hx hy hz | orb: r | tube: rmin rmax hz cos(sphi) sin(sphi) cos(ephi) sin(ephi)
                            // | cone: ki ci ko co hz cos(inner half-angle) cos(outer half-angle)
  int32_t kind, flags, mother, mat;
  int32_t vox;              // root voxel header of this volume's daughters (-1: no daughters)
  int32_t depth;            // 1 for the world
  int32_t n_dau;
  int32_t face;             // first of the volume's 6 DFace records (-1: none)
};
static_assert(sizeof(DVol) == 128, "DVol must be 128 bytes");

struct alignas(64) DWorld {
  double tx, ty, tz, c, s;  // world -> local: local = R^T (world - t)
  double pad[3];
};

struct alignas(32) DBox32 {
  float lo[3], hi[3];       // in the mother frame
  int32_t keyed;            // the volume is a kKeyBox
  float pad;
};

// Exact Inside thresholds of a world-aligned box with centre t (world frame) and
// half-lengths h.  Per axis a, with p = fl(x_a - t_a) and g = fl(|p| - h_a) (the
// operations of the FP64 test), and key() the order-preserving integer image of a
// double: g > half  <=>  key(x_a) <= k[a][0] or key(x_a) >= k[a][3];
// g >= -half  <=>  key(x_a) <= k[a][1] or key(x_a) >= k[a][2].
struct alignas(32) DKeyBox {
  int64_t k[3][4];
};

// FP32 copy of a volume's placement and solid size (for conservative FP32 bounds);
// err = relative rounding allowance of the FP32 local coordinates.
struct alignas(16) DVol32 {
  float tx, ty, tz, c, s;
  float q0, q1, q2;   // box: hx hy hz | orb: r 0 0 | tube: rmin rmax hz | cone: its bounding tube
  int32_t kind, flags;
  float scale;        // |t| + extent: magnitude of the quantities involved
  float pad;
};

// Relocation across one face of a kKeyBox volume, decided on the host for a whole
// region: the face's rectangle shrunk in-plane by a margin and thickened by tol/8
// along the normal, as world-coordinate key intervals [lo, hi] per axis.  For
// every point of the region moving outward through the face (normal direction
// component of that sign, not subnormal), the relocation after leaving the volume
// (up through the mothers, down through the daughters in id order, the Inside tests
// on their keys) ends in `leaf` (-1: left the world).  ok = 0: not decided.
// Faces are numbered 2 axis + (outward direction component > 0).
struct alignas(64) DFace {
  int64_t k[3][2];
  int32_t leaf, ok;
  int32_t pad[2];
};

struct DVoxHdr {
  double lo, width, inv_width;
  int32_t axis, nslices, slice_base;
  int32_t keyed;            // the mother is world-aligned: skey[] holds this header's slice keys
  float lo_wf, inv_wf;      // FP32 slice origin in world coordinates and 1/width (for a first guess)
};

// FP32 copy of a voxel header for the FP32 voxel walk: enclosures of lo, width and
// inv_width (the floats nearest below and above each), with which every FP64 slab
// boundary and slice index of the header is bounded.
struct alignas(32) DVoxHdr32 {
  float lo_dn, lo_up, w_dn, w_up, iw_dn, iw_up;
  int32_t slice_base;
  int32_t n_axis;           // nslices << 2 | axis
};

struct DVoxSlice {
  int32_t child;            // >= 0: candidate list id; < 0: -(sub header + 1)
  int16_t k0, k1;           // slice range of the merged node
};

struct DCandList {
  int32_t offset, count;
};

// Device view of one geometry.
struct DGeom {
  const DVol *vol;
  const DWorld *wxf;
  const DBox32 *box;
  const DVol32 *v32;
  const DVoxHdr *hdr;
  const DVoxHdr32 *hdr32;
  const DVoxSlice *slice;
  const DCandList *clist;
  const int32_t *cand;
  const double *matE, *matC, *matP;
  const int32_t *mat_off, *mat_n;
  const DKeyBox *kbox;
  const int64_t *skey;
  const DFace *face;
  int32_t n_vol, n_mat;
  int32_t shared_grid;  // all materials tabulated on one energy grid
  int32_t pad;
  double tol, half;
};

// Host-side record of a solid (cone: a = rmin1, b = rmax1 at z = -c; d = rmin2, e = rmax2 at +c).
struct HSolid {
  int32_t kind;
  double a, b, c, sphi, dphi;
  double d, e;
};

struct HMat {
  double rho;
  std::vector<double> E, muC, muP;
};

struct HPlace {
  int32_t mother, solid, mat;
  double t[3], c, s;
};

struct HGeom {
  // host copies (for validation, info and tests)
  std::vector<DVol> vol;
  std::vector<DWorld> wxf;
  std::vector<DBox32> box;
  std::vector<DVol32> v32;
  std::vector<DVoxHdr> hdr;
  std::vector<DVoxHdr32> hdr32;
  std::vector<DVoxSlice> slice;
  std::vector<DCandList> clist;
  std::vector<int32_t> cand;
  std::vector<double> matE, matC, matP;
  std::vector<int32_t> mat_off, mat_n;
  std::vector<DKeyBox> kbox;
  std::vector<int64_t> skey;
  std::vector<DFace> face;
  std::vector<int32_t> touch_lv, touch_copy;  // per volume (touchable): logical volume, copy number
  int32_t max_depth = 0;
  // device blob
  void *blob = nullptr;
  size_t blob_bytes = 0;
  DGeom dview{};
};

// A logical volume: a solid and a material with daughters placed in its own frame (reused
// wherever the logical volume is placed).
struct HLogDaughter {
  int32_t lv;
  double t[3], c, s;
};
struct HLogical {
  int32_t solid, mat;
  std::vector<HLogDaughter> dau;
};

struct Builder {
  std::vector<HMat> mats;
  std::vector<HSolid> solids;
  std::vector<HPlace> places;
  std::vector<HLogical> lvs;
  // per placement: the logical volume it expands (-1: placed directly) and its copy number
  // (index among the logical mother's daughters; 0 for a logical volume placed directly)
  std::vector<int32_t> touch_lv, touch_copy;
  g4n_voxel_params vox{0, 0, {0, 1, 2}, {0, 0, 0}, 2.0, 1000, 4};
  bool vox_set = false;
  void clear() {
    mats.clear();
    solids.clear();
    places.clear();
    lvs.clear();
    touch_lv.clear();
    touch_copy.clear();
    vox_set = false;
  }
};

}  // namespace g4n

struct g4n_ctx {
  int device = 0;
  std::string err;
  double scale = 1.0;
  // device loop caps (g4n_set_loop_caps): beyond them a kernel stops the loop and reports G4N_ERR_TIMEOUT
  int walk_cap = g4n::kDefaultWalkCap;
  int trial_cap = g4n::kDefaultTrialCap;
  double tol = 1e-9, half = 0.5e-9;
  g4n::Builder b;
  std::vector<g4n::HGeom *> geoms;
  // device geometry directory (DGeom per geometry id), grown on finalize
  g4n::DGeom *d_geoms = nullptr;
  int d_geoms_cap = 0;
  // transport workspace: queue head and status word (allocated once, never moved: graphs keep
  // its status word), and the device item table (grown by doubling)
  void *ws = nullptr;
  void *items = nullptr;
  size_t items_bytes = 0;
  // host staging for g4n_transport_batch_host
  void *h_stage = nullptr;
  size_t h_stage_bytes = 0;
  void *d_stage = nullptr;
  size_t d_stage_bytes = 0;
  // device buffers outgrown while work may still read them: freed by g4n_destroy (growth by
  // doubling bounds them by the live size), so that growing never synchronizes the device
  std::vector<void *> retired;
  // staged transport: its track-state queues behind a control block (grown by doubling, the
  // outgrown ones retired), two pinned end flags and two events (cudaEvent_t) of the chunks in flight
  void *stage_q = nullptr;
  size_t stage_q_bytes = 0;
  int *stage_flag = nullptr;
  void *stage_ev[2] = {nullptr, nullptr};
  int sm_count = 0;
  int64_t launches = 0;  // kernels launched (g4n_kernel_launches)
  // candidate-proposal MLP state (owned by mlp.cu)
  void *mlp = nullptr;
};

// error helpers shared by the translation units
int g4n_fail(g4n_ctx *ctx, int code, const std::string &msg);

namespace g4n {
namespace mlp {
struct SmemWeights;
}
}  // namespace g4n
// Device image of the loaded MLP weights (null if none) and its release.
const g4n::mlp::SmemWeights *g4n_mlp_image(g4n_ctx *ctx);
void g4n_mlp_free(g4n_ctx *ctx);
