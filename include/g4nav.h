/*
 * g4nav.h -- C ABI of the GB300 (sm_103a) Geant4-style navigation and gamma
 * transport library (libg4nav.so).
 *
 * The method is the data-parallel hot path of Seiskari, Kommeri and Niemi,
 * "GPU in Physics Computation: Case Geant4 Navigation" (arXiv:1209.5235):
 * the two navigation problems of Sec. 3.2 (locate a point in the volume
 * hierarchy; step to the next boundary) and the free-path transport of
 * Algorithm 1 (Sec. 3.1, Eqs. 1-8), extended with Compton scattering,
 * photoabsorption and per-volume energy deposits.
 *
 * Conventions
 *  - Lengths in mm, energies in MeV, attenuation coefficients in 1/mm.
 *  - Every function returns an int status: G4N_OK (0) or a negative
 *    G4N_ERR_* code; g4n_last_error() gives the context's last message.  No
 *    C++ exception crosses this boundary.
 *  - Array arguments of the query and transport calls are CALLER-OWNED
 *    DEVICE pointers (e.g. torch CUDA tensors), structure-of-arrays:
 *    a 3-vector array of n points is laid out as x[0..n), y[0..n), z[0..n).
 *    The `stream` argument is a cudaStream_t (NULL = legacy default stream).
 *    Calls are asynchronous on that stream (a transport batch on the staged
 *    schedule returns when the batch has ended); device-side errors (step caps,
 *    loop caps) are reported by the next g4n_sync() on the same stream.
 *  - The library owns the geometry tables and its workspace; g4n_destroy()
 *    frees them.  One context per host thread; one transport in flight per
 *    context at a time.
 *  - Geometry is built on the host: materials, solids and placements, then
 *    g4n_voxelize() and g4n_geom_finalize(), which validates, builds the
 *    smart-voxel candidate lists and uploads the tables.  Several geometries
 *    may be finalized in one context (the batched workload).
 */
#ifndef G4NAV_H
#define G4NAV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct g4n_ctx g4n_ctx;
typedef void *g4n_stream; /* cudaStream_t */

enum {
  G4N_OK = 0,
  G4N_ERR_ARG = -1,        /* invalid argument (null pointer, bad id, non-unit direction, bad size) */
  G4N_ERR_GEOM = -2,       /* invalid geometry (overlap, daughter outside mother, depth > G4N_DMAX) */
  G4N_ERR_OOM = -3,        /* device or host allocation failed */
  G4N_ERR_CUDA = -4,       /* a CUDA runtime call failed */
  G4N_ERR_STEP_LIMIT = -5, /* at least one track reached the per-track step cap */
  G4N_ERR_TIMEOUT = -6,    /* a device loop reached its iteration cap */
  G4N_ERR_QUEUE = -7,      /* work queue overflow */
  G4N_ERR_STATE = -8       /* call out of order (e.g. placing after finalize, query before finalize) */
};

enum { G4N_BOX = 0, G4N_TUBE = 1, G4N_ORB = 2, G4N_CONE = 3 };

/* Precision modes of compute_step / transport. */
enum {
  G4N_MODE_FP64 = 0,         /* every distance in FP64 */
  G4N_MODE_FP32_RECHECK = 1, /* FP32 intersection/safety, FP64 recheck of near-minimum candidates */
  G4N_MODE_LEARNED = 2       /* FP32_RECHECK plus the learned candidate proposal */
};

/* Limiter codes returned by g4n_compute_step. */
enum { G4N_LIM_PHYSICS = -2, G4N_LIM_MOTHER = -1 };

#define G4N_DMAX 32       /* maximum hierarchy depth, world included */
#define G4N_N_COUNTERS 32 /* length of the transport counter array */

/* Transport counters (indices into out_counters). */
enum {
  G4N_C_TRACKS = 0, G4N_C_STEPS, G4N_C_GEOM_STEPS, G4N_C_PHYS_STEPS, G4N_C_PHOTO, G4N_C_COMPTON, G4N_C_ESCAPED,
  G4N_C_CUTOFF, G4N_C_PUSHES, G4N_C_STEP_LIMIT,
  G4N_C_WALK_YIELDS = 10,    /* boundary searches that used their node budget and went on in a later round */
  G4N_C_CAND_CONE = 11,      /* DistanceToIn evaluations of cones */
  G4N_C_DIST_OUT_CURVED = 12, /* of G4N_C_DIST_OUT: those of tubes and cones */
  G4N_C_INSIDE_CURVED = 13,  /* of G4N_C_INSIDE: those of tubes and cones */
  G4N_C_FACE_RELOC = 14,     /* relocations answered by a box face's precomputed record */
  G4N_C_KEY_INSIDE = 15,     /* Inside tests of world-aligned boxes answered by exact coordinate thresholds */
  G4N_C_SAFETY_SKIPS = 16,   /* steps that skipped the boundary search because safety exceeded the physics step */
  G4N_C_CAND_BOX, G4N_C_CAND_TUBE, G4N_C_CAND_ORB, /* DistanceToIn evaluations by solid type */
  G4N_C_DIST_OUT,            /* DistanceToOut evaluations */
  G4N_C_INSIDE,              /* FP64 Inside tests (after the bounding-box prefilter) */
  G4N_C_VOX_NODES,           /* voxel nodes visited by the boundary search */
  G4N_C_RECHECKS,            /* FP64 rechecks in FP32_RECHECK mode */
  G4N_C_PROPOSALS,           /* learned proposals used */
  G4N_C_PRUNED,              /* candidates skipped by the proposal bound */
  G4N_C_CYC_REFILL = 26,     /* warp clock cycles spent refilling idle lanes (diagnostics) */
  G4N_C_CYC_INTERACT,        /* warp clock cycles spent in the interaction phase */
  G4N_C_CYC_STEP,            /* warp clock cycles spent in the step phase */
  G4N_C_STEP_LANES,          /* sum over step phases of the lanes stepping */
  G4N_C_STEP_PHASES          /* number of step phases */
};

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (>= 0), or a host-only context (device = -1) that builds,
 * validates and voxelizes geometry without touching a GPU (its queries return G4N_ERR_STATE).
 * *ctx is set to NULL on failure.  The setup that precedes the paper's benchmark program
 * (Algorithm 2); no counterpart in the paper. */
int g4n_create(g4n_ctx **ctx, int device);
/* Free every device and host resource of the context.  NULL is accepted. */
int g4n_destroy(g4n_ctx *ctx);
/* Last error message of the context ("" if none).  The string is owned by the context. */
const char *g4n_last_error(const g4n_ctx *ctx);
/* Surface tolerance = 1e-9 mm x scale (default scale 1).  Only before the first solid is added. */
int g4n_set_tolerance_scale(g4n_ctx *ctx, double scale);
/* Wait for `stream` and report any device-side error raised since the last sync. */
int g4n_sync(g4n_ctx *ctx, g4n_stream stream);
/* Kernels the context has launched so far on the device: the navigation queries, the free path,
 * every kernel of a transport batch (one per persistent launch; two per iteration and the drain
 * in the staged schedule) and one per graph replay.  A monotonic count, for measuring launch
 * rates; -1 for a null context. */
int64_t g4n_kernel_launches(const g4n_ctx *ctx);
/* Caps of the context's device loops (failure detection; the paper has no counterpart).  Every
 * loop of the kernels that is not bounded by its input is capped: the voxel walk of one boundary
 * search (default 65536 nodes) and each rejection sampler -- Kahn's method, the disc azimuth, the
 * Gaussian beam spot -- (default 1000 trials).  A kernel whose loop reaches its cap stops that loop,
 * finishes the history with what it has and raises G4N_ERR_TIMEOUT at the next g4n_sync (or in the
 * status slot of g4n_transport_batch_noalloc); results of such a run are not valid.  0 restores a
 * default; negative values give G4N_ERR_ARG.  Applies to the calls made after it. */
int g4n_set_loop_caps(g4n_ctx *ctx, int32_t max_walk_nodes, int32_t max_sampler_trials);

/* ---------------------------------------------------------------- geometry build (host) */

/* A material: density (g/cm^3) and an attenuation table of n_e >= 2 strictly increasing
 * energies with the Compton and photoabsorption linear coefficients (1/mm) at each energy.
 * Interpolated lin-lin, clamped at the ends (the mu of Eqs. 1 and 9).  Arrays are HOST
 * pointers, copied. */
int g4n_material_add(g4n_ctx *ctx, double density, int32_t n_e, const double *E_MeV, const double *mu_compton,
                     const double *mu_photo, int32_t *out_mat);

/* Solids (Sec. 3.5 uses boxes, tubes, cones and balls; this library has box, tube segment, orb
 * and full cone).  Box: half-lengths.  Tube: rmin >= 0 (0 = solid), rmax > rmin, half-length hz,
 * phi range [sphi, sphi + dphi] with 0 < dphi <= 2 pi.  Orb: a full solid sphere.  Cone: full in
 * phi, half-length hz, radii rmin1 < rmax1 at z = -hz and rmin2 < rmax2 at z = +hz varying
 * linearly in between; rmin1 and rmin2 both 0 (no inner surface) or both above the tolerance.
 * A cone's surface band is measured along r at the point's z. */
int g4n_solid_box(g4n_ctx *ctx, double hx, double hy, double hz, int32_t *out_solid);
int g4n_solid_tube(g4n_ctx *ctx, double rmin, double rmax, double hz, double sphi, double dphi, int32_t *out_solid);
int g4n_solid_orb(g4n_ctx *ctx, double r, int32_t *out_solid);
int g4n_solid_cone(g4n_ctx *ctx, double rmin1, double rmax1, double rmin2, double rmax2, double hz, int32_t *out_solid);

/* Place `solid` of material `mat` inside volume `mother` (-1 for the world, which must be the
 * first placement of a geometry).  Every placement is a distinct volume; ids are consecutive from
 * 0 (the world) within a geometry, and a daughter's id orders it among its siblings (ties in
 * locate and compute_step go to the lower id).  t: HOST pointer to the translation of the local
 * origin in the mother frame.  rot: HOST pointer to {cos theta, sin theta} of the rotation about z
 * taking local to mother coordinates, or NULL for none; it must have unit norm within 1e-12. */
int g4n_place(g4n_ctx *ctx, int32_t mother, int32_t solid, int32_t mat, const double *t, const double *rot,
              int32_t *out_vol);

/* Smart-voxel request for the geometry being built.  The paper does not describe its candidate search
 * (its port runs the isolated Geant4 navigation code, Sec. 3.3); these voxels are this library's own
 * acceleration structure, in the manner of Geant4's smart voxels, for the candidate search of the two
 * navigation problems of Sec. 3.2.  mode 0 = smart heuristic (per mother, per
 * level: slices = clamp(smartless x daughters, 1, max_slices) on the axis with the fewest
 * candidates per node, equal neighbouring nodes merged, nodes with more than refine_above
 * candidates refined on a further axis, up to 3 levels); mode 1 = fixed (n_levels levels with the
 * given axes 0/1/2 = x/y/z and slice counts, applied to every mother); mode 2 = none (one node).
 * Candidate lists are exact accelerations: results never depend on this choice. */
typedef struct {
  int32_t mode;
  int32_t n_levels;
  int32_t axes[3];
  int32_t slices[3];
  double smartless;
  int32_t max_slices;
  int32_t refine_above;
} g4n_voxel_params;
int g4n_voxelize(g4n_ctx *ctx, const g4n_voxel_params *params);

/* Logical volumes (reuse of one volume description in many places, as Geant4's logical volumes;
 * the paper's CMS geometry is built that way, Sec. 3.5).  A logical volume is a solid and a material
 * with daughters placed in its own frame.  Placing it (g4n_place_logical) expands its whole subtree
 * into physical volumes, depth first (the volume, then each daughter's subtree in the order they
 * were added), with consecutive ids: every volume id is a touchable (one physical path from the
 * world), the unit the navigation state and the tallies use.  Expansion happens on the host; the
 * device tables then hold one record per touchable.  A logical volume may not contain itself.
 * g4n_logical_add_daughter returns the daughter's copy number (its index among the logical
 * mother's daughters); a logical volume placed with g4n_place_logical has copy number 0, a volume
 * placed with g4n_place logical volume -1 and copy number -1.  t / rot: HOST pointers as for
 * g4n_place.  out_first_vol, out_n_vols: the ids [first, first + n) of the expanded volumes.
 * Logical volumes belong to the geometry being built and are discarded by g4n_geom_finalize. */
int g4n_logical_create(g4n_ctx *ctx, int32_t solid, int32_t mat, int32_t *out_lv);
int g4n_logical_add_daughter(g4n_ctx *ctx, int32_t mother_lv, int32_t daughter_lv, const double *t, const double *rot,
                             int32_t *out_copy);
int g4n_place_logical(g4n_ctx *ctx, int32_t mother_vol, int32_t lv, const double *t, const double *rot,
                      int32_t *out_first_vol, int32_t *out_n_vols);

/* Validate the volumes placed since the last finalize (every daughter inside its mother,
 * siblings not overlapping, depth <= G4N_DMAX), build the voxels and upload the tables:
 * Algorithm 2 phase 1 (load the geometry and transfer it to GPU memory).  Returns the geometry id
 * in *out_geom. */
int g4n_geom_finalize(g4n_ctx *ctx, int32_t *out_geom);

/* Table sizes of a finalized geometry (HOST array of 8): n_volumes, n_voxel_headers,
 * n_voxel_slices, n_candidate_lists, n_candidate_entries, device bytes, max depth, materials. */
int g4n_geom_info(g4n_ctx *ctx, int32_t geom, int64_t *out8);

/* The touchable path of volume `vol` of a finalized geometry: for each level from the world (0)
 * down to vol, the logical volume and copy number (-1, -1 for volumes placed with g4n_place).
 * *out_depth = number of levels; at most `cap` levels are written to the HOST arrays out_lv,
 * out_copy. */
int g4n_touchable(g4n_ctx *ctx, int32_t geom, int32_t vol, int32_t cap, int32_t *out_lv, int32_t *out_copy,
                  int32_t *out_depth);

/* ---------------------------------------------------------------- navigation queries (device) */

/* Navigation problem 1 (Sec. 3.2): the volumes containing each point.  Direction-aware: a point
 * within the tolerance band of a surface belongs to the solid iff dir points strictly inward
 * through every surface within the band.  Descends from the world, entering the first daughter in
 * placement order that contains the point.
 * pos, dir: n x 3 SoA doubles (dir of unit norm).  out_depth: n int32 (0 = outside the world,
 * 1 = world only, ...).  out_path: G4N_DMAX x n int32, level k of point i at [k * n + i], volume
 * ids from the world down, -1 below the depth. */
int g4n_locate(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir, int32_t *out_depth,
               int32_t *out_path, g4n_stream stream);

/* Navigation problem 2 (Sec. 3.2) and Algorithm 1's "next intersection": from each point inside
 * path[depth-1] (as returned by g4n_locate), the distance to the next boundary along dir, limited
 * by the proposed physics step.  out_step = min(geometric step, proposed); out_limiter = daughter
 * volume id entered, G4N_LIM_MOTHER (leaving the current volume) or G4N_LIM_PHYSICS (proposed
 * strictly shorter).  Ties: a daughter beats the mother, the lower daughter id beats a higher one,
 * geometry beats physics.  out_safety: an isotropic lower bound of the distance to any boundary.
 * proposed may be NULL (= +infinity).  mode: G4N_MODE_FP64 or G4N_MODE_FP32_RECHECK (same step
 * and limiter; the safety may be smaller).  Arrays as in g4n_locate; out_* n doubles / int32. */
int g4n_compute_step(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir,
                     const int32_t *depth, const int32_t *path, const double *proposed, double *out_step,
                     double *out_safety, int32_t *out_limiter, int32_t mode, g4n_stream stream);

/* Free path of Algorithm 1 (Sec. 3.1, Eqs. 6-7; the benchmark of Sec. 3.4, Algorithm 2 phase 5) for n rays.
 * Each ray starts at x0 along the unit direction omega.  The attenuation of a volume is its material's linear
 * coefficient (mu_compton + mu_photo, 1/mm) at `energy` (MeV), constant along a segment.  With t_j the boundary
 * crossings along the ray (t_0 = 0) and S_j the optical depth accumulated up to t_j, the result is
 * T = t_{j-1} + (Y - S_{j-1}) / mu_j for the first segment j with mu_j > 0 and S_{j-1} + mu_j (t_j - t_{j-1}) >= Y.
 * T = +inf if the ray leaves the world first or starts outside it; T = 0 if Y <= 0.  The ray only moves along its
 * line (no zero-step push); positions are x0 + t omega.
 *   pos, dir: 3 x n SoA device doubles; Y: n device doubles; out_T: n device doubles.
 *   out_steps: n device int32 (segments walked), nullable.
 *   out_counters: G4N_N_COUNTERS device uint64, accumulated (not cleared), nullable: G4N_C_TRACKS rays started,
 *     G4N_C_STEPS segments, G4N_C_GEOM_STEPS boundary crossings, G4N_C_PHYS_STEPS rays whose T is finite and > 0,
 *     G4N_C_ESCAPED rays that left the world; the diagnostic counters too with G4N_FLAG_DIAGNOSTICS in flags.
 *   mode: as g4n_compute_step.  max_steps: per-ray segment cap (0 = 10^6); a ray reaching it gets T = NaN and
 *   g4n_sync reports G4N_ERR_STEP_LIMIT.  Non-unit or non-finite directions give T = NaN and G4N_ERR_ARG at g4n_sync.
 * Rays are handed out to the warps of a persistent grid from one device queue.  Asynchronous on `stream`. */
int g4n_free_path(g4n_ctx *ctx, int32_t geom, int64_t n, const double *pos, const double *dir, const double *Y,
                  double energy, double *out_T, int32_t *out_steps, uint64_t *out_counters, int32_t mode,
                  int64_t max_steps, int32_t flags, g4n_stream stream);

/* ---------------------------------------------------------------- transport (device) */

/* Per-track source.  Every random quantity is drawn from Philox4x32-10 keyed by the 64-bit seed
 * with counter (block, track id lo, track id hi, stream 0); a block gives two uniforms in (0, 1]
 * (the top 53 bits of x1:x0 and of x3:x2, plus one, times 2^-53): a rejection trial of the spot
 * or the azimuth uses both, every single draw (z, cos theta, energy) the first of a new block.
 * Position = pos, plus a Gaussian spot of sigma spot_sigma in x and y (Marsaglia polar method) if
 * spot_sigma > 0, with z uniform in [z0, z1] if has_z.  Direction: isotropic (cos theta uniform,
 * azimuth by rejection on the unit disc) or dir.  Energy: e_kind 0 mono e0, 1 uniform [e0, e1],
 * 2 log-uniform [e0, e1]. */
typedef struct {
  double pos[3];
  double spot_sigma;
  int32_t has_z;
  double z0, z1;
  int32_t isotropic;
  double dir[3];
  int32_t e_kind;
  double e0, e1;
} g4n_source;

/* A run of n_tracks consecutive track ids starting at track_id0 in geometry `geom`.  Its deposits
 * go to columns [tally_offset, tally_offset + n_volumes + 2) of each tally row. */
typedef struct {
  int32_t geom;
  int64_t n_tracks;
  int64_t track_id0;
  g4n_source source;
  int64_t tally_offset;
} g4n_work_item;

/* A transport launch.  items: HOST array of n_items work items, processed from one device queue
 * (by the schedule below).  Physics: Algorithm 1 free paths with Y = -log W (stream 1 of the
 * track's generator), interactions Compton (Kahn's method) or photoabsorption chosen by
 * U mu_tot < mu_photo, energy below `cutoff` after a Compton scatter deposited on the spot.
 * Tally rows: track id mod n_tally_batches; tally_stride doubles per row.  max_steps: per-track
 * cap (0 = 10^6).  Launch shape (0 = defaults): block_size (multiple of 32, <= 128),
 * blocks_per_sm, refill_min (a warp refills its idle lanes once at least this many are idle,
 * 1..32, default 8), interact_min (a warp runs its interaction phase once at least this many
 * lanes wait for it, 1..32, default 8), walk_budget (voxel nodes a boundary search walks in one
 * round of its warp before it yields and continues in a later round, so that lanes with short
 * searches take their next steps meanwhile; default 16, values >= 65536 never yield and select a
 * kernel without that code), regroup_period (0 = off: every that many rounds each thread block
 * sorts its tracks by phase and solid kind of the leaf and deals them out again, so that each
 * warp runs one kind of work; every mode without diagnostics).  flags:
 * G4N_FLAG_DIAGNOSTICS also fills the diagnostic counters (G4N_C_WALK_YIELDS and above; the
 * counters below it are always filled).
 *
 * schedule: G4N_SCHEDULE_PERSISTENT (0) runs the batch in the persistent kernel described above,
 * asynchronously on the stream.  G4N_SCHEDULE_STAGED (1) keeps the tracks in flight in
 * structure-of-arrays queues in device memory and advances them in iterations of two kernels (one
 * step of every queued track, its next queue chosen by the solid kind of its leaf; then the
 * interactions and the new tracks from the source), with the last tracks of the batch finished by
 * one persistent kernel: each kernel's code is small and its warps run one kind of work.  The call
 * then returns when the batch has ended (it waits on the stream for an end flag every few
 * iterations); its device errors are reported by g4n_sync as for the persistent kernel.
 * pool_tracks: tracks in flight at most (0 = min(tracks of the batch, 2^24), halved while its queues
 * do not fit the free device memory); the library keeps 6 x pool_tracks x 172 bytes of queues
 * (10.3 GB for 10^7 tracks), grown on demand and freed by g4n_destroy; G4N_ERR_OOM if an explicit
 * pool's queues cannot be allocated.  staged_flags: G4N_STAGED_RELOCATION_KERNEL runs the relocation
 * searches after geometry-limited steps in a kernel of their own, in full warps of searching lanes
 * (it pays where most relocations need a search, as in tube segments, and costs a launch per
 * iteration where face records answer most of them, as in box cells).  drain_tracks: the persistent kernel takes over once every track has started and
 * at most this many are in flight (0 = four per resident thread of that kernel, < 0 = never).
 * The staged schedule ignores block_size (128), walk_budget (searches never yield) and
 * regroup_period; blocks_per_sm (0 = as many as fit) applies to its kernels.  Launches with
 * G4N_FLAG_DIAGNOSTICS, the sample log (g4n_mlp_log), the allocation-free entry point and CUDA
 * graphs always use the persistent kernel.  Results never depend on the schedule or the launch
 * shape. */
#define G4N_FLAG_DIAGNOSTICS 1
#define G4N_SCHEDULE_PERSISTENT 0
#define G4N_SCHEDULE_STAGED 1
#define G4N_STAGED_RELOCATION_KERNEL 1
typedef struct {
  int32_t n_items;
  const g4n_work_item *items;
  uint64_t seed;
  double cutoff;
  int32_t mode;
  int32_t n_tally_batches;
  int64_t tally_stride;
  int64_t max_steps;
  int32_t block_size;
  int32_t blocks_per_sm;
  int32_t refill_min;
  int32_t interact_min;
  int32_t flags;
  int32_t walk_budget;
  int32_t regroup_period;
  int32_t schedule;
  int32_t staged_flags;
  int64_t pool_tracks;
  int64_t drain_tracks;
} g4n_batch_desc;

/* Transport every track of the batch (Algorithm 2, phase 5).  out_edep: n_tally_batches x
 * tally_stride doubles, ACCUMULATED into (zero it first): column tally_offset + v gets the energy
 * deposited in volume v (excluding its daughters), column tally_offset + n_volumes the energy
 * that left the world, column tally_offset + n_volumes + 1 the source energy.  out_counters:
 * G4N_N_COUNTERS uint64, accumulated.  out_track_hash / out_track_len: optional (NULL) per-track
 * FNV-1a 64 hash of the step records (leaf volume after the step, limiter, event) and total path
 * length, indexed by the track's position in the concatenated items.  All DEVICE pointers. */
int g4n_transport_batch(g4n_ctx *ctx, const g4n_batch_desc *batch, double *out_edep, uint64_t *out_counters,
                        uint64_t *out_track_hash, double *out_track_len, g4n_stream stream);

/* As g4n_transport_batch, with HOST output buffers: the library zeroes its device staging
 * buffers, runs the batch on `stream`, copies the results back and synchronizes.  out_edep and
 * out_counters are overwritten (not accumulated); the hash/length outputs may be NULL. */
int g4n_transport_batch_host(g4n_ctx *ctx, const g4n_batch_desc *batch, double *out_edep, uint64_t *out_counters,
                             uint64_t *out_track_hash, double *out_track_len, g4n_stream stream);

/* ---------------------------------------------------------------- CUDA graph of a batch */

/* A batch launched repeatedly with new seeds (the same items and outputs) recorded once as a CUDA
 * graph: a node resetting the graph's own queue head, then the persistent kernel.  The items are
 * copied at creation; out_* are the DEVICE outputs every replay accumulates into (zero them between
 * replays as needed).  g4n_graph_launch replays it on `stream` with `seed`; device-side errors are
 * reported by g4n_sync of the context.  One replay in flight per graph. */
typedef struct g4n_graph g4n_graph;
int g4n_graph_create(g4n_ctx *ctx, const g4n_batch_desc *batch, double *out_edep, uint64_t *out_counters,
                     uint64_t *out_track_hash, double *out_track_len, g4n_graph **out_graph);
int g4n_graph_launch(g4n_graph *graph, uint64_t seed, g4n_stream stream);
int g4n_graph_destroy(g4n_graph *graph);

/* ---------------------------------------------------------------- learned candidate proposal */

/* A small network proposes which candidate daughter of the current voxel node the ray enters
 * first; in G4N_MODE_LEARNED that candidate is evaluated exactly before the others, and its
 * distance prunes every candidate whose rigorous FP32 lower bound exceeds it.  The network is
 * asked only where two or more of the node's candidates pass the FP32 bounds (elsewhere the
 * bounds alone leave at most one exact evaluation).  The exact
 * navigator stays the judge: results are identical in every mode.  (No counterpart in the
 * paper; part of the method's learned-proposal extension.)
 *
 * Network: 9 -> 64 -> 64 -> 32, GELU after the hidden layers, softmax over the node's first
 * n_cand <= 32 slots.  Features (9 floats per sample): the point in the node's own coordinates
 * (3, in [-1, 1]), the direction (3), (ln E[MeV] + 4.6) / 10, n_cand / 32, 1.  Label: the list
 * slot of the daughter entered.  Parameters: G4N_MLP_N_PARAMS FP32 values packed as
 * W1[9][64], b1[64], W2[64][64], b2[64], W3[64][32], b3[32] (W[k][n]: input k to output n). */
#define G4N_MLP_N_PARAMS 6880

/* Load FP32 parameters (HOST array) into the context; resets the optimizer state. */
int g4n_mlp_load(g4n_ctx *ctx, const float *params);
/* Read the current FP32 parameters into a HOST array of G4N_MLP_N_PARAMS floats. */
int g4n_mlp_get(g4n_ctx *ctx, float *params);

/* Log training samples with the plain FP64 navigator: transports the batch (batch->mode must be
 * G4N_MODE_FP64; tallies and counters are discarded) and records, for each step whose boundary
 * search entered a daughter listed in the first voxel node (2 to 32 candidates), the features,
 * the label and n_cand.  feat (capacity x 9 floats), label, ncand (capacity int32): DEVICE
 * buffers.  *out_count (HOST) = samples written (at most capacity).  Synchronous. */
int g4n_mlp_log(g4n_ctx *ctx, const g4n_batch_desc *batch, float *feat, int32_t *label, int32_t *ncand,
                int64_t capacity, int64_t *out_count, g4n_stream stream);

/* Train on n logged samples (DEVICE buffers as above) with this library's kernels: BF16
 * tensor-core GEMMs with FP32 accumulation, masked softmax cross-entropy, Adam (lr, beta
 * 0.9/0.999) on FP32 master weights.  Minibatches of `batch` (multiple of 16) per epoch from a
 * seeded permutation.  out_loss: HOST array of `epochs` mean losses, or NULL.  Synchronous. */
int g4n_mlp_train(g4n_ctx *ctx, int64_t n, const float *feat, const int32_t *label, const int32_t *ncand,
                  int32_t epochs, int32_t batch, float lr, uint64_t seed, float *out_loss, g4n_stream stream);

/* Mean loss and its gradient (HOST array of G4N_MLP_N_PARAMS) over n samples (n a multiple of
 * 16; DEVICE buffers) at the current parameters, without updating them.  precision 0: BF16
 * tensor-core GEMMs (as in training); 1: FP32 GEMMs.  Synchronous. */
int g4n_mlp_grad(g4n_ctx *ctx, int64_t n, const float *feat, const int32_t *label, const int32_t *ncand,
                 int32_t precision, float *out_grads, double *out_loss);

/* Logits (n x 32 FP32, DEVICE) of n feature rows (n x 9 FP32, DEVICE) through the same
 * warp-level BF16 inference code the transport kernel uses. */
int g4n_mlp_predict(g4n_ctx *ctx, int64_t n, const float *feat, float *out_logits, g4n_stream stream);

/* ---------------------------------------------------------------- allocation-free transport */

/* No counterpart in the paper: a library-side convenience for callers that must not allocate
 * device memory once they are running -- a process whose own allocator reserved the GPU's memory
 * up front, or a latency-critical loop that forbids cudaMalloc/cudaFree (cudaFree synchronizes the
 * whole device) after start-up.
 *
 * Same transport and arguments as g4n_transport_batch, but the queue head, status word and
 * work-item table live in one fixed device array inside libg4nav (about 43 KB, held on every GPU
 * that loads the library until the process exits) instead of the context's cudaMalloc'd
 * workspace.  The call makes no device or host heap allocation: it only clears and fills that
 * array with stream-ordered copies and launches the kernel.  (Building the geometry and creating
 * the context still allocate; do that at start-up.)
 *  - At most G4N_NOALLOC_MAX_ITEMS work items; more returns G4N_ERR_ARG.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *  - Every call shares the one array: calls whose work overlaps on the GPU (other streams, other
 *    threads, other contexts in the process) race and give wrong results.  Serialize them.
 *  - Device-side errors are not reported through g4n_sync: out_counters[G4N_NOALLOC_STATUS_SLOT] is
 *    overwritten (on `stream`) with this call's status bits -- 1 step cap reached, 2 voxel-walk
 *    cap, 4 rejection-sampling cap; 0 means no device-side error.
 * out_edep, out_counters, out_track_hash, out_track_len: DEVICE pointers as in g4n_transport_batch. */
#define G4N_NOALLOC_MAX_ITEMS 256
#define G4N_NOALLOC_STATUS_SLOT (G4N_N_COUNTERS - 1)
int g4n_transport_batch_noalloc(g4n_ctx *ctx, const g4n_batch_desc *batch, double *out_edep, uint64_t *out_counters,
                                uint64_t *out_track_hash, double *out_track_len, g4n_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* G4NAV_H */
