// transport_staged.cuh -- the staged schedule of the transport (included once, by nav_kernels.cu,
// after the persistent kernel whose per-track device functions it reuses).
//
// The persistent kernel keeps every track in a lane's registers for its whole history and runs
// the source, step and interaction code of Algorithm 1 in one loop.  On GB300 that loop is bound
// by latency: its code does not fit the instruction caches, and a warp's lanes diverge across
// the phases.  The staged schedule keeps the tracks in flight in HBM instead, as structure-of-arrays
// queues, and advances them in iterations of two kernels:
//
//   step    every queued track takes one step (Sec. 3.2 problem 2, Eq. 7): the geometric step
//           with its voxel walk, the move, the relocation.  The tracks that go on stepping are
//           written to the next iteration's queue of their leaf's solid kind (box, tube, orb,
//           cone), so that each warp of the next step kernel runs one kind of geometry; the
//           tracks whose free path ended go to the interaction queue.
//   finish  the interactions (Compton by Kahn's method or photoabsorption, the cutoff, a new
//           free path), then new tracks from the source (located in the world) up to the number
//           in flight, both written to the next step queues.
//
// Each kernel is small enough for the instruction caches and its warps are full (the queues are
// compact); the cost is one load and one store of a track's state (168 B) per step and per
// interaction (and per deferred relocation), from HBM/L2 at full coalescing.  Every history is the
// same as in the persistent kernel (the same device functions advance a track; the order of steps
// within a history is fixed), so results do not depend on the schedule.
//
// With G4N_STAGED_RELOCATION_KERNEL a third kernel runs between the two: the step kernel queues the
// steps whose relocation needs a search (not answered by a face record), and the relocation kernel
// runs those searches in full warps.
//
// The last tracks of a batch (fewer than drain_tracks in flight, no new ones left) are finished
// by one persistent kernel that takes them from the queue: an iteration costs at least the
// longest single step among its tracks, which is what a few long histories would otherwise pay
// per step.
//
// Control: a small device block (counts per queue, the source queue head, the tracks in flight)
// updated by the last block of each kernel to finish (a fence and an atomic counter of finished
// blocks); every decision (admission, the drain, the end) is taken there, so the host only
// launches iterations and reads the end flag of a chunk of iterations while the next chunk runs.

namespace {

constexpr int kSgKinds = 4;                 // solid kinds (box, tube, orb, cone)
constexpr int kSgQueues = 2 * kSgKinds + 2; // step queues of two banks, the interaction and the relocation queue
constexpr int kSgInteract = 2 * kSgKinds;
constexpr int kSgReloc = 2 * kSgKinds + 1;
constexpr int kSgArrays = 6;                // queue arrays of `pool` entries (see sg_entry)
constexpr int kSgDoubles = 16, kSgInts = 7; // the seventh int: a deferred relocation's limiter and exit flag
constexpr int kSgChunk = 8;                 // iterations launched between reads of the end flag

// Track-state queues, structure of arrays: field f of entry e at base_f[e].
struct SgQueues {
  double *d;       // kSgDoubles fields x n: x, u, 1/u, E, Y, len, safety, mu, mu_photo, bin fraction
  uint64_t *h;     // history hash
  int64_t *tid;    // track id
  int32_t *iw;     // kSgInts fields x n: leaf, item, steps, zero steps, energy bin, draw counter, relocation aux
  int64_t n;       // entries per field (kSgArrays x pool)
  int64_t pool;    // tracks in flight at most
};

// Bytes of track state per queue entry.
constexpr size_t kSgEntryBytes = (size_t)kSgDoubles * 8 + 2 * 8 + (size_t)kSgInts * 4;

struct SgCtrl {
  unsigned long long cnt[kSgQueues];  // entries per queue
  unsigned long long q_head;          // next track of the batch to start
  long long active;                   // tracks in flight
  long long n_new, base;              // admission of the current iteration: tracks [base, base + n_new)
  unsigned int fin[4];                // blocks finished per kernel (step, finish, drain, relocation)
  int done;                           // every track has ended
  int drain_now, drain_bank;          // the drain kernel takes the tracks of this bank
  long long iterations;               // iterations ended (a count for debugging; the host keeps its own)
  unsigned long long drain_head;      // drain kernel: next queue entry to take
  unsigned long long pad[4];
};

// Entry of queue q (0 <= q < kSgQueues) at position j.  A bank's four kind queues share two
// arrays of `pool` entries, one queue filling each array from the front and one from the back:
// the tracks of a bank are never more than `pool`, so no two queues of an array can meet.
__device__ __forceinline__ int64_t sg_entry(const SgQueues &Q, int q, long long j) {
  if (q == kSgInteract) return 4 * Q.pool + j;
  if (q == kSgReloc) return 5 * Q.pool + j;
  const int64_t a = (int64_t)(q >> 1) * Q.pool;  // bank b, kind k: array 2b + (k >> 1)
  return (q & 1) ? a + Q.pool - 1 - j : a + j;
}

__device__ __forceinline__ void sg_load(const SgQueues &Q, int64_t e, Track &t) {
  const double *d = Q.d + e;
  const int64_t n = Q.n;
  t.x.x = __ldcs(d + 0 * n); t.x.y = __ldcs(d + 1 * n); t.x.z = __ldcs(d + 2 * n);
  t.u.x = __ldcs(d + 3 * n); t.u.y = __ldcs(d + 4 * n); t.u.z = __ldcs(d + 5 * n);
  t.iu.x = __ldcs(d + 6 * n); t.iu.y = __ldcs(d + 7 * n); t.iu.z = __ldcs(d + 8 * n);
  t.E = __ldcs(d + 9 * n); t.Y = __ldcs(d + 10 * n); t.len = __ldcs(d + 11 * n); t.safety = __ldcs(d + 12 * n);
  t.mu = __ldcs(d + 13 * n); t.mupe = __ldcs(d + 14 * n); t.efrac = __ldcs(d + 15 * n);
  t.h = __ldcs(Q.h + e);
  t.tid = __ldcs(Q.tid + e);
  const int32_t *w = Q.iw + e;
  t.leaf = __ldcs(w + 0 * n); t.item = __ldcs(w + 1 * n); t.steps = __ldcs(w + 2 * n); t.nzero = __ldcs(w + 3 * n);
  t.ebin = __ldcs(w + 4 * n); t.draw = (uint32_t)__ldcs(w + 5 * n);
}

__device__ __forceinline__ void sg_store(const SgQueues &Q, int64_t e, const Track &t) {
  double *d = Q.d + e;
  const int64_t n = Q.n;
  d[0 * n] = t.x.x; d[1 * n] = t.x.y; d[2 * n] = t.x.z;
  d[3 * n] = t.u.x; d[4 * n] = t.u.y; d[5 * n] = t.u.z;
  d[6 * n] = t.iu.x; d[7 * n] = t.iu.y; d[8 * n] = t.iu.z;
  d[9 * n] = t.E; d[10 * n] = t.Y; d[11 * n] = t.len; d[12 * n] = t.safety;
  d[13 * n] = t.mu; d[14 * n] = t.mupe; d[15 * n] = t.efrac;
  Q.h[e] = t.h;
  Q.tid[e] = t.tid;
  int32_t *w = Q.iw + e;
  w[0 * n] = t.leaf; w[1 * n] = t.item; w[2 * n] = t.steps; w[3 * n] = t.nzero; w[4 * n] = t.ebin;
  w[5 * n] = (int32_t)t.draw;
}

// The track's position in the concatenated items (its hash / length output slot).
__device__ __forceinline__ void sg_restore_gidx(const TParams &P, Track &t) {
  const DItem &it = P.items[t.item];
  t.gidx = it.start + (t.tid - it.tid0);
}

// Append the lanes with `want` to queue q (per lane): one atomic per distinct queue of the warp
// (warp-collective).
__device__ __forceinline__ void sg_push(const SgQueues &Q, SgCtrl *C, bool want, int q, const Track &t) {
  if (!__any_sync(kFull, want)) return;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(kFull, want ? q : -1);
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (want && (int)lane == leader) base = atomicAdd(&C->cnt[q], (unsigned long long)__popc(peers));
  base = __shfl_sync(kFull, base, leader);
  if (want) sg_store(Q, sg_entry(Q, q, (long long)base + __popc(peers & ((1u << lane) - 1u))), t);
}

// Block-wide append (every thread of the block calls it, with the block's warps converged): the warps count
// their lanes per queue in shared memory, one thread per queue reserves the block's slots with one global
// atomic, and every lane stores at its slot.  The step kernel appends this way: one global atomic per queue
// per block of 128 tracks instead of per warp, and its loop over the queue runs in block-sized strides.
__shared__ unsigned s_qcount[kSgQueues];
__shared__ unsigned long long s_qbase[kSgQueues];

__device__ __forceinline__ int64_t sg_push_block(const SgQueues &Q, SgCtrl *C, bool want, int q, const Track &t) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(kFull, want ? q : -1);
  const int leader = __ffs(peers) - 1;
  unsigned woff = 0;
  if (want && (int)lane == leader) woff = atomicAdd(&s_qcount[q], (unsigned)__popc(peers));
  woff = __shfl_sync(kFull, woff, leader);
  __syncthreads();
  if (threadIdx.x < kSgQueues) {
    const unsigned c = s_qcount[threadIdx.x];
    s_qbase[threadIdx.x] = c ? atomicAdd(&C->cnt[threadIdx.x], (unsigned long long)c) : 0ull;
    s_qcount[threadIdx.x] = 0;  // ready for the next call (the barrier below orders it before any new count)
  }
  __syncthreads();
  int64_t e = -1;
  if (want) {
    e = sg_entry(Q, q, (long long)(s_qbase[q] + woff + __popc(peers & ((1u << lane) - 1u))));
    sg_store(Q, e, t);
  }
  return e;  // the lane's queue entry (-1: none)
}

// Step queue of bank b for the track's leaf.
__device__ __forceinline__ int sg_queue_of(const TParams &P, const Track &t, int b) {
  return b * kSgKinds + P.geoms[P.items[t.item].geom].vol[t.leaf].kind;
}

// The warp's tracks that ended leave the count in flight.
__device__ __forceinline__ void sg_retire(SgCtrl *C, bool ended) {
  const unsigned m = __ballot_sync(kFull, ended);
  if (m && (threadIdx.x & 31u) == 0) atomicAdd((unsigned long long *)&C->active, (unsigned long long)(-(long long)__popc(m)));
}

// The block's event counts (shared) and the lanes' step counts (registers) into the batch's counters.
__device__ __forceinline__ void sg_flush(const TParams &P, Counters &cnt) {
  cnt.c[G4N_C_STEPS] = cnt.c[G4N_C_GEOM_STEPS] + cnt.c[G4N_C_PHYS_STEPS];
  __syncthreads();
  for (int k = threadIdx.x; k < G4N_N_COUNTERS; k += blockDim.x)
    if (s_events[k]) atomicAdd(&P.counters[k], s_events[k]);
#pragma unroll
  for (int k = 0; k < G4N_N_COUNTERS; ++k) {
    unsigned long long v = cnt.c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd(&P.counters[k], v);
  }
}

__device__ __forceinline__ void sg_begin(Counters &cnt) {
#pragma unroll
  for (int k = 0; k < G4N_N_COUNTERS; ++k) cnt.c[k] = 0;
  for (int k = threadIdx.x; k < G4N_N_COUNTERS; k += blockDim.x) s_events[k] = 0;
  if (threadIdx.x < kSgQueues) s_qcount[threadIdx.x] = 0;
  __syncthreads();
}

// True in the block of the grid that finishes last (the writes of all other blocks are then
// visible to it); it resets the kernel's finished-block count for the next launch.
__device__ __forceinline__ bool sg_last_block(SgCtrl *C, int which) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&C->fin[which], 1u) == gridDim.x - 1;
    if (last) C->fin[which] = 0;
  }
  __syncthreads();
  return last;
}

// The learned mode's weights in shared memory (the first bytes of the dynamic shared memory) and
// this warp's scratch tile; other modes: none.
template <int MODE>
__device__ __forceinline__ MlpCtx sg_mlp(const TParams &P) {
  MlpCtx mc{nullptr, nullptr, nullptr, 0.f};
  if (MODE == kLearned) {
    extern __shared__ __align__(16) unsigned char smem[];
    mlp::SmemWeights *sw = reinterpret_cast<mlp::SmemWeights *>(smem);
    mlp::load_weights(*sw, P.mlp_w);
    __syncthreads();
    mc.w = sw;
    mc.scratch = reinterpret_cast<mlp::SmemWarp *>(smem + sizeof(mlp::SmemWeights)) + (threadIdx.x >> 5);
  }
  return mc;
}

// Entries of the four step queues of bank b: prefix sums in shared memory.
__device__ __forceinline__ long long sg_prefix(const SgCtrl *C, int b, long long *pref) {
  if (threadIdx.x == 0) {
    const volatile SgCtrl *V = C;
    long long acc = 0;
    pref[0] = 0;
#pragma unroll
    for (int k = 0; k < kSgKinds; ++k) {
      acc += (long long)V->cnt[b * kSgKinds + k];
      pref[k + 1] = acc;
    }
  }
  __syncthreads();
  return pref[kSgKinds];
}

// Step kernel of iteration (ib: the bank read, the other bank written).  Its last block admits
// the next tracks of the batch: as many as the tracks in flight leave room for in the pool.
// RELOC_KERNEL: a step that needs a relocation search (not answered by a face record) is queued for the
// relocation kernel instead of searching here, with its limiter and exit flag in the entry's aux int.
template <int MODE, bool RELOC_KERNEL>
__global__ void __launch_bounds__(128, 4) k_staged_step(const TParams P, const SgQueues Q, SgCtrl *C, int ib) {
  if (((const volatile SgCtrl *)C)->drain_now || ((const volatile SgCtrl *)C)->done) return;
  Counters cnt;
  sg_begin(cnt);
  const MlpCtx mc = sg_mlp<MODE>(P);
  __shared__ long long pref[kSgKinds + 1];
  const long long total = sg_prefix(C, ib, pref);
  const int ob = ib ^ 1;
  const bool want_slot = P.out_hash || P.out_len;
  // block-sized strides: the loop condition is the same for every thread of the block (sg_push_block's barriers)
#pragma unroll 1
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < total; b0 += (long long)gridDim.x * blockDim.x) {
    const long long i = b0 + threadIdx.x;
    Track t;
    t.item = 0;
    t.leaf = 0;
    int phase = kEmpty;
    if (i < total) {
      int k = 0;
#pragma unroll
      for (int s = 1; s < kSgKinds; ++s) k += i >= pref[s];
      sg_load(Q, sg_entry(Q, ib * kSgKinds + k, i - pref[k]), t);
      if (want_slot) sg_restore_gidx(P, t);
      phase = kStep;
    }
    Chain ch;
    int aux = 0;
    const int next = step_warp<MODE, false, false, true, RELOC_KERNEL>(P, t, phase, cnt, mc, ch, &aux);
    const bool was = phase == kStep;
    const bool keep = was && next != kEmpty;
    const int q = !keep ? 0 : next == kStep ? sg_queue_of(P, t, ob) : next == kReloc ? kSgReloc : kSgInteract;
    const int64_t e = sg_push_block(Q, C, keep, q, t);
    if (RELOC_KERNEL && keep && next == kReloc) Q.iw[6 * Q.n + e] = aux;
    sg_retire(C, was && next == kEmpty);
  }
  sg_flush(P, cnt);
  if (sg_last_block(C, 0) && threadIdx.x == 0) {
    volatile SgCtrl *V = C;
    const long long active = V->active;
    const long long left = P.total - (long long)V->q_head;
    long long n_new = Q.pool - active < left ? Q.pool - active : left;
    if (n_new < 0) n_new = 0;
    V->base = (long long)V->q_head;
    V->n_new = n_new;
    V->q_head = V->q_head + (unsigned long long)n_new;
    V->active = active + n_new;
    __threadfence();
  }
}

// Relocation kernel of the iteration (the option G4N_STAGED_RELOCATION_KERNEL): the steps whose relocation
// search the step kernel deferred, in full warps of searching lanes (in the step kernel a warp's lanes limited
// by physics or answered by a face record wait while the others search); then the push after ten zero
// steps and the step record, as the step kernel would have done them, and the tracks go on to bank ob.  Its
// last block empties the queue.  8 blocks of 128 per SM (64 registers): the searches wait on chains of
// dependent table loads, and more resident warps hide them (barrel 10^7: 2.4 % of the batch against 4 blocks
// at 128 registers, 6 blocks in between).
template <int MODE>
__global__ void __launch_bounds__(128, 8) k_staged_reloc(const TParams P, const SgQueues Q, SgCtrl *C, int ib) {
  const volatile SgCtrl *V0 = C;
  if (V0->drain_now || V0->done) return;
  Counters cnt;
  sg_begin(cnt);
  const long long total = (long long)V0->cnt[kSgReloc];
  const int ob = ib ^ 1;
  const bool want_slot = P.out_hash || P.out_len;
  // block-sized strides: the loop condition is the same for every thread of the block (sg_push_block's barriers)
#pragma unroll 1
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < total; b0 += (long long)gridDim.x * blockDim.x) {
    const long long i = b0 + threadIdx.x;
    const bool act = i < total;
    Track t;
    t.item = 0;
    t.leaf = 0;
    int aux = 0;
    if (act) {
      const int64_t e = sg_entry(Q, kSgReloc, i);
      sg_load(Q, e, t);
      aux = __ldcs(Q.iw + 6 * Q.n + e);
      if (want_slot) sg_restore_gidx(P, t);
    }
    const DGeom &G = P.geoms[P.items[act ? t.item : 0].geom];
    // every lane searches (the step kernel already counted the zero step); aux = limiter << 1 | left the leaf
    const int next = reloc_tail<MODE, false, true>(P, G, t, act, act, -1, (aux & 1) != 0, 0.0, aux >> 1, false, cnt,
                                                   kEmpty);
    const bool keep = act && next == kStep;
    sg_push_block(Q, C, keep, keep ? sg_queue_of(P, t, ob) : 0, t);
    sg_retire(C, act && next == kEmpty);
  }
  sg_flush(P, cnt);
  if (sg_last_block(C, 3) && threadIdx.x == 0) {
    ((volatile SgCtrl *)C)->cnt[kSgReloc] = 0;
    __threadfence();
  }
}

// Finish kernel of the iteration: the interaction queue, then the admitted new tracks, all
// written to bank ob.  Its last block ends the iteration: the queues just read are emptied, and it
// decides the end of the batch or the hand-over of the last tracks to the drain kernel.
template <int MODE>
__global__ void __launch_bounds__(128, 4) k_staged_finish(const TParams P, const SgQueues Q, SgCtrl *C, int ib,
                                                           long long drain_tracks) {
  const volatile SgCtrl *V0 = C;
  if (V0->drain_now || V0->done) return;
  Counters cnt;
  sg_begin(cnt);
  const long long n_int = (long long)V0->cnt[kSgInteract], n_new = V0->n_new, g0 = V0->base;
  const long long total = n_int + n_new;
  const int ob = ib ^ 1;
  const bool want_slot = P.out_hash || P.out_len;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
#pragma unroll 1
  for (long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < total; w += nw) {
    const long long i = w * 32 + (threadIdx.x & 31u);
    const bool is_int = i < n_int, is_new = !is_int && i < total;
    Track t;
    t.item = 0;
    t.leaf = 0;
    int next = kEmpty;
    if (is_int) {
      sg_load(Q, sg_entry(Q, kSgInteract, i), t);
      if (want_slot) sg_restore_gidx(P, t);
      next = interact<MODE, true>(P, t, cnt);
    }
    if (__any_sync(kFull, is_new)) {  // the source and the locate (warp-collective)
      const int started = start_warp<MODE, false, true>(P, is_new, g0 + (i - n_int), t, cnt);
      if (is_new) next = started;
    }
    const bool mine = is_int || is_new;
    sg_push(Q, C, mine && next == kStep, mine && next == kStep ? sg_queue_of(P, t, ob) : 0, t);
    sg_retire(C, mine && next == kEmpty);
  }
  sg_flush(P, cnt);
  if (sg_last_block(C, 1) && threadIdx.x == 0) {
    volatile SgCtrl *V = C;
    V->cnt[kSgInteract] = 0;
#pragma unroll
    for (int k = 0; k < kSgKinds; ++k) V->cnt[ib * kSgKinds + k] = 0;
    V->n_new = 0;
    V->iterations = V->iterations + 1;
    const bool all_started = (long long)V->q_head >= P.total;
    const long long active = V->active;
    if (all_started && active == 0) {
      V->done = 1;
    } else if (all_started && active <= drain_tracks) {
      V->drain_now = 1;
      V->drain_bank = ob;
      V->drain_head = 0;
    }
    __threadfence();
  }
}

// The drain: a persistent kernel (the loop of k_transport without sources) over the tracks of
// the bank the last iteration wrote; a warp refills its idle lanes from that bank.
template <int MODE>
__global__ void __launch_bounds__(128, 4) k_staged_drain(const TParams P, const SgQueues Q, SgCtrl *C) {
  const volatile SgCtrl *V0 = C;
  if (!V0->drain_now || V0->done) return;
  Counters cnt;
  sg_begin(cnt);
  const MlpCtx mc = sg_mlp<MODE>(P);
  const int bank = V0->drain_bank;
  __shared__ long long pref[kSgKinds + 1];
  const long long total = sg_prefix(C, bank, pref);
  const bool want_slot = P.out_hash || P.out_len;
  const unsigned lane = threadIdx.x & 31u;
  Track t;
  t.item = 0;
  t.leaf = 0;
  Chain ch;
  int phase = kEmpty;
  bool drained = false;
#pragma unroll 1
  for (;;) {
    const unsigned idle = __ballot_sync(kFull, phase == kEmpty);
    if (idle && !drained) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if ((int)lane == leader) base = atomicAdd(&C->drain_head, (unsigned long long)__popc(idle));
      base = __shfl_sync(kFull, base, leader);
      if (base + __popc(idle) >= (unsigned long long)total) drained = true;
      const long long g = (long long)base + __popc(idle & ((1u << lane) - 1u));
      if (phase == kEmpty && g < total) {
        int k = 0;
#pragma unroll
        for (int s = 1; s < kSgKinds; ++s) k += g >= pref[s];
        sg_load(Q, sg_entry(Q, bank * kSgKinds + k, g - pref[k]), t);
        if (want_slot) sg_restore_gidx(P, t);
        phase = kStep;
      }
    }
    const unsigned waiting = __ballot_sync(kFull, phase == kInteract);
    const unsigned stepping = __ballot_sync(kFull, phase == kStep);
    if (waiting && (__popc(waiting) >= P.interact_min || stepping == 0)) {
      if (phase == kInteract) phase = interact<MODE, true>(P, t, cnt);
    }
    __syncwarp();
    phase = step_warp<MODE, false, false, true>(P, t, phase, cnt, mc, ch);
    if (drained && __ballot_sync(kFull, phase != kEmpty) == 0) break;
  }
  sg_flush(P, cnt);
  if (sg_last_block(C, 2) && threadIdx.x == 0) {
    volatile SgCtrl *V = C;
#pragma unroll
    for (int k = 0; k < kSgKinds; ++k) V->cnt[bank * kSgKinds + k] = 0;
    V->active = 0;
    V->drain_now = 0;
    V->done = 1;
    __threadfence();
  }
}

}  // namespace

// ---------------------------------------------------------------- host side

namespace {

constexpr int64_t kSgDefaultPool = int64_t(1) << 24;

// Blocks of 128 per SM for a staged kernel: b->blocks_per_sm, else as many as fit.
template <typename K>
int sg_grid(g4n_ctx *ctx, const g4n_batch_desc *b, K kern, size_t smem) {
  int per_sm = b->blocks_per_sm;
  if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (per_sm <= 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
    per_sm = std::max(per_sm, 1);
  }
  return ctx->sm_count * per_sm;
}

// Run a validated batch (P as for the persistent kernel, its items uploaded) on the staged
// schedule; returns when the batch has ended on `st`.
template <int MODE>
int staged_run(g4n_ctx *ctx, const g4n_batch_desc *b, TParams &P, cudaStream_t st) {
  if (b->pool_tracks < 0) return g4n_fail(ctx, G4N_ERR_ARG, "transport: pool_tracks must be >= 0");
  int64_t pool = std::max<int64_t>(1, std::min<int64_t>(b->pool_tracks > 0 ? b->pool_tracks : kSgDefaultPool, P.total));
  const size_t ctrl_bytes = 1024;
  auto queue_bytes = [&](int64_t n) { return ctrl_bytes + (size_t)kSgArrays * (size_t)n * kSgEntryBytes; };
  if (ctx->stage_q_bytes < queue_bytes(pool)) {
    // grow by up to half again (batches of slowly growing size do not reallocate every call); the default pool
    // halves until its queues fit the free device memory, an explicit pool does not
    void *p = nullptr;
    size_t got = 0;
    for (;;) {
      const size_t need = queue_bytes(pool);
      const size_t want = std::max(need, std::min(2 * ctx->stage_q_bytes, need + need / 2));
      if (cudaMalloc(&p, want) == cudaSuccess) {
        got = want;
        break;
      }
      cudaGetLastError();
      if (want > need && cudaMalloc(&p, need) == cudaSuccess) {
        got = need;
        break;
      }
      cudaGetLastError();
      p = nullptr;
      if (b->pool_tracks > 0 || pool <= (int64_t(1) << 16))
        return g4n_fail(ctx, G4N_ERR_OOM, "transport: staged queue allocation failed (lower pool_tracks)");
      pool /= 2;
      if (ctx->stage_q_bytes >= queue_bytes(pool)) break;  // the queues held already suffice
    }
    if (p) {
      if (ctx->stage_q) ctx->retired.push_back(ctx->stage_q);
      ctx->stage_q = p;
      ctx->stage_q_bytes = got;
    }
  }
  if (!ctx->stage_flag) {
    if (cudaMallocHost(&ctx->stage_flag, 2 * sizeof(int)) != cudaSuccess) {
      ctx->stage_flag = nullptr;
      return g4n_fail(ctx, G4N_ERR_OOM, "transport: pinned flag allocation failed");
    }
    for (auto &e : ctx->stage_ev) {
      cudaEvent_t ev;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return g4n_fail(ctx, G4N_ERR_CUDA, "transport: event creation failed");
      e = ev;
    }
  }
  // queues: one array per field, kSgArrays x pool entries each (see sg_entry)
  char *m = (char *)ctx->stage_q;
  SgCtrl *C = (SgCtrl *)m;
  SgQueues Q;
  Q.pool = pool;
  Q.n = (int64_t)kSgArrays * pool;
  size_t off = ctrl_bytes;
  Q.d = (double *)(m + off);
  off += (size_t)Q.n * kSgDoubles * sizeof(double);
  Q.h = (uint64_t *)(m + off);
  off += (size_t)Q.n * sizeof(uint64_t);
  Q.tid = (int64_t *)(m + off);
  off += (size_t)Q.n * sizeof(int64_t);
  Q.iw = (int32_t *)(m + off);
  static_assert(sizeof(SgCtrl) <= 1024, "control block");

  const size_t smem = mlp_smem_bytes(b->mode, 128);
  P.mlp_w = g4n_mlp_image(ctx);
  const bool reloc_kernel = (b->staged_flags & G4N_STAGED_RELOCATION_KERNEL) != 0;
  const int g_step = reloc_kernel ? sg_grid(ctx, b, k_staged_step<MODE, true>, smem)
                                  : sg_grid(ctx, b, k_staged_step<MODE, false>, smem);
  const int g_reloc = sg_grid(ctx, b, k_staged_reloc<MODE>, 0);
  const int g_fin = sg_grid(ctx, b, k_staged_finish<MODE>, 0);
  int per_sm_drain = 0;
  if (smem) cudaFuncSetAttribute(k_staged_drain<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_drain, k_staged_drain<MODE>, 128, smem);
  const int g_drain = ctx->sm_count * std::max(per_sm_drain, 1);
  const long long drain_tracks = b->drain_tracks < 0 ? -1
                                 : b->drain_tracks > 0 ? b->drain_tracks
                                                       : 4LL * g_drain * 128;
  if (cudaMemsetAsync(C, 0, sizeof(SgCtrl), st) != cudaSuccess) return g4n_fail(ctx, G4N_ERR_CUDA, "transport: control reset failed");
  if (int rc = launch_error(ctx, "staged transport setup")) return rc;

  // every iteration advances each track in flight by one step: a batch ends within
  // (max_steps + 2) iterations of its last admission, and admissions never stall longer
  const long long max_iter = ((long long)(P.total / pool) + 2) * ((long long)P.max_steps + 2) + 64;
  int *flag = ctx->stage_flag;
  cudaEvent_t ev[2] = {(cudaEvent_t)ctx->stage_ev[0], (cudaEvent_t)ctx->stage_ev[1]};
  long long it = 0;
  for (long long chunk = 0;; ++chunk) {
    for (int j = 0; j < kSgChunk; ++j, ++it) {
      const int ib = (int)(it & 1);
      if (reloc_kernel) {
        k_staged_step<MODE, true><<<g_step, 128, smem, st>>>(P, Q, C, ib);
        k_staged_reloc<MODE><<<g_reloc, 128, 0, st>>>(P, Q, C, ib);
        ++ctx->launches;
      } else {
        k_staged_step<MODE, false><<<g_step, 128, smem, st>>>(P, Q, C, ib);
      }
      k_staged_finish<MODE><<<g_fin, 128, 0, st>>>(P, Q, C, ib, drain_tracks);
      ctx->launches += 2;
    }
    if (drain_tracks >= 0) {
      k_staged_drain<MODE><<<g_drain, 128, smem, st>>>(P, Q, C);
      ++ctx->launches;
    }
    if (cudaMemcpyAsync(&flag[chunk & 1], &C->done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(ev[chunk & 1], st) != cudaSuccess)
      return g4n_fail(ctx, G4N_ERR_CUDA, "transport: staged end-flag read failed");
    if (int rc = launch_error(ctx, "staged transport launch")) return rc;
    // the previous chunk's flag, read while this chunk runs
    if (chunk > 0) {
      if (cudaEventSynchronize(ev[(chunk - 1) & 1]) != cudaSuccess) return launch_error(ctx, "staged transport");
      if (flag[(chunk - 1) & 1]) break;
    }
    if (it > max_iter) {
      cudaStreamSynchronize(st);
      return g4n_fail(ctx, G4N_ERR_STATE, "transport: staged schedule did not end");
    }
  }
  return G4N_OK;
}

int staged_transport(g4n_ctx *ctx, const g4n_batch_desc *b, TParams &P, cudaStream_t st) {
  if (b->mode == G4N_MODE_FP64) return staged_run<kFP64>(ctx, b, P, st);
  if (b->mode == G4N_MODE_FP32_RECHECK) return staged_run<kFP32>(ctx, b, P, st);
  return staged_run<kLearned>(ctx, b, P, st);
}

}  // namespace
