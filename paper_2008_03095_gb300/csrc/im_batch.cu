// Batched persistent launch: many independent select queries (each its own
// graph, K, R, p, options) in one kernel launch, each query running the
// INFuseR-MG steps of Algorithm 7 (lane randoms, label init, fused sample +
// union, size memo, first gains, lazy greedy).
//
// Work is a list of items (query, phase, tile) ordered by phase: every item of
// an earlier phase of a query comes before the items that depend on it. Each
// block of the launch takes the next item from an atomic counter, waits (one
// thread, with an iteration budget) until the phases the item depends on have
// counted all their items done, runs it, and counts it done. An item only ever
// waits on items taken before it, and those are held by running blocks, so
// the launch makes progress whatever the number of co-resident blocks (it is
// an ordinary launch, and a CUDA graph can capture it). Data written by
// another block of the same launch is read through L2 (coherent loads).
//
// Phases and their tiles, each sized by the query's tiling (chosen by the
// autotuner, see im_batch_autotune):
//   lanes     one item: X_r, lane order and bucket offsets (one block)
//   init      label slots [t*c, (t+1)*c) set to -1, covered bits cleared
//   union     upper edges [t*c, (t+1)*c): hash, candidate lanes, union-find
//   compress  c size-memo tiles of 32 vertices x 32 lanes, four at a time
//   gains     vertices [t*c, (t+1)*c): mg_v and its key
//   celf      one item: the lazy greedy of the query in one block, with
//             block-local prefix extraction and bound refreshes
#include "im_celf.cuh"
#include "im_lanes.cuh"
#include "im_union.cuh"

namespace imgb {

enum : uint32_t {
  kPhLanes = 0,
  kPhInit = 1,
  kPhUnion = 2,
  kPhCompress = 3,
  kPhGains = 4,
  kPhCelf = 5,
  kNumPhases = 6
};

// Device descriptor of one batched query (written by the host at creation).
struct BatchInst {
  // graph, resident
  const int32_t *eu, *ev;
  const uint32_t *code_up;
  int64_t m_up;
  uint32_t n;
  // query
  uint32_t R, K, seed, T32;
  int all_live, none_live, nb, weighted, mix;
  // slices of the batch arena
  int32_t *P;
  uint32_t *cov;
  uint64_t ncov;
  uint64_t *keys, *keyrange;
  uint8_t *chosen;
  uint32_t *X, *Xs, *perm, *boff;
  int32_t *out_seeds;
  uint64_t *out_sigma;
  int32_t *status;
  unsigned long long *stats;
  // tiling: work per item of each phase, and item counts
  uint64_t init_chunk;  // label slots
  uint32_t union_chunk;  // upper edges
  uint32_t comp_chunk;   // size-memo tiles
  uint32_t gains_chunk;  // vertices
  uint32_t items[kNumPhases];
  // lazy greedy
  int B;
  uint32_t magic_R, refresh_after, round_cap, uf_cap;
};

// A bound refresh of one query's lazy greedy, opened to other blocks: its
// vertices are cut into chunks that any block may claim. Records are never
// reused within a launch, so a stale reference to one is harmless.
struct HelpJob {
  unsigned int state;  // 1 while chunks may be claimed
  unsigned int query, lb, nchunks, next, done;
  unsigned long long kmin, kmax;
};
constexpr uint32_t kHelpSlots = 8;        // refreshes open to help at once
constexpr uint32_t kHelpChunk = 512;      // vertices per refresh chunk
constexpr uint64_t kHelpMinSlots = 1u << 22;  // smaller refreshes stay with their block
constexpr uint32_t kMaxJobs = 4096;       // refresh jobs per launch (later ones stay local)

struct BatchArgs {
  const BatchInst *inst;
  const uint64_t *items;  // (query << 44) | (phase << 40) | tile
  uint32_t nitems;
  unsigned int *head;     // next item
  unsigned int *done;     // done[query * kNumPhases + phase]
  unsigned int *abort;    // set by the first wait that runs out of budget
  uint32_t spin_cap;      // polls of a dependency wait before IM_ETIMEOUT
  HelpJob *jobs;          // kMaxJobs records
  unsigned int *job_count;  // jobs published
  unsigned int *help_open;  // jobs open to help
  unsigned int *help_slot;  // kHelpSlots words: job id + 1, 0 = empty
  unsigned int *celf_done;  // lazy-greedy items finished
  uint32_t ncelf;           // lazy-greedy items of the launch
  uint32_t idle_cap;        // polls of an idle block before it gives up
  unsigned long long *phase_cyc;  // SM cycles per phase: 2 x kNumPhases (waiting, working)
  unsigned long long *help_cyc;   // SM cycles of claimed refresh chunks
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until phase ph of query q has counted `need` items done;
// a wait that exceeds the budget records IM_ETIMEOUT for the query, raises
// the launch's abort flag (every later wait then gives up at once, so the
// launch ends within about one budget) and gives up (the item still runs and
// counts, on whatever the tables hold, so no other wait can hang on it). The
// barrier hands the acquired state to the block.
__device__ void wait_done(const BatchArgs &a, uint32_t q, uint32_t ph, uint32_t need,
                          int32_t *status, int *s_flag) {
  if (threadIdx.x == 0) {
    uint32_t it = 0;
    while (ld_acquire(a.done + (size_t)q * kNumPhases + ph) < need) {
      if (++it > a.spin_cap || ld_acquire(a.abort)) {
        set_status(status, IM_ETIMEOUT);
        atomicExch(a.abort, 1u);
        break;
      }
      __nanosleep(256);
    }
    *s_flag = 1;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ tiles

__device__ void batch_init(const BatchInst &I, uint64_t t) {
  const uint64_t nR = (uint64_t)I.n * I.R;
  const uint64_t s0 = t * I.init_chunk;
  const uint64_t s1 = s0 + I.init_chunk < nR ? s0 + I.init_chunk : nR;
  // label slots: chunks are multiples of 128 slots, so [s0, s1) starts 16-byte aligned
  const int4 m1 = make_int4(-1, -1, -1, -1);
  int4 *p4 = reinterpret_cast<int4 *>(I.P + s0);
  const uint64_t n4 = (s1 - s0) >> 2;
  for (uint64_t i = threadIdx.x; i < n4; i += blockDim.x) p4[i] = m1;
  for (uint64_t i = s0 + (n4 << 2) + threadIdx.x; i < s1; i += blockDim.x) I.P[i] = -1;
  // covered bits of the same slots
  const uint64_t w0 = s0 >> 5, w1 = (s1 + 31) >> 5 < I.ncov ? (s1 + 31) >> 5 : I.ncov;
  for (uint64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) I.cov[w] = 0u;
}

template <bool OPTS>
__device__ void batch_union(const BatchInst &I, uint64_t t, uint32_t *s_boff) {
  UnionArgs u;
  u.eu = I.eu;
  u.ev = I.ev;
  u.m_up = I.m_up;
  u.Xs = I.Xs;
  u.boff = I.boff;
  u.nb = I.nb;
  u.T32 = I.T32;
  u.all_live = I.all_live;
  u.R = I.R;
  u.cap = I.uf_cap;
  u.P = I.P;
  u.status = I.status;
  u.weighted = I.weighted;
  u.mix = I.mix;
  u.code_up = I.code_up;
  u.mask = nullptr;
  u.xadj = nullptr;
  u.adj = nullptr;
  u.gate = nullptr;
  const int nbk = 1 << I.nb;
  for (int i = threadIdx.x; i <= nbk; i += blockDim.x) s_boff[i] = __ldcg(I.boff + i);
  __syncthreads();
  const int64_t e0 = (int64_t)t * I.union_chunk;
  const int64_t e1 = e0 + I.union_chunk < I.m_up ? e0 + I.union_chunk : I.m_up;
  const int64_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int64_t base = e0 + warp * 32; base < e1; base += nwarps * 32)
    union_group<false, OPTS, true>(u, s_boff, base, e1);
}

// Four groups of 256 threads, each its own size-memo tile (named barriers
// 1..4), the next tile's rows loaded while the current one is walked (as in
// the standalone size-memo kernel); the item covers tiles [t*c, (t+1)*c).
// Root counts go straight to the root slots: a group's tiles change lanes
// from one tile to the next, and an order that kept the lanes (so that the
// accumulators of the standalone kernel could be used) measured slower here.
template <int BAR>
__device__ __forceinline__ void compress_tiles(const BatchInst &I, uint32_t k, uint32_t t1,
                                               int32_t (*tile)[kCompL + 1], uint32_t gtid) {
  const uint32_t tl = (I.R + kCompL - 1) / kCompL;  // tile k: vertices 32 (k / tl) .., lanes 32 (k % tl) ..
  uint32_t tv = k / tl, tj = k % tl;
  int32_t e[4];
  compress_load(I.P, I.n, I.R, tv * kCompV, tj * kCompL, gtid, e);
  for (; k < t1; k += 4) {  // a group's barrier counts its 256 threads
    compress_stage(e, gtid, tile);
    group_sync<BAR>();
    uint32_t nv = tv, nj = tj + 4;
    while (nj >= tl) {  // at most four steps
      nj -= tl;
      ++nv;
    }
    if (k + 4 < t1) compress_load(I.P, I.n, I.R, nv * kCompV, nj * kCompL, gtid, e);
    compress_walk<BAR>(I.P, I.R, I.status, I.uf_cap, tv * kCompV, tj * kCompL, tile, gtid);
    tv = nv;
    tj = nj;
  }
}

__device__ void batch_compress(const BatchInst &I, uint64_t t, int32_t (*tiles)[kCompV][kCompL + 1]) {
  const uint64_t ntiles = (uint64_t)((I.n + kCompV - 1) / kCompV) * ((I.R + kCompL - 1) / kCompL);
  const uint64_t t0 = t * I.comp_chunk;
  const uint64_t t1 = t0 + I.comp_chunk < ntiles ? t0 + I.comp_chunk : ntiles;
  const uint32_t grp = threadIdx.x >> 8, gtid = threadIdx.x & 255u;
  if (t0 + grp >= t1) return;
  const uint32_t k0 = (uint32_t)(t0 + grp), k1 = (uint32_t)t1;  // n R < 2^32: tiles fit 32 bits
  switch (grp) {
    case 0: compress_tiles<1>(I, k0, k1, tiles[0], gtid); break;
    case 1: compress_tiles<2>(I, k0, k1, tiles[1], gtid); break;
    case 2: compress_tiles<3>(I, k0, k1, tiles[2], gtid); break;
    default: compress_tiles<4>(I, k0, k1, tiles[3], gtid); break;
  }
}

// mg_v = sum_r |C_r(v)| for vertices [t*c, (t+1)*c), a warp per vertex, and
// the key range of the query.
__device__ void batch_gains(const BatchInst &I, uint64_t t) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint64_t v0 = t * I.gains_chunk;
  const uint64_t v1 = v0 + I.gains_chunk < I.n ? v0 + I.gains_chunk : I.n;
  const uint32_t R = I.R;
  uint64_t kmin = ~0ull, kmax = 0ull;
  for (uint64_t v = v0 + warp; v < v1; v += nwarps) {
    const int32_t *row = I.P + v * R;
    uint32_t sum = 0;
    if ((R & 3u) == 0) {  // rows start 16-byte aligned: four slots per load
      const int4 *row4 = reinterpret_cast<const int4 *>(row);
#pragma unroll 4
      for (uint32_t q4 = lane; q4 < (R >> 2); q4 += 32) {
        const int4 x = __ldcg(row4 + q4);
        const uint32_t j = q4 << 2;
        const int32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          sum += xs[k] < 0 ? (uint32_t)(-xs[k])
                           : (uint32_t)(-__ldcg(I.P + (uint64_t)(uint32_t)xs[k] * R + j + k));
      }
    } else {
      for (uint32_t j = lane; j < R; j += 32) {
        const int32_t x = __ldcg(row + j);
        sum += x < 0 ? (uint32_t)(-x) : (uint32_t)(-__ldcg(I.P + (uint64_t)(uint32_t)x * R + j));
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
    const uint64_t key = ((uint64_t)sum << 32) | (uint64_t)(0xffffffffu - (uint32_t)v);
    if (lane == 0) I.keys[v] = key;
    kmin = key < kmin ? key : kmin;
    kmax = key > kmax ? key : kmax;
  }
  if (lane == 0 && kmax != 0ull) {
    atomicMin(reinterpret_cast<unsigned long long *>(I.keyrange), (unsigned long long)kmin);
    atomicMax(reinterpret_cast<unsigned long long *>(I.keyrange + 1), (unsigned long long)kmax);
  }
}

// ------------------------------------------------------------------ lazy greedy

// Vertices [v0, v1) of a bound refresh (grid_refresh's rule: a vertex whose
// bound reaches lb gets its exact gain, a chosen vertex key 0), by the calling
// block; every lane returns its warp's min / max of the valid keys.
__device__ void refresh_range(const CelfArgs &a, uint32_t lb, uint32_t v_begin, uint32_t v_end,
                              uint64_t &mn, uint64_t &mx) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  mn = ~0ull;
  mx = 0ull;
  for (uint32_t base = v_begin + warp * 32; base < v_end; base += nwarps * 32) {
    const uint32_t v0 = base + lane;
    uint64_t key = 0;
    bool eval = false;
    if (v0 < v_end && !__ldcg(a.chosen + v0)) {
      key = __ldcg(a.keys + v0);
      eval = (uint32_t)(key >> 32) >= lb;
    }
    unsigned todo = __ballot_sync(kFull, eval);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t v = base + (uint32_t)src;
      const uint32_t g = exact_gain<true>(a, v);
      if (lane == src) key = make_key(g, (int32_t)v);
    }
    if (v0 < v_end) {
      if (eval || key == 0) a.keys[v0] = key;
      if (key) {
        mn = umin64(mn, key);
        mx = umax64(mx, key);
      }
    }
  }
  mn = warp_min_u64(mn);
  mx = warp_max_u64(mx);
}

// The bound refresh of one block, with the key range.
__device__ void block_refresh(const CelfArgs &a, uint32_t lb, CelfSmem &s, uint64_t &kmin,
                              uint64_t &kmax) {
  uint64_t mn, mx;
  refresh_range(a, lb, 0, a.n, mn, mx);
  kmin = block_reduce_u64(mn, false, s);
  kmax = block_reduce_u64(mx, true, s);
}

// One claimed chunk of a help job: its vertices, the key range folded into
// the job, and the chunk counted done.
__device__ void help_chunk(const CelfArgs &a, HelpJob *job, uint32_t c) {
  const uint32_t v0 = c * kHelpChunk;
  const uint32_t v1 = v0 + kHelpChunk < a.n ? v0 + kHelpChunk : a.n;
  uint64_t mn, mx;
  refresh_range(a, __ldcg(&job->lb), v0, v1, mn, mx);
  if ((threadIdx.x & 31) == 0) {
    if (mx) {
      atomicMin(&job->kmin, (unsigned long long)mn);
      atomicMax(&job->kmax, (unsigned long long)mx);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&job->done, 1u);
  }
}

// A bound refresh that other blocks may join: large refreshes are published
// as a help job (chunks of kHelpChunk vertices), this block claims chunks like
// any helper, then waits (with a budget) until every chunk is done. Small
// refreshes, and any beyond kMaxJobs, stay with this block.
__device__ void shared_refresh(const BatchArgs &ba, uint32_t q, const CelfArgs &a, uint32_t lb,
                               CelfSmem &s, uint64_t &kmin, uint64_t &kmax) {
  __shared__ unsigned int s_jid, s_c;
  __shared__ unsigned long long s_kmin, s_kmax;
  if ((uint64_t)a.n * a.R < kHelpMinSlots || a.n < 4 * kHelpChunk) {
    block_refresh(a, lb, s, kmin, kmax);
    return;
  }
  __syncthreads();  // this block's commits (chosen flags, covered bits) precede the job
  if (threadIdx.x == 0) {
    const unsigned int jid = atomicAdd(ba.job_count, 1u);
    if (jid < kMaxJobs) {
      HelpJob *job = ba.jobs + jid;
      job->query = q;
      job->lb = lb;
      job->nchunks = (a.n + kHelpChunk - 1) / kHelpChunk;
      job->next = 0;
      job->done = 0;
      job->kmin = ~0ull;
      job->kmax = 0ull;
      __threadfence();
      atomicExch(&job->state, 1u);
      atomicExch(ba.help_slot + jid % kHelpSlots, jid + 1);
      atomicAdd(ba.help_open, 1u);
    }
    s_jid = jid;
  }
  __syncthreads();
  const unsigned int jid = s_jid;
  if (jid >= kMaxJobs) {
    block_refresh(a, lb, s, kmin, kmax);
    return;
  }
  HelpJob *job = ba.jobs + jid;
  const uint32_t nch = (a.n + kHelpChunk - 1) / kHelpChunk;
  for (;;) {
    if (threadIdx.x == 0) s_c = atomicAdd(&job->next, 1u);
    __syncthreads();
    const unsigned int c = s_c;
    __syncthreads();
    if (c >= nch) break;
    help_chunk(a, job, c);
  }
  if (threadIdx.x == 0) {
    uint32_t it = 0;
    while (ld_acquire(&job->done) < nch) {
      if (++it > ba.spin_cap) {
        set_status(a.status, IM_ETIMEOUT);
        atomicExch(ba.abort, 1u);
        break;
      }
      __nanosleep(256);
    }
    atomicExch(&job->state, 0u);
    atomicCAS(ba.help_slot + jid % kHelpSlots, jid + 1, 0u);
    atomicSub(ba.help_open, 1u);
    s_kmin = __ldcg(&job->kmin);
    s_kmax = __ldcg(&job->kmax);
  }
  __syncthreads();
  kmin = s_kmin;
  kmax = s_kmax;
  __syncthreads();
}

__device__ CelfArgs celf_args(const BatchInst &I);

__device__ CelfArgs celf_args(const BatchInst &I) {
  CelfArgs a;
  a.P = I.P;
  a.cov = I.cov;
  a.keys = I.keys;
  a.keyrange = I.keyrange;
  a.chosen = I.chosen;
  a.ctl = nullptr;
  a.n = I.n;
  a.R = I.R;
  a.K = (int)I.K;
  a.B = I.B;
  a.pool_smem = 1;
  a.refresh_after = I.refresh_after;
  a.magic_R = I.magic_R;
  a.round_cap = I.round_cap;
  a.g_pool = nullptr;
  a.out_seeds = I.out_seeds;
  a.out_sigma = I.out_sigma;
  a.status = I.status;
  a.stats = I.stats;
  return a;
}

// The whole lazy greedy of one query in one block: the steps of k_celf with
// the block-local prefix extraction, bound refreshes shared with idle blocks,
// and the pool evaluated by this block alone (a cluster of one).
__device__ void batch_celf(const BatchArgs &ba, uint32_t q, const BatchInst &I, CelfSmem &s,
                           uint32_t *dyn) {
  const int tid = threadIdx.x;
  const CelfArgs a = celf_args(I);
  uint32_t *proot = dyn;
  uint32_t *pcont = proot + (size_t)a.B * a.R;
  for (uint32_t i = tid; i < a.n; i += blockDim.x) a.chosen[i] = 0;
  __syncthreads();
  const long long t_item = clock64();
  Driver d;
  bool bounded = false;
  uint64_t hi = 0;
  uint64_t A0 = __ldcg(I.keyrange), B0 = __ldcg(I.keyrange + 1);
  unsigned long long cyc_refresh = 0;
  uint32_t extracts = 0, refreshes = 0;
  int cmd = kCmdExtract;
  uint32_t outer = 0;
  for (; outer < a.round_cap; ++outer) {
    const long long t0 = clock64();
    if (cmd == kCmdRefresh) {
      const long long tr = clock64();
      shared_refresh(ba, q, a, d.lb, s, A0, B0);
      cyc_refresh += (unsigned long long)(clock64() - tr);
      bounded = false;
      hi = 0;
      ++refreshes;
    }
    uint64_t A = A0, B = B0;
    if (bounded) {
      uint64_t mn = ~0ull, mx = 0ull;
      for (uint32_t i = tid; i < a.n; i += blockDim.x) {
        const uint64_t k = __ldcg(a.keys + i);
        if (k == 0 || k >= hi) continue;
        mn = umin64(mn, k);
        mx = umax64(mx, k);
      }
      A = block_reduce_u64(mn, false, s);
      B = block_reduce_u64(mx, true, s);
    }
    if (B == 0 || A > B) {  // no vertex left anywhere: cannot happen with K <= n
      if (tid == 0) set_status(a.status, IM_EINTERNAL);
      break;
    }
    const uint64_t t = block_select(a, bounded, hi, A, B, kTarget, kCap, s);
    uint64_t so = 0;
    d.nC = block_compact(a, bounded, hi, t, s, so);
    d.sig_out = so;
    hi = t;
    bounded = true;
    ++extracts;
    if (d.nC > (uint32_t)kCap || d.nC == 0) {
      if (tid == 0) set_status(a.status, IM_EINTERNAL);
      break;
    }
    d.head = 0;
    sort_desc(s, d.nC);
    d.cyc[0] += (unsigned long long)(clock64() - t0);
    cmd = drive_rounds<true, true>(a, s, proot, pcont, d);
    if (cmd == kCmdExtract) {  // write the bounds of C back before the next search
      for (uint32_t i = d.head + tid; i < d.nC; i += blockDim.x) {
        const uint64_t k = s.C[i];
        a.keys[key_vertex(k)] = k;
      }
    }
    __syncthreads();
    if (cmd == kCmdDone || cmd == kCmdFail) break;
  }
  if (outer >= a.round_cap && tid == 0) set_status(a.status, IM_ETIMEOUT);
  if (tid == 0 && a.stats) {
    atomicAdd(a.stats + 0, (unsigned long long)d.rounds);
    atomicAdd(a.stats + 1, (unsigned long long)d.evals);
    atomicAdd(a.stats + 2, (unsigned long long)extracts);
    atomicAdd(a.stats + 8, (unsigned long long)refreshes);
    // SM cycles: 4 = prefix extraction (with refreshes), 5 = the whole item,
    // 12 = refreshes alone
    atomicAdd(a.stats + 4, d.cyc[0]);
    atomicAdd(a.stats + 5, (unsigned long long)(clock64() - t_item));
    atomicAdd(a.stats + 12, cyc_refresh);
  }
}

// ------------------------------------------------------------------ the launch

// What a block does next (decided by its thread 0).
enum : uint32_t { kTakeItem = 0, kTakeHelp = 1, kTakeIdle = 2, kTakeExit = 3 };

__global__ void __launch_bounds__(kCelfThreads, 1) k_batch(BatchArgs a) {
  __shared__ CelfSmem s;
  __shared__ uint32_t s_item_lo, s_item_hi, s_kind, s_job, s_chunk;
  __shared__ int s_flag;
  extern __shared__ uint32_t dyn[];
  const int tid = threadIdx.x;
  bool queue_empty = false;  // thread 0's view
  uint32_t idle_polls = 0;   // thread 0's count
  for (;;) {
    if (tid == 0) {
      uint32_t kind = kTakeIdle;
      // an open refresh chunk first: it is on some query's critical path
      if (ld_acquire(a.help_open) > 0) {
        for (uint32_t h = 0; h < kHelpSlots && kind == kTakeIdle; ++h) {
          const unsigned int js = ld_acquire(a.help_slot + h);
          if (!js) continue;
          HelpJob *job = a.jobs + (js - 1);
          if (ld_acquire(&job->state) != 1u || *(volatile unsigned int *)&job->next >= job->nchunks)
            continue;
          const unsigned int c = atomicAdd(&job->next, 1u);
          if (c < job->nchunks) {
            kind = kTakeHelp;
            s_job = js - 1;
            s_chunk = c;
          }
        }
      }
      if (kind == kTakeIdle && !queue_empty) {
        const unsigned int k = atomicAdd(a.head, 1u);
        if (k < a.nitems) {
          const uint64_t it = a.items[k];
          s_item_lo = (uint32_t)it;
          s_item_hi = (uint32_t)(it >> 32);
          kind = kTakeItem;
        } else {
          queue_empty = true;
        }
      }
      if (kind == kTakeIdle) {
        // every item is taken: stay to help refreshes until every lazy greedy
        // is done (bounded; the abort flag ends it early)
        if (ld_acquire(a.celf_done) >= a.ncelf || ld_acquire(a.abort)) {
          kind = kTakeExit;
        } else if (++idle_polls > a.idle_cap) {
          atomicExch(a.abort, 1u);
          kind = kTakeExit;
        } else {
          __nanosleep(512);
        }
      }
      s_kind = kind;
    }
    __syncthreads();
    const uint32_t kind = s_kind;
    const uint64_t it = ((uint64_t)s_item_hi << 32) | s_item_lo;
    const uint32_t hjob = s_job, hchunk = s_chunk;
    __syncthreads();  // the shared words are rewritten by the next take
    if (kind == kTakeExit) return;
    if (kind == kTakeIdle) continue;
    if (kind == kTakeHelp) {
      const long long th = clock64();
      HelpJob *job = a.jobs + hjob;
      help_chunk(celf_args(a.inst[__ldcg(&job->query)]), job, hchunk);
      if (tid == 0) atomicAdd(a.help_cyc, (unsigned long long)(clock64() - th));
      continue;
    }
    const long long t_wait = clock64();
    const uint32_t q = (uint32_t)(it >> 44);
    const uint32_t ph = (uint32_t)(it >> 40) & 0xfu;
    const uint64_t t = it & ((1ull << 40) - 1);
    const BatchInst &I = a.inst[q];
    // dependencies: union needs the lanes and the whole label init; every
    // later phase needs the whole previous phase
    if (ph == kPhUnion) {
      wait_done(a, q, kPhLanes, I.items[kPhLanes], I.status, &s_flag);
      wait_done(a, q, kPhInit, I.items[kPhInit], I.status, &s_flag);
    } else if (ph > kPhUnion) {
      const uint32_t prev = ph == kPhCompress ? kPhUnion : ph - 1;
      wait_done(a, q, prev, I.items[prev], I.status, &s_flag);
      if (ph == kPhGains && I.items[kPhCompress] == 0) {  // nothing was live: wait for the init
        wait_done(a, q, kPhLanes, I.items[kPhLanes], I.status, &s_flag);
        wait_done(a, q, kPhInit, I.items[kPhInit], I.status, &s_flag);
      }
    }
    const long long t_work = clock64();
    switch (ph) {
      case kPhLanes:
        draw_lanes(I.seed, I.R, I.nb, I.X, I.Xs, I.perm, I.boff, dyn, nullptr, I.keyrange);
        break;
      case kPhInit:
        batch_init(I, t);
        break;
      case kPhUnion:
        if (I.weighted || I.mix)
          batch_union<true>(I, t, dyn);
        else
          batch_union<false>(I, t, dyn);
        break;
      case kPhCompress:
        batch_compress(I, t, reinterpret_cast<int32_t(*)[kCompV][kCompL + 1]>(dyn));
        break;
      case kPhGains:
        batch_gains(I, t);
        break;
      default:
        batch_celf(a, q, I, s, dyn);
        break;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(a.done + (size_t)q * kNumPhases + ph, 1u);
      if (ph == kPhCelf) atomicAdd(a.celf_done, 1u);
      const long long t_end = clock64();
      atomicAdd(a.phase_cyc + ph, (unsigned long long)(t_work - t_wait));
      atomicAdd(a.phase_cyc + kNumPhases + ph, (unsigned long long)(t_end - t_work));
    }
  }
}

}  // namespace imgb

// ------------------------------------------------------------------ host side

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

namespace {

using namespace imgb;

constexpr uint32_t kBatchMaxR = 16384;          // lane sort and pool stay in shared memory
constexpr size_t kBatchDynSmem = 160 * 1024;     // pool, sort keys, compress tiles, bucket offsets
constexpr int kTilings = 5;                      // granularity multipliers 1, 2, 4, 8, 16
constexpr int kSchedules = 8;                    // group sizes 1, 2, 4, 8, 16, 32, 64, all
constexpr uint32_t kSpinCap = 1u << 22;          // polls of one dependency wait (about a second)
constexpr uint32_t kIdleCap = 1u << 25;          // polls of an idle block (tens of seconds)
// control words: head, abort, job count, open jobs, lazy greedies done, 3
// spare, kHelpSlots help slots; the done counters follow
constexpr size_t kCtlWords = 8 + kHelpSlots;

// Work per item at granularity multiplier g = 2^level.
struct Tiling {
  uint64_t init_chunk;
  uint32_t union_chunk, comp_chunk, gains_chunk;
};
Tiling tiling_of(int level) {
  const uint32_t g = 1u << level;
  return Tiling{(uint64_t)131072 * g, 4096u * g, 16u * g, 256u * g};
}

// Autotuner cache: the best tiling level per size class, process-wide. A
// class is (floor(log2(n * R)), R, sampling flags): items of one class do
// the same work per slot, so their best granularity agrees.
using TuneKey = std::tuple<int, uint32_t, uint32_t>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

TuneKey tune_key(uint32_t n, uint32_t R, uint32_t flags) {
  const uint64_t nR = (uint64_t)n * R;
  int lg = 0;
  while ((1ull << (lg + 1)) <= nR) ++lg;
  return TuneKey(lg, R, flags);
}

int tuned_level(const TuneKey &k) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  return it == g_tune.end() ? -1 : it->second;
}

// A level for classes the autotuner has not seen: about 32 items per phase
// for the class's size, so that large queries spread over the GPU and small
// ones do not pay per-item overhead many times.
int default_level(uint32_t n, uint32_t R) {
  const uint64_t nR = (uint64_t)n * R;
  for (int l = 0; l < kTilings; ++l)
    if (nR / tiling_of(l).init_chunk <= 32) return l;
  return kTilings - 1;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct im_batch {
  int device = 0;
  int num_sms = 0;
  int32_t count = 0;
  std::vector<const im_graph *> graph;   // per query
  std::vector<im_batch_query> query;
  std::vector<QueryParams> params;
  std::vector<int> level;                // tiling level per query
  int group = 0;                         // schedule: queries per group (0 = all of them)
  std::vector<int64_t> seed_off;         // prefix sums of K
  int64_t total_K = 0;
  void *arena = nullptr;                 // every per-query table, one allocation
  size_t arena_bytes = 0;
  BatchInst *d_inst = nullptr;
  uint64_t *d_items = nullptr;
  unsigned int *d_ctl = nullptr;         // kCtlWords control words, then done[count * kNumPhases]
  HelpJob *d_jobs = nullptr;             // kMaxJobs refresh job records
  unsigned long long *d_cyc = nullptr;   // 2 x kNumPhases phase cycles, then help cycles
  std::vector<BatchInst> h_inst;
  uint32_t nitems = 0;
  size_t items_cap = 0;
  int32_t *d_seeds = nullptr;            // total_K
  uint64_t *d_sigma = nullptr;           // total_K
  int32_t *d_status = nullptr;           // count
  unsigned long long *d_stats = nullptr; // count * IM_NUM_STATS
};

namespace {

// Item lists of the batch for its queries' current tiling levels. The
// schedule cuts the queries, largest first, into groups of G and lists each
// group phase by phase before the next group. G = all queries is phase by
// phase: a query's items never wait long for the previous phase, but every
// lazy greedy comes last. G = 1 is query by query: the largest lazy greedies
// start early, but a query's compress items wait behind its own unions.
// Every order puts each item after the items it depends on.
int batch_plan(im_batch *b) {
  std::vector<int32_t> order(b->count);
  for (int32_t i = 0; i < b->count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    const uint64_t cx = (uint64_t)b->graph[x]->n * b->params[x].R;
    const uint64_t cy = (uint64_t)b->graph[y]->n * b->params[y].R;
    return cx != cy ? cx > cy : x < y;
  });
  std::vector<uint64_t> items;
  for (int32_t i = 0; i < b->count; ++i) {
    BatchInst &I = b->h_inst[i];
    const Tiling t = tiling_of(b->level[i]);
    const uint64_t nR = (uint64_t)I.n * I.R;
    const uint64_t ntiles = (uint64_t)((I.n + kCompV - 1) / kCompV) * ((I.R + kCompL - 1) / kCompL);
    const bool live = !I.none_live && I.m_up > 0;
    I.init_chunk = t.init_chunk;
    I.union_chunk = t.union_chunk;
    I.comp_chunk = t.comp_chunk;
    I.gains_chunk = t.gains_chunk;
    I.items[kPhLanes] = 1;
    I.items[kPhInit] = (uint32_t)((nR + t.init_chunk - 1) / t.init_chunk);
    I.items[kPhUnion] = live ? (uint32_t)((I.m_up + t.union_chunk - 1) / t.union_chunk) : 0u;
    I.items[kPhCompress] = live ? (uint32_t)((ntiles + t.comp_chunk - 1) / t.comp_chunk) : 0u;
    I.items[kPhGains] = (uint32_t)((I.n + t.gains_chunk - 1) / t.gains_chunk);
    I.items[kPhCelf] = I.K > 0 ? 1u : 0u;
  }
  int G = b->group;
  const int64_t sched_ovr = override_value(IM_OVR_BATCH_GROUP);
  if (sched_ovr > 0) G = (int)sched_ovr;
  if (G <= 0 || G > b->count) G = b->count;
  for (int32_t g0 = 0; g0 < b->count; g0 += G) {
    const int32_t g1 = g0 + G < b->count ? g0 + G : b->count;
    for (uint32_t ph = 0; ph < kNumPhases; ++ph)
      for (int32_t r = g0; r < g1; ++r) {
        const int32_t i = order[r];
        for (uint32_t k = 0; k < b->h_inst[i].items[ph]; ++k)
          items.push_back(((uint64_t)i << 44) | ((uint64_t)ph << 40) | k);
      }
  }
  if (items.size() >= (1ull << 32)) return api_error(IM_EINVAL, "batch has too many work items");
  cudaError_t e = cudaSuccess;
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    e = dev_malloc(reinterpret_cast<void **>(&b->d_items), sizeof(uint64_t) * items.size());
    if (e != cudaSuccess) return api_cuda_error(e, "batch item list");
    b->items_cap = items.size();
  }
  b->nitems = (uint32_t)items.size();
  e = cudaMemcpy(b->d_items, items.data(), sizeof(uint64_t) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return api_cuda_error(e, "batch plan upload");
  return IM_OK;
}

void batch_free(im_batch *b) {
  void *ptrs[] = {b->arena, b->d_inst, b->d_items, b->d_ctl, b->d_jobs, b->d_cyc, b->d_seeds,
                  b->d_sigma, b->d_status,
                  b->d_stats};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

// Tiling levels: forced (>= 0) for every query, else the autotuner's cached
// choice for the query's class, else the default.
int batch_build(const im_graph *const *graphs, int32_t num_graphs, const im_batch_query *qs,
                int32_t count, int force_level, im_batch **out) {
  if (!graphs || !qs || !out || num_graphs < 1 || count < 1)
    return api_error(IM_EINVAL, "null arguments or empty batch");
  if (count >= (1 << 20)) return api_error(IM_EINVAL, "at most 2^20 - 1 queries in a batch");
  im_batch *b = new (std::nothrow) im_batch();
  if (!b) return api_error(IM_ENOMEM, "host allocation failed");
  b->count = count;
  b->graph.resize(count);
  b->query.assign(qs, qs + count);
  b->params.resize(count);
  b->level.resize(count);
  b->seed_off.resize(count + 1);
  b->h_inst.resize(count);
  int rc = IM_OK;
  for (int32_t i = 0; i < count && rc == IM_OK; ++i) {
    const im_batch_query &q = qs[i];
    if (q.graph < 0 || q.graph >= num_graphs || !graphs[q.graph]) {
      rc = api_error(IM_EINVAL, "query %d: graph index %d outside [0, %d)", i, q.graph, num_graphs);
      break;
    }
    const im_graph *g = graphs[q.graph];
    b->graph[i] = g;
    if (i == 0) {
      b->device = g->device;
      b->num_sms = g->num_sms;
    } else if (g->device != b->device) {
      rc = api_error(IM_EINVAL, "query %d: all graphs of a batch must be on one device", i);
      break;
    }
    if (q.R < 1 || (uint32_t)q.R > kBatchMaxR) {
      rc = api_error(IM_EINVAL, "query %d: R=%d outside [1, %u] for a batch", i, q.R, kBatchMaxR);
      break;
    }
    if (q.K < 1 || q.K > g->n) {
      rc = api_error(IM_EINVAL, "query %d: K=%d outside [1, n=%d]", i, q.K, g->n);
      break;
    }
    if (q.flags & IM_ALGO_FUSED_SAMPLING) {
      rc = api_error(IM_EINVAL, "query %d: IM_ALGO_FUSED_SAMPLING is not batched", i);
      break;
    }
    rc = api_query_params(g, q.R, q.p, q.rng_seed, q.flags, &b->params[i]);
    if (rc != IM_OK) break;
    const TuneKey key = tune_key((uint32_t)g->n, (uint32_t)q.R, q.flags);
    int lv = force_level >= 0 ? force_level : tuned_level(key);
    b->level[i] = lv >= 0 ? lv : default_level((uint32_t)g->n, (uint32_t)q.R);
    b->seed_off[i + 1] = b->seed_off[i] + q.K;
  }
  if (rc != IM_OK) {
    delete b;
    return rc;
  }
  b->total_K = b->seed_off[count];
  // arena: every query's tables at 256-byte offsets
  std::vector<size_t> off(count);
  size_t bytes = 0;
  for (int32_t i = 0; i < count; ++i) {
    const size_t n = (size_t)b->graph[i]->n, R = (size_t)qs[i].R, nR = n * R;
    off[i] = bytes;
    bytes += align256(4 * nR) + align256(4 * ((nR + 31) / 32)) + align256(8 * n) + align256(16) +
             align256(n) + 3 * align256(4 * R) + align256(4 * ((1u << kMaxBucketBits) + 1));
  }
  b->arena_bytes = bytes;
  DeviceGuard dg(b->device);
  cudaError_t e = dev_malloc(&b->arena, bytes ? bytes : 1);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&b->d_inst), sizeof(BatchInst) * count);
  if (e == cudaSuccess)
    e = dev_malloc(reinterpret_cast<void **>(&b->d_ctl),
                   sizeof(unsigned int) * (kCtlWords + (size_t)count * kNumPhases));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&b->d_jobs), sizeof(HelpJob) * kMaxJobs);
  if (e == cudaSuccess)
    e = dev_malloc(reinterpret_cast<void **>(&b->d_cyc), sizeof(unsigned long long) * (2 * kNumPhases + 1));
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&b->d_seeds), sizeof(int32_t) * b->total_K);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&b->d_sigma), sizeof(uint64_t) * b->total_K);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&b->d_status), sizeof(int32_t) * count);
  if (e == cudaSuccess)
    e = dev_malloc(reinterpret_cast<void **>(&b->d_stats),
                   sizeof(unsigned long long) * IM_NUM_STATS * (size_t)count);
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return api_cuda_error(e, "batch allocation");
  }
  for (int32_t i = 0; i < count; ++i) {
    const im_graph *g = b->graph[i];
    const QueryParams &q = b->params[i];
    BatchInst &I = b->h_inst[i];
    const size_t n = (size_t)g->n, R = q.R, nR = n * R;
    unsigned char *p = static_cast<unsigned char *>(b->arena) + off[i];
    I.eu = g->d_eu;
    I.ev = g->d_ev;
    I.code_up = g->d_code_up;
    I.m_up = g->m_up;
    I.n = (uint32_t)g->n;
    I.R = q.R;
    I.K = (uint32_t)qs[i].K;
    I.seed = q.seed;
    I.T32 = q.T32;
    I.all_live = q.all_live;
    I.none_live = q.none_live;
    I.nb = q.nb;
    I.weighted = q.weighted;
    I.mix = q.mix;
    I.P = reinterpret_cast<int32_t *>(p);
    p += align256(4 * nR);
    I.cov = reinterpret_cast<uint32_t *>(p);
    I.ncov = (nR + 31) / 32;
    p += align256(4 * I.ncov);
    I.keys = reinterpret_cast<uint64_t *>(p);
    p += align256(8 * n);
    I.keyrange = reinterpret_cast<uint64_t *>(p);
    p += align256(16);
    I.chosen = p;
    p += align256(n);
    I.X = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * R);
    I.Xs = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * R);
    I.perm = reinterpret_cast<uint32_t *>(p);
    p += align256(4 * R);
    I.boff = reinterpret_cast<uint32_t *>(p);
    I.out_seeds = b->d_seeds + b->seed_off[i];
    I.out_sigma = b->d_sigma + b->seed_off[i];
    I.status = b->d_status + i;
    I.stats = b->d_stats + (size_t)IM_NUM_STATS * i;
    I.B = celf_pool_size(q.R);
    I.magic_R = q.R == 1 ? 0u : (uint32_t)(((1ull << 32) + q.R - 1) / q.R);
    I.refresh_after = 64;
    I.round_cap = (uint32_t)(qs[i].K + 2) * (I.refresh_after + 8) + 1024;
    const int64_t rc_ovr = override_value(IM_OVR_CELF_ROUND_CAP);
    if (rc_ovr > 0 && (uint64_t)rc_ovr < I.round_cap) I.round_cap = (uint32_t)rc_ovr;
    I.uf_cap = uf_budget((uint32_t)g->n);
  }
  rc = batch_plan(b);
  if (rc == IM_OK) {  // set here, not at launch, so that a stream capture sees stream work only
    e = cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBatchDynSmem);
    if (e != cudaSuccess) rc = api_cuda_error(e, "batch shared memory");
  }
  if (rc != IM_OK) {
    batch_free(b);
    delete b;
    return rc;
  }
  *out = b;
  return IM_OK;
}

// Queue one run: reset the control words and done counters, the refresh job
// records, statuses and stats, then the persistent launch (one 1024-thread
// block per SM).
int batch_enqueue(im_batch *b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_ctl, 0,
                                  sizeof(unsigned int) * (kCtlWords + (size_t)b->count * kNumPhases), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_jobs, 0, sizeof(HelpJob) * kMaxJobs, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_cyc, 0, sizeof(unsigned long long) * (2 * kNumPhases + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int32_t) * b->count, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_stats, 0, sizeof(unsigned long long) * IM_NUM_STATS * b->count, s);
  if (e != cudaSuccess) return api_cuda_error(e, "batch reset");
  BatchArgs a;
  a.inst = b->d_inst;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.head = b->d_ctl;
  a.abort = b->d_ctl + 1;
  a.job_count = b->d_ctl + 2;
  a.help_open = b->d_ctl + 3;
  a.celf_done = b->d_ctl + 4;
  a.help_slot = b->d_ctl + 8;
  a.done = b->d_ctl + kCtlWords;
  a.jobs = b->d_jobs;
  a.ncelf = (uint32_t)b->count;  // every batched query has K >= 1
  a.phase_cyc = b->d_cyc;
  a.help_cyc = b->d_cyc + 2 * kNumPhases;
  a.idle_cap = kIdleCap;
  a.spin_cap = kSpinCap;
  k_batch<<<b->num_sms, kCelfThreads, kBatchDynSmem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return api_cuda_error(e, "k_batch");
  api_count_launch();
  return IM_OK;
}

}  // namespace

extern "C" {

int im_batch_create(const im_graph *const *graphs, int32_t num_graphs,
                    const im_batch_query *queries, int32_t count, im_batch **out) {
  return batch_build(graphs, num_graphs, queries, count, -1, out);
}

int im_batch_destroy(im_batch *b) {
  if (!b) return api_error(IM_EINVAL, "null batch");
  DeviceGuard dg(b->device);
  batch_free(b);
  delete b;
  return IM_OK;
}

int im_batch_run_async(im_batch *b) {
  if (!b) return api_error(IM_EINVAL, "null batch");
  DeviceGuard dg(b->device);
  return batch_enqueue(b, api_stream());
}

int im_batch_results(im_batch *b, int32_t *out_seeds, uint64_t *out_sigma_R, int32_t *out_status) {
  if (!b || !out_seeds || !out_sigma_R) return api_error(IM_EINVAL, "null argument");
  DeviceGuard dg(b->device);
  cudaStream_t s = api_stream();
  std::vector<int32_t> st(b->count);
  cudaError_t e = cudaMemcpyAsync(out_seeds, b->d_seeds, sizeof(int32_t) * b->total_K,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_sigma_R, b->d_sigma, sizeof(uint64_t) * b->total_K,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st.data(), b->d_status, sizeof(int32_t) * b->count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return api_cuda_error(e, "batch results");
  int first = IM_OK;
  for (int32_t i = 0; i < b->count; ++i) {
    if (out_status) out_status[i] = st[i];
    if (st[i] != 0 && first == IM_OK) first = st[i];
  }
  if (first != IM_OK)
    return api_error(first, "a batched query failed on the device (see the per-query statuses)");
  return IM_OK;
}

int im_batch_query_stats(im_batch *b, int32_t query, int64_t *out) {
  if (!b || !out || query < 0 || query >= b->count) return api_error(IM_EINVAL, "bad arguments");
  DeviceGuard dg(b->device);
  unsigned long long h[IM_NUM_STATS];
  cudaStream_t s = api_stream();
  cudaError_t e = cudaMemcpyAsync(h, b->d_stats + (size_t)IM_NUM_STATS * query, sizeof(h),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return api_cuda_error(e, "batch stats");
  for (int i = 0; i < IM_NUM_STATS; ++i) out[i] = (int64_t)h[i];
  return IM_OK;
}

int im_batch_phase_cycles(im_batch *b, int64_t *out) {
  if (!b || !out) return api_error(IM_EINVAL, "null argument");
  DeviceGuard dg(b->device);
  unsigned long long h[2 * kNumPhases + 1];
  cudaStream_t s = api_stream();
  cudaError_t e = cudaMemcpyAsync(h, b->d_cyc, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return api_cuda_error(e, "batch cycles");
  for (int i = 0; i < 2 * (int)kNumPhases + 1; ++i) out[i] = (int64_t)h[i];
  return IM_OK;
}

int im_batch_info(const im_batch *b, int64_t *out) {
  if (!b || !out) return api_error(IM_EINVAL, "null argument");
  out[IM_BATCH_INFO_QUERIES] = b->count;
  out[IM_BATCH_INFO_ITEMS] = b->nitems;
  out[IM_BATCH_INFO_DEVICE_BYTES] = (int64_t)b->arena_bytes;
  out[IM_BATCH_INFO_TOTAL_K] = b->total_K;
  int64_t hist = 0;
  for (int32_t i = 0; i < b->count; ++i) hist += (int64_t)1 << (4 * b->level[i]);
  out[IM_BATCH_INFO_LEVELS] = hist;
  out[IM_BATCH_INFO_SCHEDULE] = b->group > 0 && b->group < b->count ? b->group : b->count;
  return IM_OK;
}

// Autotuner: for every size class among the batch's queries, up to four of
// its largest queries are run as a batch of their own at each tiling level
// (`trials` timed runs after one warm-up, CUDA events on the thread's stream);
// the level with the smallest median time goes into the process-wide cache
// and the batch is planned again with the cached levels. The selection itself
// does not depend on the tiling.
int im_batch_autotune(im_batch *b, int32_t trials) {
  if (!b || trials < 1) return api_error(IM_EINVAL, "null batch or trials < 1");
  DeviceGuard dg(b->device);
  cudaStream_t s = api_stream();
  std::map<TuneKey, std::vector<int32_t>> classes;
  for (int32_t i = 0; i < b->count; ++i)
    classes[tune_key((uint32_t)b->graph[i]->n, (uint32_t)b->query[i].R, b->query[i].flags)]
        .push_back(i);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return api_error(IM_ECUDA, "event creation");
  int rc = IM_OK;
  for (auto &kv : classes) {
    std::vector<int32_t> &members = kv.second;
    std::sort(members.begin(), members.end(), [&](int32_t x, int32_t y) {
      return b->graph[x]->n > b->graph[y]->n || (b->graph[x]->n == b->graph[y]->n && x < y);
    });
    if (members.size() > 4) members.resize(4);
    std::vector<const im_graph *> gs;
    std::vector<im_batch_query> qs;
    for (int32_t i : members) {
      im_batch_query q = b->query[i];
      q.graph = (int32_t)gs.size();
      gs.push_back(b->graph[i]);
      qs.push_back(q);
    }
    int best = -1;
    float best_ms = 0.f;
    for (int lv = 0; lv < kTilings && rc == IM_OK; ++lv) {
      im_batch *t = nullptr;
      rc = batch_build(gs.data(), (int32_t)gs.size(), qs.data(), (int32_t)qs.size(), lv, &t);
      if (rc != IM_OK) break;
      std::vector<float> ms;
      for (int r = 0; r <= trials && rc == IM_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = batch_enqueue(t, s);
        cudaEventRecord(e1, s);
        if (rc == IM_OK && cudaEventSynchronize(e1) != cudaSuccess)
          rc = api_error(IM_ECUDA, "autotune timing");
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) ms.push_back(x);
      }
      batch_free(t);
      delete t;
      if (rc != IM_OK) break;
      std::sort(ms.begin(), ms.end());
      const float med = ms[ms.size() / 2];
      if (best < 0 || med < best_ms) {
        best = lv;
        best_ms = med;
      }
    }
    if (rc != IM_OK) break;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[kv.first] = best;
  }
  if (rc == IM_OK) {
    for (int32_t i = 0; i < b->count; ++i) {
      const int lv = tuned_level(tune_key((uint32_t)b->graph[i]->n, (uint32_t)b->query[i].R,
                                          b->query[i].flags));
      if (lv >= 0) b->level[i] = lv;
    }
    // the schedule: group sizes 1, 2, 4, ..., 64 and all on the whole batch,
    // the fastest kept (on the 256-query recipe, groups of 8 ran 1.4x faster
    // than query by query and 1.9x faster than phase by phase)
    const int groups[kSchedules] = {1, 2, 4, 8, 16, 32, 64, 0};
    float sched_ms[kSchedules] = {0.f};
    for (int sc = 0; sc < kSchedules && rc == IM_OK; ++sc) {
      b->group = groups[sc];
      rc = batch_plan(b);
      std::vector<float> ms;
      for (int r = 0; r <= trials && rc == IM_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = batch_enqueue(b, s);
        cudaEventRecord(e1, s);
        if (rc == IM_OK && cudaEventSynchronize(e1) != cudaSuccess)
          rc = api_error(IM_ECUDA, "autotune timing");
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) ms.push_back(x);
      }
      if (rc == IM_OK) {
        std::sort(ms.begin(), ms.end());
        sched_ms[sc] = ms[ms.size() / 2];
      }
    }
    if (rc == IM_OK) {
      int best = 0;
      for (int sc = 1; sc < kSchedules; ++sc)
        if (sched_ms[sc] < sched_ms[best]) best = sc;
      b->group = groups[best];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != IM_OK) return rc;
  return batch_plan(b);
}

int im_autotune_cache_save(const char *path) {
  if (!path) return api_error(IM_EINVAL, "null path");
  FILE *f = std::fopen(path, "w");
  if (!f) return api_error(IM_EINVAL, "cannot write %s", path);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::fprintf(f, "# log2(n*R) R flags tiling_level\n");
  for (auto &kv : g_tune)
    std::fprintf(f, "%d %u %u %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), kv.second);
  std::fclose(f);
  return IM_OK;
}

int im_autotune_cache_load(const char *path) {
  if (!path) return api_error(IM_EINVAL, "null path");
  FILE *f = std::fopen(path, "r");
  if (!f) return api_error(IM_EINVAL, "cannot read %s", path);
  char line[256];
  std::map<TuneKey, int> loaded;
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    int lg = 0, lv = 0;
    unsigned R = 0, flags = 0;
    if (std::sscanf(line, "%d %u %u %d", &lg, &R, &flags, &lv) == 4 && lv >= 0 && lv < kTilings)
      loaded[TuneKey(lg, R, flags)] = lv;
  }
  std::fclose(f);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto &kv : loaded) g_tune[kv.first] = kv.second;
  return IM_OK;
}

int im_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  return IM_OK;
}

}  // extern "C"
