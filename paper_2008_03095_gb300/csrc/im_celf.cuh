// Device side of the on-device lazy greedy (CELF) over the memoized samples
// (Algorithm 7): constants, the shared-memory and grid-shared state, the
// prefix extraction steps, the exact pool evaluation and the driver's rounds.
// Included by im_celf.cu (the cooperative k_celf launch) and im_batch.cu (the
// block-local lazy greedy of a batched launch). COH selects coherent (L2)
// loads of the label table for kernels that wrote it earlier in the same
// launch; the read-only path is kept where the table is constant.
#pragma once
#include <cooperative_groups.h>

#include "im_common.cuh"

namespace cg = cooperative_groups;

namespace imgb {

template <bool COH>
static __device__ __forceinline__ int32_t ld_label(const int32_t *p) {
  return COH ? __ldcg(p) : __ldg(p);
}

constexpr int kCelfThreads = 1024;

// Zero the contributions of the lanes whose root equals the committed seed's
// root (the lanes the seed now covers), adding them to dsum; true when any
// of the four lanes changed.
static __device__ __forceinline__ bool drop_shared4(uint4 &cv, const uint4 r, const uint4 b,
                                             uint32_t &dsum) {
  bool dirty = false;
  if (cv.x && r.x == b.x) { dsum += cv.x; cv.x = 0; dirty = true; }
  if (cv.y && r.y == b.y) { dsum += cv.y; cv.y = 0; dirty = true; }
  if (cv.z && r.z == b.z) { dsum += cv.z; cv.z = 0; dirty = true; }
  if (cv.w && r.w == b.w) { dsum += cv.w; cv.w = 0; dirty = true; }
  return dirty;
}
constexpr int kCelfWarps = kCelfThreads / 32;
constexpr int kCap = 4096;     // candidate prefix capacity
constexpr int kTarget = 2048;  // prefix size aimed for per extraction
constexpr int kBins = 2048;    // histogram bins of the threshold search
constexpr int kPoolMax = 32;
// Blocks of the first thread-block cluster (the driver and its helpers) that
// evaluate each round's pool together when the pool lives in shared memory.
constexpr int kEvalCluster = 8;
constexpr size_t kPoolSmemBudget = 160 * 1024;

enum : int { kCmdExtract = 1, kCmdRefresh = 2, kCmdDone = 3, kCmdFail = 4, kCmdEval = 5 };

// Grid-shared control block (global memory).
struct CelfCtl {
  unsigned long long kmin, kmax, sig_out;
  unsigned int kcount, nC;
  int cmd;
  unsigned int refresh_lb;  // driver -> grid: the refresh bound (see grid_refresh)
  unsigned int hist[3][kBins];
  unsigned long long C[kCap];
  // A launch that stops for an external refresh (large graphs; see
  // launch_celf) leaves its state here for the launch that resumes.
  int ext_state;  // 1: stopped for a refresh, not yet resumed
  int s_nsel;
  unsigned long long s_sigma;
  unsigned int s_rounds, s_evals, s_lb, s_outer, s_extracts, s_refreshes, s_pass;
  unsigned long long s_cyc[4], s_fine[2];
};




struct CelfArgs {
  const int32_t *P;
  uint32_t *cov;
  uint64_t *keys;
  const uint64_t *keyrange;
  uint8_t *chosen;
  CelfCtl *ctl;
  uint32_t n, R;
  int K;
  int B;
  int pool_smem;
  uint32_t refresh_after;  // evaluations without a commit that trigger a refresh
  uint32_t magic_R;        // ceil(2^32 / R) for div_R (0 when R == 1)
  uint32_t round_cap;      // budget of driver rounds (see launch_celf)
  uint32_t *g_pool;
  int32_t *out_seeds;
  uint64_t *out_sigma;
  int32_t *status;
  unsigned long long *stats;
  int resume;    // continue a launch that stopped for an external refresh (else return)
  int ext_left;  // external refreshes this launch may stop for (0: refresh in the launch)
};

struct CelfSmem {
  uint64_t C[kCap];
  uint32_t hist[kBins];
  uint64_t red[kCelfWarps];
  int32_t pid[kPoolMax];
  uint32_t pgain[2][kPoolMax];   // exact gains of the pool, double-buffered by commit
  int32_t pactive[2][kPoolMax];  // pool member still a candidate, same buffering
  int32_t committed[kPoolMax];
  uint64_t Y[kPoolMax];
  uint32_t ny;
  int ccmd;      // driver -> helpers: kCmdEval or the command drive_rounds returns
  uint32_t cnp;  // driver -> helpers: pool size of the round
  uint64_t sel_t, sel_A, sel_B;
  uint32_t sel_above;
  int sel_done;
};

static __device__ __forceinline__ uint64_t make_key(uint32_t gain, int32_t v) {
  return ((uint64_t)gain << 32) | (uint64_t)(0xffffffffu - (uint32_t)v);
}
static __device__ __forceinline__ int32_t key_vertex(uint64_t k) {
  return (int32_t)(0xffffffffu - (uint32_t)k);
}
static __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
static __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

static __device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = umax64(v, __shfl_xor_sync(kFull, v, d));
  return v;
}
static __device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = umin64(v, __shfl_xor_sync(kFull, v, d));
  return v;
}

// ------------------------------------------------------------------ grid steps

// Grid-wide min / max / count of the valid keys (nonzero, < hi) into ctl.
static __device__ void grid_key_stats(const CelfArgs &a, uint64_t hi) {
  const int lane = threadIdx.x & 31;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t gthreads = gridDim.x * blockDim.x;
  uint64_t mn = ~0ull, mx = 0ull;
  uint32_t c = 0;
  for (uint32_t i = gtid; i < a.n; i += gthreads) {
    const uint64_t k = __ldcg(a.keys + i);
    if (k == 0 || k >= hi) continue;
    mn = umin64(mn, k);
    mx = umax64(mx, k);
    ++c;
  }
  mn = warp_min_u64(mn);
  mx = warp_max_u64(mx);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
  if (lane == 0 && c) {
    atomicMin(&a.ctl->kmin, (unsigned long long)mn);
    atomicMax(&a.ctl->kmax, (unsigned long long)mx);
    atomicAdd(&a.ctl->kcount, c);
  }
}

// Threshold search over the valid keys (nonzero and, if bounded, < hi) of
// keys[0..n): every block returns the same t such that the number of valid
// keys >= t lies in [min(target, count), cap]. Each pass histograms the
// current range [A, B] into kBins equal bins (shared-memory counts per block,
// summed into a global histogram), finds the bin where the running count from
// the top reaches the target, and stops there if everything down to that bin
// fits in cap, else narrows to that bin. Global histograms rotate over three
// buffers so that one grid barrier per pass suffices.
static __device__ __noinline__ uint64_t grid_select(const CelfArgs &a, cg::grid_group &grid, bool bounded,
                                uint64_t hi, uint64_t A, uint64_t B, uint32_t target,
                                uint32_t cap, CelfSmem &s, uint32_t &pass_id) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t gthreads = gridDim.x * blockDim.x;
  uint32_t above = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const uint32_t buf = pass_id % 3, zbuf = (pass_id + 1) % 3;
    ++pass_id;
    const uint64_t span = B - A;
    const int bl = span ? 64 - __clzll((long long)span) : 0;
    const int shift = bl > 11 ? bl - 11 : 0;
    if (blockIdx.x == gridDim.x - 1)
      for (int i = tid; i < kBins; i += blockDim.x) a.ctl->hist[zbuf][i] = 0u;
    for (int i = tid; i < kBins; i += blockDim.x) s.hist[i] = 0u;
    __syncthreads();
    for (uint32_t base = blockIdx.x * blockDim.x + (uint32_t)warp * 32; base < a.n;
         base += gthreads) {
      const uint32_t i = base + lane;
      const uint64_t k = i < a.n ? __ldcg(a.keys + i) : 0ull;
      const bool in = k != 0 && (!bounded || k < hi) && k >= A && k <= B;
      const unsigned act = __ballot_sync(kFull, in);
      if (in) {
        const uint32_t d = (uint32_t)((k - A) >> shift);
        const unsigned peers = __match_any_sync(act, d);
        if (lane == __ffs(peers) - 1) atomicAdd(&s.hist[d], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    for (int i = tid; i < kBins; i += blockDim.x)
      if (s.hist[i]) atomicAdd(&a.ctl->hist[buf][i], s.hist[i]);
    grid.sync();
    if (warp == 0) {
      // lane l covers bins 2047-64l down to 1984-64l
      uint32_t lsum = 0;
      for (int i = 0; i < 64; ++i) lsum += __ldcg(&a.ctl->hist[buf][kBins - 1 - 64 * lane - i]);
      uint32_t incl = lsum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
      }
      const uint32_t excl = incl - lsum;
      const unsigned ball = __ballot_sync(kFull, above + incl >= target);
      if (!ball) {  // fewer valid keys than the target: take the whole range
        if (lane == 0) {
          s.sel_done = 1;
          s.sel_t = A;
        }
      } else if (lane == __ffs(ball) - 1) {
        uint32_t cum = above + excl;
        int d = kBins - 1 - 64 * lane;
        uint32_t hd = 0;
        for (int i = 0; i < 64; ++i) {
          d = kBins - 1 - 64 * lane - i;
          hd = __ldcg(&a.ctl->hist[buf][d]);
          if (cum + hd >= target) break;
          cum += hd;
        }
        const uint64_t lo = A + ((uint64_t)d << shift);
        if (cum + hd <= cap || shift == 0) {
          s.sel_done = 1;
          s.sel_t = lo;
        } else {
          s.sel_done = 0;
          s.sel_A = lo;
          const uint64_t top = lo + (((uint64_t)1 << shift) - 1);
          s.sel_B = top < B ? top : B;
          s.sel_above = cum;
        }
      }
    }
    __syncthreads();
    if (s.sel_done) {
      const uint64_t t = s.sel_t;
      __syncthreads();
      return t;
    }
    A = s.sel_A;
    B = s.sel_B;
    above = s.sel_above;
    __syncthreads();
  }
  if (tid == 0) set_status(a.status, IM_EINTERNAL);
  return A;
}

// Grid-wide compaction of the valid keys >= t into ctl->C, and the largest
// valid key below t into ctl->sig_out.
static __device__ void grid_compact(const CelfArgs &a, bool bounded, uint64_t hi, uint64_t t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t gthreads = gridDim.x * blockDim.x;
  uint64_t below = 0;
  for (uint32_t base = blockIdx.x * blockDim.x + (uint32_t)warp * 32; base < a.n;
       base += gthreads) {
    const uint32_t i = base + lane;
    const uint64_t k = i < a.n ? __ldcg(a.keys + i) : 0ull;
    const bool valid = k != 0 && (!bounded || k < hi);
    const bool take = valid && k >= t;
    if (valid && !take) below = umax64(below, k);
    const unsigned ball = __ballot_sync(kFull, take);
    if (ball) {
      uint32_t base_pos = 0;
      if (lane == __ffs(ball) - 1) base_pos = atomicAdd(&a.ctl->nC, (uint32_t)__popc(ball));
      base_pos = __shfl_sync(kFull, base_pos, __ffs(ball) - 1);
      const uint32_t pos = base_pos + __popc(ball & ((1u << lane) - 1u));
      if (take && pos < (uint32_t)kCap) a.ctl->C[pos] = k;
    }
  }
  below = warp_max_u64(below);
  if (lane == 0 && below) atomicMax(&a.ctl->sig_out, (unsigned long long)below);
}

// Exact marginal gain of v against the covered bitmap, summed over the warp:
// g(v | S) = sum_r [component of v in r not covered] * |C_r(v)|. Lane l takes
// slots l, l + 32, ... (consecutive lanes read consecutive slots, so a warp's
// gathers of one giant component's root fall into one cache line), four
// unrolled steps in flight. Batching eight slots per lane explicitly, in
// 16-byte groups or lane-consecutive, measured 1.3-1.6x slower on the bound
// refresh of every workload.
template <bool COH>
__device__ __forceinline__ uint32_t exact_gain(const CelfArgs &a, uint32_t v) {
  const int lane = threadIdx.x & 31;
  const uint32_t R = a.R;
  const int32_t *row = a.P + (size_t)v * R;
  uint32_t g = 0;
#pragma unroll 8
  for (uint32_t j = lane; j < R; j += 32) {
    const int32_t x = ld_label<COH>(row + j);
    const uint32_t root = x < 0 ? v : (uint32_t)x;
    const uint32_t sz = x < 0 ? (uint32_t)(-x) : (uint32_t)(-ld_label<COH>(a.P + (size_t)x * R + j));
    const uint32_t bit = root * R + j;
    const uint32_t cw = (x != -1) ? __ldcg(a.cov + (bit >> 5)) : 0u;
    g += ((cw >> (bit & 31)) & 1u) ? 0u : sz;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) g += __shfl_xor_sync(kFull, g, d);
  return g;
}

// Refresh of the bounds (a NewGreedy step on the memoized samples, limited to
// the vertices that can still matter): every vertex whose bound reaches lb --
// the largest gain known to be exact for the current seed set -- gets its
// exact gain; a vertex below lb cannot be the next commit, and its bound stays
// a valid upper bound (gains only shrink as seeds are added), so it is kept.
// Chosen vertices get key 0. Key statistics of all valid keys go into ctl.
// A warp scans 32 keys at once and evaluates the ones that qualify in turn.
static __device__ __noinline__ void grid_refresh(const CelfArgs &a, uint32_t lb) {
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t R = a.R;
  uint64_t mn = ~0ull, mx = 0ull;
  uint32_t c = 0, evaluated = 0;
  for (uint32_t base = gwarp * 32; base < a.n; base += nwarps * 32) {
    const uint32_t v0 = base + lane;
    uint64_t key = 0;
    bool eval = false;
    if (v0 < a.n && !__ldcg(a.chosen + v0)) {
      key = __ldcg(a.keys + v0);
      eval = (uint32_t)(key >> 32) >= lb;
    }
    unsigned todo = __ballot_sync(kFull, eval);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t v = base + (uint32_t)src;
      const uint32_t g = exact_gain<false>(a, v);
      if (lane == src) key = make_key(g, (int32_t)v);
      ++evaluated;
    }
    if (v0 < a.n) {
      if (eval || key == 0) a.keys[v0] = key;  // chosen vertices get 0
      if (key) {
        mn = umin64(mn, key);
        mx = umax64(mx, key);
        ++c;
      }
    }
  }
  mn = warp_min_u64(mn);
  mx = warp_max_u64(mx);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
  if (lane == 0 && c) {
    atomicMin(&a.ctl->kmin, (unsigned long long)mn);
    atomicMax(&a.ctl->kmax, (unsigned long long)mx);
    atomicAdd(&a.ctl->kcount, c);
  }
  if (lane == 0 && evaluated && a.stats) atomicAdd(a.stats + 11, (unsigned long long)evaluated);
}

// Single-block versions of the extraction steps, used by the driver alone when
// n is small enough that grid barriers would cost more than the work.
constexpr uint32_t kLocalN = 65536;

static __device__ uint64_t block_reduce_u64(uint64_t v, bool is_max, CelfSmem &s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = is_max ? warp_max_u64(v) : warp_min_u64(v);
  if (lane == 0) s.red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kCelfWarps ? s.red[lane] : (is_max ? 0ull : ~0ull);
    v = is_max ? warp_max_u64(v) : warp_min_u64(v);
    if (lane == 0) s.red[0] = v;
  }
  __syncthreads();
  v = s.red[0];
  __syncthreads();
  return v;
}

static __device__ __noinline__ uint64_t block_select(const CelfArgs &a, bool bounded, uint64_t hi, uint64_t A,
                                 uint64_t B, uint32_t target, uint32_t cap, CelfSmem &s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t above = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const uint64_t span = B - A;
    const int bl = span ? 64 - __clzll((long long)span) : 0;
    const int shift = bl > 11 ? bl - 11 : 0;
    for (int i = tid; i < kBins; i += blockDim.x) s.hist[i] = 0u;
    __syncthreads();
    for (uint32_t base = (uint32_t)warp * 32; base < a.n; base += blockDim.x) {
      const uint32_t i = base + lane;
      const uint64_t k = i < a.n ? __ldcg(a.keys + i) : 0ull;
      const bool in = k != 0 && (!bounded || k < hi) && k >= A && k <= B;
      const unsigned act = __ballot_sync(kFull, in);
      if (in) {
        const uint32_t d = (uint32_t)((k - A) >> shift);
        const unsigned peers = __match_any_sync(act, d);
        if (lane == __ffs(peers) - 1) atomicAdd(&s.hist[d], (uint32_t)__popc(peers));
      }
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t lsum = 0;
      for (int i = 0; i < 64; ++i) lsum += s.hist[kBins - 1 - 64 * lane - i];
      uint32_t incl = lsum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
      }
      const uint32_t excl = incl - lsum;
      const unsigned ball = __ballot_sync(kFull, above + incl >= target);
      if (!ball) {
        if (lane == 0) {
          s.sel_done = 1;
          s.sel_t = A;
        }
      } else if (lane == __ffs(ball) - 1) {
        uint32_t cum = above + excl;
        int d = kBins - 1 - 64 * lane;
        uint32_t hd = 0;
        for (int i = 0; i < 64; ++i) {
          d = kBins - 1 - 64 * lane - i;
          hd = s.hist[d];
          if (cum + hd >= target) break;
          cum += hd;
        }
        const uint64_t lo = A + ((uint64_t)d << shift);
        if (cum + hd <= cap || shift == 0) {
          s.sel_done = 1;
          s.sel_t = lo;
        } else {
          s.sel_done = 0;
          s.sel_A = lo;
          const uint64_t top = lo + (((uint64_t)1 << shift) - 1);
          s.sel_B = top < B ? top : B;
          s.sel_above = cum;
        }
      }
    }
    __syncthreads();
    if (s.sel_done) {
      const uint64_t t = s.sel_t;
      __syncthreads();
      return t;
    }
    A = s.sel_A;
    B = s.sel_B;
    above = s.sel_above;
    __syncthreads();
  }
  if (tid == 0) set_status(a.status, IM_EINTERNAL);
  return A;
}

// Valid keys >= t into s.C (returns the count) and the largest key below t.
static __device__ __noinline__ uint32_t block_compact(const CelfArgs &a, bool bounded, uint64_t hi, uint64_t t,
                                  CelfSmem &s, uint64_t &sig_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s.ny = 0;  // reused as the fill counter
  __syncthreads();
  uint64_t below = 0;
  for (uint32_t base = (uint32_t)warp * 32; base < a.n; base += blockDim.x) {
    const uint32_t i = base + lane;
    const uint64_t k = i < a.n ? __ldcg(a.keys + i) : 0ull;
    const bool valid = k != 0 && (!bounded || k < hi);
    const bool take = valid && k >= t;
    if (valid && !take) below = umax64(below, k);
    const unsigned ball = __ballot_sync(kFull, take);
    if (ball) {
      uint32_t base_pos = 0;
      if (lane == __ffs(ball) - 1) base_pos = atomicAdd(&s.ny, (uint32_t)__popc(ball));
      base_pos = __shfl_sync(kFull, base_pos, __ffs(ball) - 1);
      const uint32_t pos = base_pos + __popc(ball & ((1u << lane) - 1u));
      if (take && pos < (uint32_t)kCap) s.C[pos] = k;
    }
  }
  sig_out = block_reduce_u64(below, true, s);  // barriers
  return s.ny;
}

// Descending bitonic sort of s.C[0..npow2) (entries past nC padded with 0).
static __device__ __noinline__ void sort_desc(CelfSmem &s, uint32_t nC) {
  uint32_t npow2 = 1;
  while (npow2 < nC) npow2 <<= 1;
  for (uint32_t i = nC + threadIdx.x; i < npow2; i += blockDim.x) s.C[i] = 0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= npow2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < npow2; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = s.C[i], y = s.C[ixj];
          const bool desc = (i & k) == 0;
          if ((x < y) == desc) {
            s.C[i] = y;
            s.C[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ driver state
struct Driver {
  int nsel = 0;
  uint64_t sigma = 0;  // thread 0
  uint32_t head = 0, nC = 0;
  uint64_t sig_out = 0;
  uint32_t rounds = 0, evals = 0, evals_since_commit = 0;
  uint32_t lb = 0;  // the largest gain known to be exact for the current seed set
  unsigned long long cyc[4] = {0, 0, 0, 0};
  unsigned long long fine[2] = {0, 0};  // commit loop, cover atomics
};

// Block 0: lazy-greedy rounds over the prefix in shared memory until the
// query is done or a grid step is needed. Returns the next command. POOL_SMEM:
// the per-lane pool arrays live in shared memory (else in global memory).
// Invariant check: the first violation (code, two values) goes to the work
// counters and the status becomes IM_EINTERNAL; the caller keeps every index
// in range.
static __device__ __forceinline__ void celf_violation(const CelfArgs &a, uint32_t code, uint64_t v0,
                                               uint64_t v1) {
  if (atomicCAS(a.status, 0, IM_EINTERNAL) == 0 && a.stats) {
    a.stats[13] = code;
    a.stats[14] = v0;
    a.stats[15] = v1;
  }
}

// i / R for i < 2^21 by a multiply-high with M = ceil(2^32 / R) and one
// correction step (M = 0 encodes R = 1).
static __device__ __forceinline__ uint32_t div_R(uint32_t i, uint32_t R, uint32_t M) {
  if (M == 0) return i;
  uint32_t c = __umulhi(i, M);
  if (c * R > i) --c;
  return c;
}

// Exact gains of the pool's (candidate, lane) items, rank-th of nranks equal
// shares: g(u | S) = sum_r [component of u in r not covered] * |C_r(u)|. A
// thread issues the label loads of four items together, then their dependent
// size and covered-bit gathers together; root and uncovered size of every
// item go to proot / pcont (the driver's shared memory, possibly remote).
template <bool COH>
static __device__ __forceinline__ void eval_items(const CelfArgs &a, const int32_t *pid, uint32_t np,
                                           uint32_t *proot, uint32_t *pcont, uint32_t rank,
                                           uint32_t nranks) {
  const uint32_t R = a.R;
  const uint32_t items = np * R;
  const uint32_t stride = nranks * kCelfThreads;
  for (uint32_t base = rank * kCelfThreads + threadIdx.x; base < items; base += 4 * stride) {
    int32_t xv[4];
    uint32_t uv[4], jv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = base + q * stride;
      xv[q] = -1;
      uv[q] = 0;
      jv[q] = 0;
      if (i < items) {
        const uint32_t c = div_R(i, R, a.magic_R);
        jv[q] = i - c * R;
        uv[q] = (uint32_t)pid[c];
        xv[q] = ld_label<COH>(a.P + (size_t)uv[q] * R + jv[q]);
      }
    }
    uint32_t szv[4], cwv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int32_t x = xv[q];
      uint32_t root = x < 0 ? uv[q] : (uint32_t)x;
      szv[q] = 0;
      cwv[q] = 0;
      if (base + q * stride < items) {
        if (root >= a.n) {  // a label outside [0, n) cannot come from the size pass
          celf_violation(a, 2000u, root, ((uint64_t)uv[q] << 32) | jv[q]);
          root = uv[q];
        } else {
          const uint32_t bit = root * R + jv[q];
          // a singleton {u} (x == -1) is covered only if u is a seed
          szv[q] = x < 0 ? (uint32_t)(-x) : (uint32_t)(-ld_label<COH>(a.P + (size_t)x * R + jv[q]));
          cwv[q] = (x != -1) ? (__ldcg(a.cov + (bit >> 5)) >> (bit & 31)) & 1u : 0u;
          if (szv[q] > a.n) {
            celf_violation(a, 2001u, szv[q], ((uint64_t)uv[q] << 32) | jv[q]);
            szv[q] = 0;
          }
        }
      }
      uv[q] = root;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = base + q * stride;
      if (i < items) {
        proot[i] = uv[q];
        pcont[i] = cwv[q] ? 0u : szv[q];
      }
    }
  }
}

// Helper blocks of the driver's cluster: evaluate their share of every
// round's pool into the driver's shared memory until the driver announces
// another command, which is returned. The shares are cut by the cluster's
// actual size and rank, read at run time, so that every (candidate, lane)
// item is written whatever cluster shape the launch received.
static __device__ __noinline__ int helper_rounds(const CelfArgs &a, CelfSmem &s, uint32_t *dyn) {
  cg::cluster_group cl = cg::this_cluster();
  const CelfSmem *ds = cl.map_shared_rank(&s, 0);
  uint32_t *rroot = cl.map_shared_rank(dyn, 0);
  uint32_t *rcont = rroot + (size_t)a.B * a.R;
  const uint32_t rank = cl.block_rank(), nranks = cl.num_blocks();
  for (;;) {  // bounded by the driver's round budget: every driver exit is announced
    cl.sync();  // the driver has published ccmd (and the pool)
    const int cmd = *(volatile const int *)&ds->ccmd;
    if (cmd != kCmdEval) return cmd;
    const uint32_t np = *(volatile const uint32_t *)&ds->cnp;
    eval_items<false>(a, ds->pid, np, rroot, rcont, rank, nranks);
    cl.sync();  // the driver reads the results
  }
}

template <bool POOL_SMEM, bool COH>
static __device__ __noinline__ int drive_rounds(const CelfArgs &a, CelfSmem &s, uint32_t *proot, uint32_t *pcont,
                            Driver &d) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t R = a.R;
  const uint32_t B = (uint32_t)a.B;
  cg::cluster_group cl = cg::this_cluster();
  // every exit is announced to the helper blocks of the cluster (POOL_SMEM)
  auto leave = [&](int cmd) -> int {
    if (POOL_SMEM) {
      if (tid == 0) s.ccmd = cmd;
      cl.sync();
    }
    return cmd;
  };
  long long t_mark = clock64();
  for (;;) {
    if (d.nsel >= a.K) return leave(kCmdDone);
    if (d.rounds >= a.round_cap) {
      if (tid == 0) set_status(a.status, IM_ETIMEOUT);
      return leave(kCmdFail);
    }
    if (d.head >= d.nC || s.C[d.head] < d.sig_out) return leave(kCmdExtract);
    if (d.evals_since_commit >= a.refresh_after) {
      d.evals_since_commit = 0;  // the refresh makes every key exact
      return leave(kCmdRefresh);
    }
    ++d.rounds;
    const uint32_t np = (d.nC - d.head) < B ? (d.nC - d.head) : B;
    if (tid < (int)np) {
      const uint64_t kv = s.C[d.head + tid];
      int32_t v = key_vertex(kv);
      if (kv == 0 || v < 0 || (uint32_t)v >= a.n) {  // cannot happen: record, stay in range
        celf_violation(a, 1000u + (uint32_t)tid, kv, ((uint64_t)d.head << 32) | d.nC);
        v = 0;
      }
      s.pid[tid] = v;
      s.pactive[0][tid] = 1;
    }
    const uint64_t kc = d.head + np < d.nC ? s.C[d.head + np] : 0ull;
    const uint64_t top_out = umax64(kc, d.sig_out);
    d.evals += np;
    d.evals_since_commit += np;
    __syncthreads();

    // ---------------------------------------------------------- exact gains
    // With the pool in shared memory the first cluster's blocks share the
    // evaluation: the pool is published with one cluster barrier and the
    // results are complete after the next.
    if (POOL_SMEM) {
      if (tid == 0) {
        s.cnp = np;
        s.ccmd = kCmdEval;
      }
      cl.sync();
      eval_items<COH>(a, s.pid, np, proot, pcont, 0, cl.num_blocks());
      cl.sync();
    } else {
      eval_items<COH>(a, s.pid, np, proot, pcont, 0, 1);
      __syncthreads();
    }
    for (uint32_t m = (uint32_t)warp; m < np; m += kCelfWarps) {
      const uint32_t *cc = pcont + (size_t)m * R;
      uint32_t g = 0;
      if ((R & 3u) == 0) {
        const uint4 *c4 = reinterpret_cast<const uint4 *>(cc);
        for (uint32_t q = lane; q < (R >> 2); q += 32) {
          const uint4 v = c4[q];
          g += v.x + v.y + v.z + v.w;
        }
      } else {
        for (uint32_t j = lane; j < R; j += 32) g += cc[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(kFull, g, o);
      if (lane == 0) s.pgain[0][m] = g;
    }
    __syncthreads();
    {
      const long long t_now = clock64();
      d.cyc[1] += (unsigned long long)(t_now - t_mark);
      t_mark = t_now;
    }

    // ---------------------------------------------------------- commits
    // Every warp picks the best active pool member from buffer `cur` (all
    // warps read the same values, so all make the same choice); warp m then
    // writes member m's state after the commit (its gain minus the lanes it
    // shares a component with the committed seed) into buffer cur ^ 1, and one
    // barrier per commit publishes it. Nothing writes buffer cur while any
    // warp may still read it.
    uint32_t cur = 0, ncm = 0;
    for (;;) {
      uint64_t k = 0;
      if ((uint32_t)lane < np && s.pactive[cur][lane]) k = make_key(s.pgain[cur][lane], s.pid[lane]);
      const uint64_t bk = warp_max_u64(k);
      const unsigned bb = __ballot_sync(kFull, k != 0 && k == bk);
      if (bk == 0 || bk < top_out) break;
      const int bw = __ffs(bb) - 1;
      const uint32_t gsel = s.pgain[cur][bw];
      if (tid == 0) {
        const int32_t vsel = s.pid[bw];
        a.out_seeds[d.nsel] = vsel;
        a.out_sigma[d.nsel] = d.sigma + gsel;
        a.chosen[vsel] = 1;
        s.committed[ncm] = bw;
      }
      d.sigma += gsel;
      ++d.nsel;
      ++ncm;
      d.evals_since_commit = 0;
      for (uint32_t m = (uint32_t)warp; m < np; m += kCelfWarps) {
        uint32_t g = s.pgain[cur][m];
        const int32_t act = (s.pactive[cur][m] && (int)m != bw) ? 1 : 0;
        if (act && d.nsel < a.K) {
          const uint32_t *rb = proot + (size_t)bw * R;
          const uint32_t *rr = proot + (size_t)m * R;
          uint32_t *cc = pcont + (size_t)m * R;
          uint32_t dsum = 0;
          if ((R & 3u) == 0) {
            const uint4 *rb4 = reinterpret_cast<const uint4 *>(rb);
            const uint4 *rr4 = reinterpret_cast<const uint4 *>(rr);
            uint4 *cc4 = reinterpret_cast<uint4 *>(cc);
            // Two 16-byte groups per lane and step, all six loads issued
            // before any store, so a step waits for one memory round trip
            // (shared memory when the pool fits there, else global).
            const uint32_t R4 = R >> 2;
            for (uint32_t q = lane; q < R4; q += 64) {
              const uint32_t q1 = q + 32;
              const uint4 z = make_uint4(0u, 0u, 0u, 0u);
              uint4 cv0 = cc4[q];
              const uint4 r0 = rr4[q], b0 = rb4[q];
              uint4 cv1 = z, r1 = z, b1 = z;
              if (q1 < R4) {
                cv1 = cc4[q1];
                r1 = rr4[q1];
                b1 = rb4[q1];
              }
              if (drop_shared4(cv0, r0, b0, dsum)) cc4[q] = cv0;
              if (drop_shared4(cv1, r1, b1, dsum)) cc4[q1] = cv1;
            }
          } else {
            for (uint32_t j = lane; j < R; j += 32) {
              const uint32_t cv = cc[j];
              if (cv && rr[j] == rb[j]) {
                dsum += cv;
                cc[j] = 0;
              }
            }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
          g -= dsum;
        }
        if (lane == 0) {
          s.pgain[cur ^ 1][m] = g;
          s.pactive[cur ^ 1][m] = act;
        }
      }
      cur ^= 1;
      __syncthreads();
      if (d.nsel >= a.K) break;
    }
    {
      // The pool's active gains are exact for the current seed set (a commit
      // updates them); exact gains of earlier rounds stay exact until the next
      // commit. Every thread reads the same final buffer.
      uint32_t rb = 0;
      for (uint32_t m = 0; m < np; ++m)
        if (s.pactive[cur][m] && s.pgain[cur][m] > rb) rb = s.pgain[cur][m];
      d.lb = ncm ? rb : (rb > d.lb ? rb : d.lb);
    }
    const long long t_cover = clock64();
    d.fine[0] += (unsigned long long)(t_cover - t_mark);
    // The round's seeds cover their components: the lanes whose contribution
    // is still > 0 are exactly those no earlier seed had covered.
    if ((R & 31u) == 0) {
      // With R a multiple of 32, lane j of an aligned group of 32 lanes owns
      // bit j & 31 of word (root * R + j) >> 5, so the lanes of a warp that
      // share a root set exactly the bits of their match mask: one atomic per
      // distinct word instead of one per lane.
      const uint32_t groups = R >> 5;
      for (uint32_t t = (uint32_t)warp; t < ncm * groups; t += kCelfWarps) {
        const uint32_t ci = t / groups;
        const uint32_t c = (uint32_t)s.committed[ci];
        const uint32_t j = (t - ci * groups) * 32 + (uint32_t)lane;
        uint32_t cv = pcont[(size_t)c * R + j];
        const uint32_t root = proot[(size_t)c * R + j];
        if (cv && root >= a.n) {  // never written by eval_items: record, skip the bit
          celf_violation(a, 2002u, root, ((uint64_t)c << 32) | j);
          cv = 0;
        }
        const uint32_t word = cv ? (root * R + j) >> 5 : 0xffffffffu;
        const unsigned peers = __match_any_sync(kFull, word);
        if (cv && lane == __ffs(peers) - 1) atomicOr(a.cov + word, peers);
      }
    } else {
      for (uint32_t i = tid; i < ncm * R; i += blockDim.x) {
        const uint32_t c = (uint32_t)s.committed[i / R], j = i % R;
        if (pcont[(size_t)c * R + j]) {
          const uint32_t root = proot[(size_t)c * R + j];
          if (root >= a.n) {
            celf_violation(a, 2002u, root, ((uint64_t)c << 32) | j);
            continue;
          }
          const uint32_t bit = root * R + j;
          atomicOr(a.cov + (bit >> 5), 1u << (bit & 31));
        }
      }
    }
    {
      const long long t_now = clock64();
      d.fine[1] += (unsigned long long)(t_now - t_cover);
      d.cyc[2] += (unsigned long long)(t_now - t_mark);
      t_mark = t_now;
    }
    if (d.nsel >= a.K) {
      __syncthreads();
      return leave(kCmdDone);
    }

    // ---------------------------------------------------------- merge survivors back
    if (warp == 0) {
      const bool alive = (uint32_t)lane < np && s.pactive[cur][lane];
      uint64_t y = alive ? make_key(s.pgain[cur][lane], s.pid[lane]) : 0ull;
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1) {  // bitonic sort across the warp, descending
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
          const uint64_t o = __shfl_xor_sync(kFull, y, j);
          const bool lower = (lane & j) == 0;
          const bool desc = (lane & k) == 0;
          y = (lower == desc) ? umax64(o, y) : umin64(o, y);
        }
      }
      s.Y[lane] = y;
      const unsigned ball = __ballot_sync(kFull, alive);
      if (lane == 0) s.ny = __popc(ball);
    }
    __syncthreads();
    {
      const uint32_t ny = s.ny;
      const uint32_t xs = d.head + np;  // rest of C: [xs, nC), sorted descending
      const uint32_t L = d.nC - xs;
      const uint32_t ob = xs - ny;      // merged output starts here
      uint64_t vx[kCap / kCelfThreads];
      uint32_t px[kCap / kCelfThreads];
#pragma unroll
      for (int q = 0; q < kCap / kCelfThreads; ++q) {
        const uint32_t i = (uint32_t)tid + (uint32_t)q * kCelfThreads;
        vx[q] = 0;
        px[q] = 0;
        if (i < L) {
          const uint64_t x = s.C[xs + i];
          uint32_t lo = 0, h2 = ny;  // number of Y greater than x
          while (lo < h2) {
            const uint32_t mid = (lo + h2) >> 1;
            if (s.Y[mid] > x) lo = mid + 1; else h2 = mid;
          }
          vx[q] = x;
          px[q] = ob + i + lo;
        }
      }
      uint64_t vy = 0;
      uint32_t py = 0;
      if ((uint32_t)tid < ny) {
        vy = s.Y[tid];
        uint32_t lo = 0, h2 = L;  // number of X greater than y
        while (lo < h2) {
          const uint32_t mid = (lo + h2) >> 1;
          if (s.C[xs + mid] > vy) lo = mid + 1; else h2 = mid;
        }
        py = ob + tid + lo;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kCap / kCelfThreads; ++q)
        if ((uint32_t)tid + (uint32_t)q * kCelfThreads < L) s.C[px[q]] = vx[q];
      if ((uint32_t)tid < ny) s.C[py] = vy;
      d.head = ob;
    }
    __syncthreads();
    {
      const long long t_now = clock64();
      d.cyc[3] += (unsigned long long)(t_now - t_mark);
      t_mark = t_now;
    }
  }
}

}  // namespace imgb
