// Spread of a seed set on the fixed hash samples: sigmaR(S) = sum_r
// |union_{s in S} C_r(s)| (Algorithm 4 evaluated on the samples of Eq. 2).
//
// Bit-parallel multi-source BFS over all R samples at once: every vertex has an
// R-bit visited mask V and a frontier mask F (bit j = internal lane j). A level
// is a list of work chunks (a frontier vertex u and the first of 32 of its
// arcs), one warp per chunk, so hubs spread over many warps. The warp holds u's frontier row
// in registers; for each arc u->v the edge hash selects the lane bucket that
// can be live (the same bucket test as the component kernel), and only the
// lanes of that bucket that are in u's frontier are tested against Eq. 2. v
// gains the live frontier lanes it has not seen (atomicOr on V[v] decides who
// won each bit); newly set bits form v's next frontier mask and are counted
// into sigmaR.
// Three frontier buffers rotate so that one grid-wide barrier per level
// suffices: level L reads F[L%3], writes F[(L+1)%3] and clears the rows of
// the level L-1 frontier in F[(L+2)%3]. Per-level counters and level stamps
// (instead of reset flags) build the frontier lists.
//
// The spread is reachability, not distance: BFS levels are only a schedule.
// A vertex reached at different depths in different samples is on several
// levels' frontiers and its arcs are scanned once per such level, so a seed
// set whose samples reach a giant component costs several scans of most of
// the graph. On tables larger than L2 the BFS therefore hands over when a
// frontier exceeds n/16 vertices (where the BFS's arcs per vertex, times the
// levels that rescan them, outweigh the R slots per vertex the components
// cost; the caller decides): the BFS initialises the label table, the
// components of every sample are formed by the select path's union-find (each
// edge once), every (seed, sample) pair marks its root, and sigmaR counts the
// (vertex, sample) slots whose root is marked (each slot once; no size memo).
// The hand-over kernels are queued behind every such BFS and return at once
// unless it handed over, so the choice costs no host round trip.
#include <cooperative_groups.h>

#include "im_common.cuh"

namespace cg = cooperative_groups;

namespace imgb {

struct SpreadArgs {
  const int32_t *xadj, *adj;
  uint32_t n, R, W;
  int32_t narcs;        // 2m
  const uint32_t *Xs, *boff;
  int nb;
  int boff_smem;        // the bucket offsets are staged in shared memory after the randoms
  uint32_t T32;
  int all_live;
  int precheck;         // read V before each atomicOr (table larger than L2)
  int xs_smem;          // the R lane randoms are staged in shared memory
  const uint8_t *mask;  // explicit-mask test mode: mask[arc * R + j]
  const int32_t *seeds;
  int num_seeds;
  uint32_t *V;
  uint32_t *F[3];
  int32_t *L[3];         // frontier vertices per level (for clearing F rows)
  uint64_t *Q[3];        // frontier work chunks per level: (vertex << 32) | first arc
  uint32_t *stamp;       // n: last list index (+1) a vertex was appended to
  uint32_t *cntlev;      // n + 4: frontier vertices per level
  uint32_t *chklev;      // n + 4: frontier chunks per level
  unsigned long long *acc;
  uint64_t *out;
  int32_t *status;
  unsigned long long *stats;
  uint32_t level_cap;    // budget of BFS levels (a BFS has at most n levels)
  unsigned long long *gate;  // hand-over word (null: the BFS always finishes)
  uint32_t handover;     // a frontier of more vertices hands over
  int32_t *P;            // hand-over: the label table (n R, set to -1) and the
  uint32_t *cov;         // marked-root bitmap (n R bits, cleared)
  int weighted, mix;     // sampling options: per-arc codes, mixed hash
  const uint32_t *code_arc;
};

template <class T>
__device__ __forceinline__ T pick3(T a0, T a1, T a2, uint32_t i) {
  return i == 0 ? a0 : (i == 1 ? a1 : a2);
}

__device__ __forceinline__ uint32_t lane_range_mask(uint32_t w, uint32_t j0, uint32_t j1) {
  const uint32_t b0 = w << 5;
  const uint32_t lo = j0 > b0 ? j0 - b0 : 0u;
  const uint32_t hi = j1 < b0 + 32u ? j1 - b0 : 32u;
  const uint32_t upper = hi >= 32u ? 0xffffffffu : ((1u << hi) - 1u);
  return upper & ~((1u << lo) - 1u);
}

// Append v to frontier list `lev` with one work chunk per 32 arcs.
__device__ __forceinline__ void push_frontier(const SpreadArgs &a, int32_t v, uint32_t lev,
                                              int32_t *Ln, uint64_t *Qn) {
  Ln[atomicAdd(a.cntlev + lev, 1u)] = v;
  const int32_t beg = a.xadj[v];
  const uint32_t deg = (uint32_t)(a.xadj[v + 1] - beg);
  const uint32_t nch = (deg + 31u) >> 5;
  if (nch) {
    const uint32_t at = atomicAdd(a.chklev + lev, nch);
    for (uint32_t c = 0; c < nch; ++c)
      Qn[at + c] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)(beg + (int32_t)(c << 5));
  }
}

// Live lanes among the frontier lanes f of word w (Eq. 2), two lanes per
// step so that their loads of X overlap; xs is the shared-memory copy of the
// lane randoms or the global one.
template <bool OPTS>
__device__ __forceinline__ uint32_t live_lanes(uint32_t f, uint32_t w, const uint32_t *xs,
                                               uint32_t h, uint32_t T32, int all_live,
                                               int weighted, uint32_t code, int mix) {
  uint32_t nbits = 0;
  while (f) {
    const int b0 = __ffs(f) - 1;
    f &= f - 1;
    const int b1 = f ? __ffs(f) - 1 : b0;  // a lone last lane is tested twice
    f &= f - 1;
    const uint32_t x0 = xs[(w << 5) + (uint32_t)b0];
    const uint32_t x1 = xs[(w << 5) + (uint32_t)b1];
    if (OPTS) {
      nbits |= (uint32_t)lane_live_opt(x0, h, T32, all_live, weighted, code, mix) << b0;
      nbits |= (uint32_t)lane_live_opt(x1, h, T32, all_live, weighted, code, mix) << b1;
    } else {
      nbits |= (uint32_t)lane_live(x0, h, T32, all_live) << b0;
      nbits |= (uint32_t)lane_live(x1, h, T32, all_live) << b1;
    }
  }
  return nbits;
}

// Up to this many lane randoms (32 KB) are staged in shared memory; the
// frontier-bit tests then read them there instead of through L1.
constexpr uint32_t kSpreadSmemLanes = 8192;

// Two blocks per SM (at most 64 registers): measured faster than one block
// with more registers and than three or four blocks with spills.
template <bool OPTS>
__global__ void __launch_bounds__(512, 2) k_spread(SpreadArgs a) {
  extern __shared__ uint32_t sXs[];
  cg::grid_group grid = cg::this_grid();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const uint64_t gwarp = tid >> 5, nwarps = nthr >> 5;
  const uint32_t W = a.W;
  const uint64_t nW = (uint64_t)a.n * W;

  for (uint64_t i = tid; i < nW; i += nthr) {
    a.V[i] = 0u;
    a.F[0][i] = 0u;
    a.F[1][i] = 0u;
    a.F[2][i] = 0u;
  }
  for (uint64_t i = tid; i < a.n; i += nthr) a.stamp[i] = 0u;
  for (uint64_t i = tid; i < (uint64_t)a.n + 4; i += nthr) {
    a.cntlev[i] = 0u;
    a.chklev[i] = 0u;
  }
  if (tid == 0) {
    *a.acc = 0ull;
    if (a.gate) *a.gate = 0ull;
  }
  if (a.xs_smem)
    for (uint32_t j = threadIdx.x; j < a.R; j += blockDim.x) sXs[j] = a.Xs[j];
  if (a.boff_smem)
    for (uint32_t j = threadIdx.x; j <= (1u << a.nb); j += blockDim.x) sXs[a.R + j] = a.boff[j];
  const uint32_t *boff = a.boff_smem ? sXs + a.R : a.boff;
  grid.sync();

  // sources: deduplicated seed set (list 0, stamp 1), all R lanes reached
  for (uint64_t i = tid; i < (uint64_t)a.num_seeds; i += nthr) {
    const int32_t s = a.seeds[i];
    if (s < 0 || (uint32_t)s >= a.n) {
      set_status(a.status, IM_EINVAL);
      continue;
    }
    if (atomicMax(a.stamp + s, 1u) < 1u) push_frontier(a, s, 0, a.L[0], a.Q[0]);
  }
  grid.sync();
  const uint32_t c0 = __ldcg(a.cntlev);
  const uint32_t lastmask = (a.R & 31u) ? ((1u << (a.R & 31u)) - 1u) : 0xffffffffu;
  for (uint64_t i = tid; i < (uint64_t)c0 * W; i += nthr) {
    const uint32_t k = (uint32_t)(i / W), w = (uint32_t)(i % W);
    const uint32_t m = (w == W - 1) ? lastmask : 0xffffffffu;
    const uint64_t o = (uint64_t)a.L[0][k] * W + w;
    a.V[o] = m;
    a.F[0][o] = m;
  }
  unsigned long long local = (tid == 0) ? (unsigned long long)c0 * a.R : 0ull;
  grid.sync();

  const bool row_in_regs = W <= 64;
  uint32_t level = 0;
  for (; level < a.level_cap; ++level) {
    const uint32_t cc = __ldcg(a.cntlev + level);
    if (cc == 0) break;
    if (a.gate && cc > a.handover) {  // the same decision in every thread
      if (tid == 0) {
        *a.gate = 1ull;
        if (a.stats) atomicAdd(a.stats + 3, (unsigned long long)level);
      }
      const uint64_t nR = (uint64_t)a.n * a.R;
      const int4 m1 = make_int4(-1, -1, -1, -1);
      for (uint64_t i = tid; i < (nR >> 2); i += nthr) reinterpret_cast<int4 *>(a.P)[i] = m1;
      for (uint64_t i = ((nR >> 2) << 2) + tid; i < nR; i += nthr) a.P[i] = -1;
      const uint64_t nc = (nR + 31) >> 5;
      const uint4 z = make_uint4(0, 0, 0, 0);
      for (uint64_t i = tid; i < (nc >> 2); i += nthr) reinterpret_cast<uint4 *>(a.cov)[i] = z;
      for (uint64_t i = ((nc >> 2) << 2) + tid; i < nc; i += nthr) a.cov[i] = 0u;
      return;
    }
    const uint32_t nq = __ldcg(a.chklev + level);
    const uint64_t *Qc = pick3(a.Q[0], a.Q[1], a.Q[2], level % 3);
    int32_t *Ln = pick3(a.L[0], a.L[1], a.L[2], (level + 1) % 3);
    uint64_t *Qn = pick3(a.Q[0], a.Q[1], a.Q[2], (level + 1) % 3);
    const uint32_t *Fc = pick3(a.F[0], a.F[1], a.F[2], level % 3);
    uint32_t *Fn = pick3(a.F[0], a.F[1], a.F[2], (level + 1) % 3);
    const uint32_t next_stamp = level + 2;
    // clear the frontier rows of level-1 (buffer (level+2)%3 is written next level)
    if (level > 0) {
      const uint32_t cp = __ldcg(a.cntlev + level - 1);
      const int32_t *Lp = pick3(a.L[0], a.L[1], a.L[2], (level + 2) % 3);
      uint32_t *Fp = pick3(a.F[0], a.F[1], a.F[2], (level + 2) % 3);
      // a row per group of gs threads (gs a power of two, the least >= W up to 32)
      const uint32_t lg = W >= 32u ? 5u : (uint32_t)(32 - __clz(W - 1u));
      const uint32_t gs = 1u << lg, rows = 32u >> lg;
      for (uint64_t k = gwarp * rows + ((uint32_t)lane >> lg); k < cp; k += nwarps * rows) {
        const uint64_t base = (uint64_t)Lp[k] * W;
        for (uint32_t w = (uint32_t)lane & (gs - 1u); w < W; w += gs) Fp[base + w] = 0u;
      }
    }
    // one warp per chunk of 32 arcs of a frontier vertex; the next chunk's
    // entry is loaded while this one runs
    uint64_t qnext = gwarp < nq ? Qc[gwarp] : 0ull;
    for (uint64_t q = gwarp; q < nq; q += nwarps) {
      const uint64_t qe = qnext;
      if (q + nwarps < nq) qnext = Qc[q + nwarps];
      const int32_t u = (int32_t)(qe >> 32);
      const uint32_t *fu = Fc + (uint64_t)u * W;
      // u's frontier row: word w sits in lane w & 31, register w >> 5
      uint32_t r0 = 0, r1 = 0;
      if (row_in_regs) {
        if ((uint32_t)lane < W) r0 = __ldcg(fu + lane);
        if ((uint32_t)lane + 32 < W) r1 = __ldcg(fu + lane + 32);
      }
      // the chunk's arcs and u's end load together (the entry holds the first arc)
      const uint32_t e = (uint32_t)qe + (uint32_t)lane;  // < 2^31 + 32
      const int32_t end = a.xadj[u + 1];
      const int32_t ve = e < (uint32_t)a.narcs ? a.adj[e] : -1;
      int32_t v = -1;
      uint32_t j0 = 0, j1 = 0, h = 0, code = 0;
      if (e < (uint32_t)end) {
        v = ve;
        if (v != u) {
          if (a.mask) {
            j1 = a.R;
          } else if (OPTS) {
            h = edge_hash(u, v);
            if (a.weighted) code = __ldg(a.code_arc + e);
            edge_lanes(h, a.nb, a.weighted, code, a.mix, boff, j0, j1);
          } else {
            h = edge_hash(u, v);
            const uint32_t b = lane_bucket(h, a.nb);
            j0 = boff[b];
            j1 = boff[b + 1];
          }
        }
      }
      bool tried = false, push = false;
      const uint32_t w0 = j0 >> 5;
      const uint32_t nw = j1 > j0 ? ((j1 - 1) >> 5) - w0 + 1 : 0u;
      uint32_t maxw = nw;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const uint32_t o = __shfl_xor_sync(kFull, maxw, d);
        maxw = o > maxw ? o : maxw;
      }
      for (uint32_t k = 0; k < maxw; ++k) {
        const uint32_t w = w0 + k;
        uint32_t f;
        if (row_in_regs) {
          const uint32_t src = w & 31u;
          const uint32_t x0 = __shfl_sync(kFull, r0, src);
          const uint32_t x1 = __shfl_sync(kFull, r1, src);
          f = (w >> 5) ? x1 : x0;
        } else {
          f = k < nw ? __ldcg(fu + w) : 0u;
        }
        if (k >= nw) continue;
        f &= lane_range_mask(w, j0, j1);
        uint32_t nbits = 0;
        if (a.mask) {
          while (f) {  // test only the frontier lanes of this word
            const int bit = __ffs(f) - 1;
            f &= f - 1;
            nbits |= (uint32_t)(a.mask[(uint64_t)e * a.R + (w << 5) + (uint32_t)bit] != 0) << bit;
          }
        } else if (a.xs_smem) {
          nbits = live_lanes<OPTS>(f, w, sXs, h, a.T32, a.all_live, a.weighted, code, a.mix);
        } else {
          nbits = live_lanes<OPTS>(f, w, a.Xs, h, a.T32, a.all_live, a.weighted, code, a.mix);
        }
        if (!nbits) continue;
        const uint64_t o = (uint64_t)v * W + w;
        // V only gains bits during the launch, so a word read from L2 that
        // already holds every live bit proves the atomic would gain nothing.
        // When V does not fit in L2, revisited hubs then cost a read instead
        // of an atomic; an L2-resident V takes the atomic at once.
        if (a.precheck && (__ldcg(a.V + o) & nbits) == nbits) continue;
        const uint32_t old = atomicOr(a.V + o, nbits);
        const uint32_t gained = nbits & ~old;
        if (!gained) continue;
        atomicOr(Fn + o, gained);
        local += __popc(gained);
        // One stamp attempt per chunk: after it, v is in the next list
        // whether this thread or another one put it there.
        if (!tried) {
          tried = true;
          push = atomicMax(a.stamp + v, next_stamp) < next_stamp;
        }
      }
      // The warp appends its new frontier vertices together: one atomic on
      // each level counter per warp, chunk slots from a warp prefix sum.
      const unsigned pm = __ballot_sync(kFull, push);
      if (pm) {
        uint32_t nch = 0;
        int32_t vbeg = 0;
        if (push) {
          vbeg = a.xadj[v];
          nch = ((uint32_t)(a.xadj[v + 1] - vbeg) + 31u) >> 5;
        }
        uint32_t incl = nch;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += t;
        }
        const uint32_t total = __shfl_sync(kFull, incl, 31);
        const int leader = __ffs(pm) - 1;
        uint32_t lbase = 0, qbase = 0;
        if (lane == leader) {
          lbase = atomicAdd(a.cntlev + level + 1, (uint32_t)__popc(pm));
          if (total) qbase = atomicAdd(a.chklev + level + 1, total);
        }
        lbase = __shfl_sync(kFull, lbase, leader);
        qbase = __shfl_sync(kFull, qbase, leader);
        if (push) {
          Ln[lbase + (uint32_t)__popc(pm & ((1u << lane) - 1u))] = v;
          const uint32_t q0 = qbase + incl - nch;
          for (uint32_t c = 0; c < nch; ++c)
            Qn[q0 + c] = ((uint64_t)(uint32_t)v << 32) | (uint32_t)(vbeg + (int32_t)(c << 5));
        }
      }
    }
    grid.sync();
  }
  if (level >= a.level_cap && tid == 0) set_status(a.status, IM_ETIMEOUT);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) local += __shfl_xor_sync(kFull, local, d);
  if (lane == 0 && local) atomicAdd(a.acc, local);
  grid.sync();
  if (tid == 0) {
    *a.out = (uint64_t)__ldcg(a.acc);
    if (a.stats) atomicAdd(a.stats + 3, (unsigned long long)level);
  }
}

// ------------------------------------------------------------ hand-over path
// After a hand-over the union's forest is in the label table: a root slot
// holds -1, any other slot a vertex of its component nearer the root. sigmaR
// (Eq. 2 summed over the samples) is the number of slots (v, j) whose
// component holds a seed in sample j: each (seed, sample) pair sets its
// root's bit in the covered bitmap (cleared by the BFS), then every slot walks
// to its root and counts itself if that bit is set.
struct SpreadCountArgs {
  const int32_t *P;      // the union's forest, n * R slots
  uint32_t n, R;
  uint32_t *cov;         // bit (root R + lane): the root's component holds a seed
  const int32_t *seeds;
  int num_seeds;
  uint32_t cap;          // walk budget (IM_ETIMEOUT past it)
  const unsigned long long *gate;
  unsigned long long *acc, *done;
  uint64_t *out;
  int32_t *status;
  unsigned long long *stats;
};

// Root of x in lane j of the forest, read only (the table is not written).
static __device__ __forceinline__ uint32_t forest_root(const int32_t *__restrict__ P, uint32_t R,
                                                       uint32_t cap, int32_t *status, uint32_t x,
                                                       uint32_t j) {
  for (uint32_t it = 0; it < cap; ++it) {
    const int32_t y = __ldg(P + x * R + j);
    if (y < 0) return x;
    x = (uint32_t)y;
  }
  set_status(status, IM_ETIMEOUT);
  return x;
}

// Every (seed, lane) pair marks the root of the seed's component.
__global__ void __launch_bounds__(256) k_spread_mark(SpreadCountArgs a) {
  if (__ldcg(a.gate) == 0ull) return;
  const uint64_t total = (uint64_t)a.num_seeds * a.R;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t s = a.seeds[i / a.R];
    const uint32_t j = (uint32_t)(i % a.R);
    if (s < 0 || (uint32_t)s >= a.n) continue;  // the BFS recorded IM_EINVAL
    const uint32_t bit = forest_root(a.P, a.R, a.cap, a.status, (uint32_t)s, j) * a.R + j;
    atomicOr(a.cov + (bit >> 5), 1u << (bit & 31u));
  }
}

// 1 when slot (v, j), holding x, lies in a marked component.
static __device__ __forceinline__ uint32_t slot_marked(const int32_t *__restrict__ P,
                                                       const uint32_t *__restrict__ cov, uint32_t R,
                                                       uint32_t cap, int32_t *status, int32_t x,
                                                       uint32_t v, uint32_t j) {
  const uint32_t bit = (x < 0 ? v : forest_root(P, R, cap, status, (uint32_t)x, j)) * R + j;
  return (__ldg(cov + (bit >> 5)) >> (bit & 31u)) & 1u;
}

// A warp per table row (lane-consecutive 16-byte loads, as the first-gains
// kernel reads it). Four root slots in a row test four consecutive bits of
// their own row's marks, one word; a non-root slot walks to its root. The
// last block writes sigmaR.
__global__ void __launch_bounds__(256, 4) k_spread_count(SpreadCountArgs a) {
  __shared__ unsigned long long s_sum[8];
  __shared__ bool s_last;
  if (__ldcg(a.gate) == 0ull) return;
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const int32_t *__restrict__ P = a.P;
  const uint32_t *__restrict__ cov = a.cov;
  const uint32_t R = a.R, n = a.n, cap = a.cap;
  int32_t *status = a.status;
  uint32_t cnt = 0;
  for (uint32_t v = gwarp; v < n; v += nwarps) {
    const uint32_t base = v * R;
    if ((R & 3u) == 0) {
      const int4 *row4 = reinterpret_cast<const int4 *>(P + base);
#pragma unroll 4
      for (uint32_t q4 = lane; q4 < (R >> 2); q4 += 32) {
        const int4 x = __ldg(row4 + q4);
        const uint32_t j = q4 << 2;
        if ((x.x & x.y & x.z & x.w) < 0) {  // four roots: bits base + j .. + 3
          const uint32_t b = base + j;
          cnt += __popc((__ldg(cov + (b >> 5)) >> (b & 31u)) & 0xfu);
        } else {
          cnt += slot_marked(P, cov, R, cap, status, x.x, v, j) +
                 slot_marked(P, cov, R, cap, status, x.y, v, j + 1) +
                 slot_marked(P, cov, R, cap, status, x.z, v, j + 2) +
                 slot_marked(P, cov, R, cap, status, x.w, v, j + 3);
        }
      }
    } else {
      for (uint32_t j = lane; j < R; j += 32)
        cnt += slot_marked(P, cov, R, cap, status, __ldg(P + base + j), v, j);
    }
  }
  unsigned long long sum = cnt;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
  if (lane == 0) s_sum[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_sum[w];
    if (b) atomicAdd(a.acc, b);
    __threadfence();
    s_last = atomicAdd(a.done, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    *a.out = (uint64_t)__ldcg(a.acc);
    *a.done = 0ull;
    if (a.stats) atomicAdd(a.stats + IM_STAT_SPREAD_COMPONENTS, 1ull);
  }
}

static SpreadCountArgs count_args(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                                  const int32_t *d_seeds, int num_seeds, uint64_t *d_sigma) {
  SpreadCountArgs a;
  a.P = ws->d_P;
  a.n = (uint32_t)g->n;
  a.R = q.R;
  a.cov = ws->d_cov;
  a.seeds = d_seeds;
  a.num_seeds = num_seeds;
  a.cap = uf_budget((uint32_t)g->n);
  a.gate = ws->d_acc + 1;
  a.acc = ws->d_acc;
  a.done = ws->d_acc + 2;
  a.out = d_sigma;
  a.status = ws->d_status;
  a.stats = ws->d_stats;
  return a;
}

cudaError_t launch_spread_mark(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                               const int32_t *d_seeds, int num_seeds, cudaStream_t s) {
  const SpreadCountArgs a = count_args(g, ws, q, d_seeds, num_seeds, nullptr);
  const uint64_t pairs = (uint64_t)num_seeds * q.R;
  uint64_t blocks = (pairs + 255) / 256;
  if (blocks > (uint64_t)g->num_sms * 4) blocks = (uint64_t)g->num_sms * 4;
  if (blocks == 0) blocks = 1;
  k_spread_mark<<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_spread_count(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                                uint64_t *d_sigma, cudaStream_t s) {
  const SpreadCountArgs a = count_args(g, ws, q, nullptr, 0, d_sigma);
  int per_sm = 0;
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_count, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t blocks = ((uint64_t)g->n + 7) / 8;  // a warp per row
  if (blocks > (uint64_t)g->num_sms * per_sm) blocks = (uint64_t)g->num_sms * per_sm;
  k_spread_count<<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_spread(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                          const int32_t *d_seeds, int num_seeds, const uint8_t *d_mask,
                          uint64_t *d_sigma, bool handover, cudaStream_t s) {
  SpreadArgs a;
  a.xadj = g->d_xadj;
  a.adj = g->d_adj;
  a.n = (uint32_t)g->n;
  a.R = q.R;
  a.W = (q.R + 31) / 32;
  a.narcs = (int32_t)(2 * g->m);
  a.Xs = ws->d_Xs;
  a.boff = ws->d_boff;
  a.nb = d_mask ? 0 : q.nb;
  a.T32 = q.T32;
  a.all_live = q.all_live;
  a.precheck = (uint64_t)g->n * a.W * 4u > (uint64_t)g->l2_bytes;
  a.mask = d_mask;
  a.seeds = d_seeds;
  a.num_seeds = num_seeds;
  a.V = ws->d_V;
  a.F[0] = ws->d_F0;
  a.F[1] = ws->d_F1;
  a.F[2] = ws->d_F2;
  a.L[0] = ws->d_L0;
  a.L[1] = ws->d_L1;
  a.L[2] = ws->d_L2;
  a.Q[0] = ws->d_Q0;
  a.Q[1] = ws->d_Q1;
  a.Q[2] = ws->d_Q2;
  a.stamp = ws->d_inlist;
  a.cntlev = ws->d_cnt;
  a.chklev = ws->d_cnt + (g->n + 4);
  a.acc = ws->d_acc;
  a.out = d_sigma;
  a.status = ws->d_status;
  a.stats = ws->d_stats;
  a.weighted = q.weighted;
  a.mix = q.mix;
  a.code_arc = g->d_code_arc;
  a.level_cap = (uint32_t)g->n + 2u;
  a.gate = handover ? ws->d_acc + 1 : nullptr;
  a.handover = (uint32_t)(g->n / 16);
  a.P = ws->d_P;
  a.cov = ws->d_cov;
  const int64_t lo = override_value(IM_OVR_SPREAD_LEVEL_CAP);
  if (lo > 0 && (uint64_t)lo < a.level_cap) a.level_cap = (uint32_t)lo;
  a.xs_smem = (!d_mask && q.R <= kSpreadSmemLanes) ? 1 : 0;
  // the bucket offsets follow the randoms while both fit the default 48 KB
  const size_t nboff = d_mask ? 0 : ((size_t)1 << a.nb) + 1;
  a.boff_smem = (a.xs_smem && (q.R + nboff) * sizeof(uint32_t) <= 48 * 1024) ? 1 : 0;
  const size_t smem = a.xs_smem ? (q.R + (a.boff_smem ? nboff : 0)) * sizeof(uint32_t) : 0;
  const void *fn = (!d_mask && (q.weighted || q.mix)) ? (const void *)k_spread<true>
                                                       : (const void *)k_spread<false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 512, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > 2) per_sm = 2;
  // Small tables: one block per SM keeps the per-level grid barrier cheap and
  // leaves room for queries running concurrently on other streams.
  if ((uint64_t)g->n * a.W < (4u << 20)) per_sm = 1;
  dim3 grid(g->num_sms * per_sm), block(512);
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s);
}

}  // namespace imgb
