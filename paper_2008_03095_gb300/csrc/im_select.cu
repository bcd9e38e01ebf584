// Fused hash-sample + connected components of all R samples, size memo and
// first-seed gains (Algorithm 5, NewGreedyStep-Vec, redesigned for sm_103a).
//
// Kernels, in launch order for one query:
//   k_prep     block 0: X_0..X_{R-1} = MT19937(seed) and the lane order
//              (lanes sorted by the top bits of X); other blocks: label table
//              init P = -1 ("every vertex its own component", Alg. 5 lines
//              1-2) and covered-bitmap clear, 128-bit stores.
//   k_union    one pass over the upper-triangle edge list: for every edge the
//              hash h (Eq. 1) selects the only lane bucket whose lanes can be
//              live (Eq. 2 needs the top bits of X_r and h to agree), each
//              candidate lane is tested and live lanes hook the two components.
//   k_compress every non-root slot is pointed at its root and counted into the
//              root slot, which ends as -(component size) (Section 3.3).
//   k_gains    mg_v = sum_r |C_r(v)| per vertex (Alg. 5 final loop), packed as
//              the CELF key (mg << 32 | ~v).
#include <cooperative_groups.h>

#include "im_common.cuh"
#include "im_lanes.cuh"
#include "im_union.cuh"

namespace imgb {

struct PrepArgs {
  // lanes
  uint32_t seed, R;
  int nb;
  uint32_t *X, *Xs, *perm, *boff, *sortbuf;
  uint64_t *keyrange;
  // init
  int32_t *P;
  uint64_t nR;
  uint32_t *cov;
  uint64_t ncov;
};

__device__ void prep_lanes(const PrepArgs &a, uint32_t *s_sort) {
  draw_lanes(a.seed, a.R, a.nb, a.X, a.Xs, a.perm, a.boff, s_sort, a.sortbuf, a.keyrange);
}

__global__ void __launch_bounds__(512) k_prep(PrepArgs a) {
  extern __shared__ uint32_t s_sort[];
  if (blockIdx.x == 0) {
    prep_lanes(a, s_sort);
    return;
  }
  const uint64_t tid = (uint64_t)(blockIdx.x - 1) * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)(gridDim.x - 1) * blockDim.x;
  if (a.P) {
    const int4 m1 = make_int4(-1, -1, -1, -1);
    int4 *p4 = reinterpret_cast<int4 *>(a.P);
    const uint64_t n4 = a.nR >> 2;
    for (uint64_t i = tid; i < n4; i += nthr) p4[i] = m1;
    for (uint64_t i = (n4 << 2) + tid; i < a.nR; i += nthr) a.P[i] = -1;
  }
  if (a.cov) {
    const uint4 z = make_uint4(0, 0, 0, 0);
    uint4 *c4 = reinterpret_cast<uint4 *>(a.cov);
    const uint64_t n4 = a.ncov >> 2;
    for (uint64_t i = tid; i < n4; i += nthr) c4[i] = z;
    for (uint64_t i = (n4 << 2) + tid; i < a.ncov; i += nthr) a.cov[i] = 0u;
  }
}

size_t lane_sort_smem(uint32_t R) {
  size_t npow2 = 1;
  while (npow2 < R) npow2 <<= 1;
  return npow2 <= (size_t)kSortSmemMax ? npow2 * sizeof(uint32_t) : 0;
}

cudaError_t launch_prep(const im_workspace *ws, const QueryParams &q, bool init_table,
                        bool zero_cov, cudaStream_t s) {
  const im_graph *g = ws->g;
  PrepArgs a;
  a.seed = q.seed;
  a.R = q.R;
  a.nb = q.nb;
  a.X = ws->d_X;
  a.Xs = ws->d_Xs;
  a.perm = ws->d_perm;
  a.boff = ws->d_boff;
  a.sortbuf = ws->d_sortbuf;
  a.keyrange = ws->d_keyrange;
  a.nR = (uint64_t)g->n * q.R;
  a.P = init_table ? ws->d_P : nullptr;
  a.ncov = (a.nR + 31) >> 5;
  a.cov = zero_cov ? ws->d_cov : nullptr;
  size_t smem = lane_sort_smem(q.R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSortSmemMax * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
  }
  int init_blocks = (init_table || zero_cov) ? g->num_sms * 3 : 0;
  k_prep<<<1 + init_blocks, 512, smem, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ union
template <bool MASKED, bool OPTS>
__global__ void __launch_bounds__(256) k_union(UnionArgs a) {
  extern __shared__ uint32_t s_boff[];
  if (a.gate && __ldcg(a.gate) == 0ull) return;
  if (!MASKED) {
    const int nbk = 1 << a.nb;
    for (int i = threadIdx.x; i <= nbk; i += blockDim.x) s_boff[i] = a.boff[i];
    __syncthreads();
  }
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32; base < a.m_up; base += nwarps * 32)
    union_group<MASKED, OPTS, false>(a, s_boff, base, a.m_up);
}

cudaError_t launch_union(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                         const uint8_t *d_mask, cudaStream_t s, const unsigned long long *gate) {
  if (g->m_up == 0) return cudaSuccess;
  UnionArgs a;
  a.eu = g->d_eu;
  a.ev = g->d_ev;
  a.m_up = g->m_up;
  a.Xs = ws->d_Xs;
  a.boff = ws->d_boff;
  a.nb = q.nb;
  a.T32 = q.T32;
  a.all_live = q.all_live;
  a.R = q.R;
  a.cap = uf_budget((uint32_t)g->n);
  a.P = ws->d_P;
  a.status = ws->d_status;
  a.mask = d_mask;
  a.xadj = g->d_xadj;
  a.adj = g->d_adj;
  a.weighted = q.weighted;
  a.mix = q.mix;
  a.code_up = g->d_code_up;
  a.gate = gate;
  int64_t warps_needed = (g->m_up + 31) / 32;
  int64_t blocks = (warps_needed + 7) / 8;
  int64_t cap = (int64_t)g->num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (d_mask) {
    k_union<true, false><<<(unsigned)blocks, 256, 0, s>>>(a);
  } else {
    size_t smem = ((1u << q.nb) + 1) * sizeof(uint32_t);
    if (q.weighted || q.mix)
      k_union<false, true><<<(unsigned)blocks, 256, smem, s>>>(a);
    else
      k_union<false, false><<<(unsigned)blocks, 256, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ compress
// The size memo's walk depends on the samples: where a sample holds a large
// component (a share of the vertices above kMemoAccShare), nearly every tile
// of a lane adds to its root slot, those atomics pile onto one L2 slice, and
// the warps' root-count accumulators pay (on the 4M-vertex power-law graph,
// 7.6 vs 9.7 ms); where components are small, the plain walk with path
// compression does the least work per slot (the clustered 335k-vertex graph:
// 1.36 vs 2.07 ms). A one-block-per-lane probe estimates the share from the
// union-find table before the size memo: in kProbeLanes lanes spread over R,
// kProbeVertices vertices (a multiplicative hash of the index) are walked to
// their roots and the most frequent root's count is summed; the last block
// writes the choice. 16 x 256 samples put the estimate within about 0.3% of
// the share near the threshold. The probe also counts the sampled slots that
// are not roots: below kMemoLiveShare of them, the accumulator walk lists a
// warp's few non-root slots and walks only those (4M-vertex graph, 10% of
// slots: 6.73 vs 7.60 ms); above it the list takes several passes and the
// walk over all four items of a thread is faster (the 37k-vertex graph at
// p = 0.05, 27%: 323 vs 373 µs).
constexpr uint32_t kProbeLanes = 16, kProbeVertices = 256;
constexpr double kMemoAccShare = 0.045, kMemoLiveShare = 0.15;
enum : unsigned long long { kMemoPlain = 0, kMemoAcc = 1, kMemoNone = 2, kMemoAccLive = 3 };

__global__ void __launch_bounds__(kProbeVertices) k_memo_probe(const int32_t *P, uint32_t n,
                                                               uint32_t R, uint32_t cap,
                                                               int32_t *status,
                                                               unsigned long long *probe,
                                                               unsigned long long *stats,
                                                               const unsigned long long *gate) {
  // probe[0]: the choice (kMemo*; kMemoNone when the gate is closed);
  // [1]: summed mode counts; [2]: blocks done; [3]: non-root samples
  __shared__ uint32_t s_root[kProbeVertices];
  __shared__ uint32_t s_max[kProbeVertices / 32], s_nr[kProbeVertices / 32];
  __shared__ bool s_last;
  if (gate && __ldcg(gate) == 0ull) {
    if (blockIdx.x == 0 && threadIdx.x == 0) probe[0] = kMemoNone;
    return;
  }
  const uint32_t j = (uint32_t)(((uint64_t)blockIdx.x * R) / gridDim.x);
  const uint32_t v = (uint32_t)(((uint64_t)threadIdx.x * 2654435761u + blockIdx.x) % n);
  uint32_t r = v;
  int32_t x = __ldcg(P + (uint64_t)v * R + j);
  const unsigned nr = __ballot_sync(kFull, x >= 0);
  for (uint32_t it = 0; x >= 0; ++it) {
    if (it >= cap) {
      set_status(status, IM_ETIMEOUT);
      break;
    }
    r = (uint32_t)x;
    x = __ldcg(P + (uint64_t)r * R + j);
  }
  s_root[threadIdx.x] = r;
  __syncthreads();
  uint32_t c = 0;
  for (uint32_t k = 0; k < kProbeVertices; ++k) c += s_root[k] == r;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint32_t o = __shfl_xor_sync(kFull, c, d);
    c = o > c ? o : c;
  }
  if ((threadIdx.x & 31) == 0) {
    s_max[threadIdx.x >> 5] = c;
    s_nr[threadIdx.x >> 5] = (uint32_t)__popc(nr);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0, nrs = 0;
    for (uint32_t w = 0; w < kProbeVertices / 32; ++w) {
      m = s_max[w] > m ? s_max[w] : m;
      nrs += s_nr[w];
    }
    atomicAdd(probe + 1, (unsigned long long)m);
    atomicAdd(probe + 3, (unsigned long long)nrs);
    __threadfence();
    s_last = atomicAdd(probe + 2, 1ull) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const double samples = (double)gridDim.x * kProbeVertices;
    const double share = (double)__ldcg(probe + 1) / samples;
    const double nonroot = (double)__ldcg(probe + 3) / samples;
    probe[0] = share > kMemoAccShare ? (nonroot < kMemoLiveShare ? kMemoAccLive : kMemoAcc)
                                     : kMemoPlain;
    if (probe[0] != kMemoPlain && stats) atomicAdd(stats + IM_STAT_MEMO_ACCUMULATORS, 1ull);
    if (probe[0] == kMemoAccLive && stats) atomicAdd(stats + IM_STAT_MEMO_LIVE, 1ull);
    probe[1] = 0ull;
    probe[2] = 0ull;
    probe[3] = 0ull;
  }
}

// Eight blocks per SM (32 registers): measured faster than six or three
// blocks with more registers. The three instances are queued; the two that
// *mode (from k_memo_probe) does not pick return at once (holding the walks
// in one kernel, behind a run-time branch or as non-inlined loops, compiled
// the accumulator walk 3-45% slower). Tile t covers vertices 32 (t / tl) ..,
// lanes 32 (t % tl) ..; n R < 2^32 keeps the tile count within 32 bits.
template <bool ACC, bool LIVE = false>
__global__ void __launch_bounds__(256, 8) k_compress(int32_t *P, uint32_t n, uint32_t R,
                                                     int32_t *status, uint32_t cap,
                                                     const unsigned long long *mode) {
  __shared__ int32_t tile[kCompV][kCompL + 1];
  __shared__ RootAcc s_acc[ACC ? 8 : 1];
  const uint32_t tl = (R + kCompL - 1) / kCompL;
  const uint32_t ntiles = (n + kCompV - 1) / kCompV * tl;
  uint32_t t = blockIdx.x;
  if (t >= ntiles || __ldcg(mode) != (ACC ? (LIVE ? kMemoAccLive : kMemoAcc) : kMemoPlain)) return;
  const uint32_t gq = gridDim.x / tl, gr = gridDim.x % tl;  // the grid stride in tiles
  uint32_t tv = t / tl, tj = t % tl;
  // The next tile's rows are loaded while the current tile's chains are
  // walked. A prefetched slot may predate another tile's root write or root
  // count: a parent pointer then still leads to the same root, and a root
  // slot is still negative, so the result is the same.
  int32_t e[4];
  compress_load(P, n, R, tv * kCompV, tj * kCompL, threadIdx.x, e);
  RootAcc *acc = s_acc + (ACC ? (threadIdx.x >> 5) : 0);
  if (ACC) root_acc_clear(acc, threadIdx.x);
  uint32_t acc_tj = tj;  // the lanes the accumulators count for
  for (; t < ntiles; t += gridDim.x) {
    compress_stage(e, threadIdx.x, tile);
    group_sync<0>();
    uint32_t nv = tv + gq, nj = tj + gr;
    if (nj >= tl) {
      nj -= tl;
      ++nv;
    }
    if (t + gridDim.x < ntiles) compress_load(P, n, R, nv * kCompV, nj * kCompL, threadIdx.x, e);
    if (ACC) {
      if (tj != acc_tj) {
        root_acc_flush(P, R, acc_tj * kCompL, threadIdx.x, acc);
        acc_tj = tj;
      }
      if (LIVE)
        compress_walk_acc_live<0>(P, R, status, cap, tv * kCompV, tj * kCompL, tile, threadIdx.x,
                                  acc);
      else
        compress_walk_acc<0>(P, R, status, cap, tv * kCompV, tj * kCompL, tile, threadIdx.x, acc);
    } else {
      compress_walk<0>(P, R, status, cap, tv * kCompV, tj * kCompL, tile, threadIdx.x);
    }
    tv = nv;
    tj = nj;
  }
  if (ACC) root_acc_flush(P, R, acc_tj * kCompL, threadIdx.x, acc);
}

cudaError_t launch_compress(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                            cudaStream_t s, const unsigned long long *gate) {
  unsigned long long *probe = ws->d_acc + 3;
  const uint32_t cap = uf_budget((uint32_t)g->n);
  k_memo_probe<<<kProbeLanes, kProbeVertices, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R, cap,
                                                      ws->d_status, probe, ws->d_stats, gate);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  api_count_launch();
  const uint64_t tl = (q.R + kCompL - 1) / kCompL;
  const uint64_t ntiles = ((uint64_t)g->n + kCompV - 1) / kCompV * tl;
  uint64_t blocks = ntiles;
  const uint64_t bcap = (uint64_t)g->num_sms * 8;
  // a grid of whole lane groups keeps each block on one set of lanes, so its
  // root-count accumulators are paid once at the end
  if (blocks > bcap) blocks = bcap >= tl ? bcap / tl * tl : bcap;
  if (blocks == 0) blocks = 1;
  k_compress<true, true><<<(unsigned)blocks, 256, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R,
                                                          ws->d_status, cap, probe);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  api_count_launch();
  k_compress<true><<<(unsigned)blocks, 256, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R, ws->d_status,
                                                    cap, probe);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  api_count_launch();
  k_compress<false><<<(unsigned)blocks, 256, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R, ws->d_status,
                                                     cap, probe);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ first gains
__device__ __forceinline__ uint32_t slot_size(const int32_t *P, int32_t x, uint32_t j,
                                              uint32_t R) {
  return x < 0 ? (uint32_t)(-x) : (uint32_t)(-__ldg(P + (uint32_t)x * R + j));
}

__global__ void __launch_bounds__(256) k_gains(const int32_t *__restrict__ P, uint32_t n,
                                               uint32_t R, uint64_t *keys, uint64_t *keyrange) {
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint64_t kmin = ~0ull, kmax = 0ull;
  for (uint32_t v = gwarp; v < n; v += nwarps) {
    const int32_t *row = P + (uint64_t)v * R;
    uint32_t sum = 0;
    if ((R & 3u) == 0) {
      const int4 *row4 = reinterpret_cast<const int4 *>(row);
      const uint32_t R4 = R >> 2;
#pragma unroll 4
      for (uint32_t q4 = lane; q4 < R4; q4 += 32) {
        const int4 x = __ldg(row4 + q4);
        const uint32_t j = q4 << 2;
        sum += slot_size(P, x.x, j, R) + slot_size(P, x.y, j + 1, R) +
               slot_size(P, x.z, j + 2, R) + slot_size(P, x.w, j + 3, R);
      }
    } else {
      for (uint32_t j = lane; j < R; j += 32) sum += slot_size(P, __ldg(row + j), j, R);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
    const uint64_t key = ((uint64_t)sum << 32) | (uint64_t)(0xffffffffu - v);
    if (lane == 0) keys[v] = key;
    kmin = key < kmin ? key : kmin;
    kmax = key > kmax ? key : kmax;
  }
  if (lane == 0 && kmax != 0ull) {
    atomicMin(reinterpret_cast<unsigned long long *>(keyrange), (unsigned long long)kmin);
    atomicMax(reinterpret_cast<unsigned long long *>(keyrange + 1), (unsigned long long)kmax);
  }
}

cudaError_t launch_gains(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                         cudaStream_t s) {
  uint64_t blocks = ((uint64_t)g->n + 7) / 8;
  uint64_t cap = (uint64_t)g->num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_gains<<<(unsigned)blocks, 256, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R, ws->d_keys,
                                           ws->d_keyrange);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ test hooks
// Paper layout of the tables: labels[v*R + r] and sizes[l*R + r] by simulation
// index r (the internal lane j maps to r = perm[j]).
__global__ void k_expand(const int32_t *P, const uint32_t *perm, uint32_t n, uint32_t R,
                         int32_t *labels, uint32_t *sizes) {
  const uint64_t nR = (uint64_t)n * R;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nR;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(i / R), j = (uint32_t)(i % R);
    const int32_t x = P[i];
    const uint64_t o = (uint64_t)v * R + perm[j];
    if (labels) labels[o] = x < 0 ? (int32_t)v : x;
    if (sizes) sizes[o] = x < 0 ? (uint32_t)(-x) : 0u;
  }
}

cudaError_t launch_expand(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                          int32_t *d_labels, uint32_t *d_sizes, cudaStream_t s) {
  k_expand<<<g->num_sms * 4, 256, 0, s>>>(ws->d_P, ws->d_perm, (uint32_t)g->n, q.R, d_labels,
                                          d_sizes);
  return cudaGetLastError();
}

// Selected simulations only: lanes[k] is the internal lane of the k-th
// requested simulation; out[v*nl + k] in the layout of the size memo.
__global__ void k_gather_lanes(const int32_t *P, const uint32_t *lanes, uint32_t n, uint32_t R,
                               uint32_t nl, int32_t *labels, uint32_t *sizes) {
  const uint64_t total = (uint64_t)n * nl;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(i / nl), k = (uint32_t)(i % nl);
    const int32_t x = P[(uint64_t)v * R + lanes[k]];
    labels[i] = x < 0 ? (int32_t)v : x;
    sizes[i] = x < 0 ? (uint32_t)(-x) : 0u;
  }
}

cudaError_t launch_gather_lanes(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                                const uint32_t *d_lanes, uint32_t nl, int32_t *d_labels,
                                uint32_t *d_sizes, cudaStream_t s) {
  k_gather_lanes<<<g->num_sms * 4, 256, 0, s>>>(ws->d_P, d_lanes, (uint32_t)g->n, q.R, nl,
                                                d_labels, d_sizes);
  return cudaGetLastError();
}

__global__ void k_edge_hash(const int32_t *u, const int32_t *v, int64_t count, uint32_t *h) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    h[i] = edge_hash(u[i], v[i]);
}

cudaError_t launch_edge_hash(const int32_t *d_u, const int32_t *d_v, int64_t count,
                             uint32_t *d_h, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_edge_hash<<<(unsigned)blocks, 256, 0, s>>>(d_u, d_v, count, d_h);
  return cudaGetLastError();
}

}  // namespace imgb
