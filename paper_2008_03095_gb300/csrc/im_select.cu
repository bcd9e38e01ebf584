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

namespace imgb {

// ------------------------------------------------------------------ MT19937
// Matsumoto & Nishimura (1998), 32-bit: n = 624, m = 397, matrix 0x9908b0df,
// tempering (11, 7 0x9d2c5680, 15 0xefc60000, 18), init multiplier 1812433253.
// The state refresh ("twist") is done by one block in four dependency-safe
// phases: entries [0,227) read only old state, [227,454) and [454,623) read
// entries refreshed by the previous phase, and entry 623 reads entry 0.
__device__ __forceinline__ uint32_t mt_next_word(uint32_t cur, uint32_t nxt, uint32_t far) {
  uint32_t y = (cur & 0x80000000u) | (nxt & 0x7fffffffu);
  return far ^ (y >> 1) ^ ((y & 1u) ? 0x9908b0dfu : 0u);
}

__device__ void mt_twist(uint32_t *mt) {
  const int t = threadIdx.x;
  uint32_t nv = 0;
  if (t < 227) nv = mt_next_word(mt[t], mt[t + 1], mt[t + 397]);
  __syncthreads();
  if (t < 227) mt[t] = nv;
  __syncthreads();
  if (t < 227) nv = mt_next_word(mt[t + 227], mt[t + 228], mt[t]);
  __syncthreads();
  if (t < 227) mt[t + 227] = nv;
  __syncthreads();
  if (t < 169) nv = mt_next_word(mt[t + 454], mt[t + 455], mt[t + 227]);
  __syncthreads();
  if (t < 169) mt[t + 454] = nv;
  __syncthreads();
  if (t == 0) mt[623] = mt_next_word(mt[623], mt[0], mt[396]);
  __syncthreads();
}

__device__ __forceinline__ uint32_t mt_temper(uint32_t y) {
  y ^= y >> 11;
  y ^= (y << 7) & 0x9d2c5680u;
  y ^= (y << 15) & 0xefc60000u;
  y ^= y >> 18;
  return y;
}

// Ascending bitonic sort of npow2 keys (shared or global memory) by one block.
__device__ void block_bitonic_sort(uint32_t *a, int npow2) {
  for (int k = 2; k <= npow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint32_t x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

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
  __shared__ uint32_t mt[624];
  const int t = threadIdx.x;
  if (t == 0) {  // the seeding recurrence is sequential; keep it in a register
    uint32_t x = a.seed;
    mt[0] = x;
    for (int i = 1; i < 624; ++i) {
      x = 1812433253u * (x ^ (x >> 30)) + (uint32_t)i;
      mt[i] = x;
    }
  }
  __syncthreads();
  for (uint32_t base = 0; base < a.R; base += 624) {
    mt_twist(mt);
    for (uint32_t i = t; i < 624 && base + i < a.R; i += blockDim.x) a.X[base + i] = mt_temper(mt[i]);
    __syncthreads();
  }
  // Lane order: sort keys (bucket << 16 | r); a stable, deterministic order.
  int npow2 = 1;
  while (npow2 < (int)a.R) npow2 <<= 1;
  uint32_t *keys = (npow2 <= kSortSmemMax) ? s_sort : a.sortbuf;
  for (int i = t; i < npow2; i += blockDim.x)
    keys[i] = (i < (int)a.R) ? ((lane_bucket(a.X[i], a.nb) << 16) | (uint32_t)i) : 0xffffffffu;
  __syncthreads();
  if (a.nb > 0) block_bitonic_sort(keys, npow2);
  for (uint32_t j = t; j < a.R; j += blockDim.x) {
    const uint32_t r = keys[j] & 0xffffu;
    a.perm[j] = r;
    a.Xs[j] = a.X[r];
  }
  // boff[b] = first internal lane whose bucket is >= b
  const uint32_t nbk = 1u << a.nb;
  for (uint32_t b = t; b <= nbk; b += blockDim.x) {
    uint32_t lo = 0, hi = a.R;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if ((keys[mid] >> 16) < b) lo = mid + 1; else hi = mid;
    }
    a.boff[b] = lo;
  }
  if (t == 0 && a.keyrange) {
    a.keyrange[0] = ~0ull;
    a.keyrange[1] = 0ull;
  }
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
struct UnionArgs {
  const int32_t *eu, *ev;
  int64_t m_up;
  const uint32_t *Xs, *boff;
  int nb;
  uint32_t T32;
  int all_live;
  uint32_t R;
  uint32_t cap;
  int32_t *P;
  int32_t *status;
  // sampling options: per-edge codes (weighted), mixed hash
  int weighted, mix;
  const uint32_t *code_up;
  // explicit-mask mode (test hook)
  const uint8_t *mask;
  const int32_t *xadj, *adj;
};

// OPTS: the sampling options (per-edge threshold codes, mixed hash) are in
// play; the uniform-p path keeps its own instantiation.
template <bool MASKED, bool OPTS>
__global__ void __launch_bounds__(256) k_union(UnionArgs a) {
  extern __shared__ uint32_t s_boff[];
  if (!MASKED) {
    const int nbk = 1 << a.nb;
    for (int i = threadIdx.x; i <= nbk; i += blockDim.x) s_boff[i] = a.boff[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gwarp * 32; base < a.m_up; base += nwarps * 32) {
    const int64_t e = base + lane;
    const bool valid = e < a.m_up;
    int32_t u = 0, v = 0;
    uint32_t h = 0, j0 = 0, c = 0, code = 0;
    if (valid) {
      u = a.eu[e];
      v = a.ev[e];
      if (MASKED) {
        c = a.R;
      } else if (OPTS) {
        h = edge_hash_ordered((uint32_t)u, (uint32_t)v);
        if (a.weighted) code = a.code_up[e];
        uint32_t j1;
        edge_lanes(h, a.nb, a.weighted, code, a.mix, s_boff, j0, j1);
        c = j1 - j0;
      } else {
        h = edge_hash_ordered((uint32_t)u, (uint32_t)v);
        const uint32_t b = lane_bucket(h, a.nb);
        j0 = s_boff[b];
        c = s_boff[b + 1] - j0;
      }
    }
    // Flatten the (edge, candidate lane) pairs of the 32 edges: item k of the
    // warp belongs to the edge whose inclusive prefix first exceeds k.
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t k = 0; k < total; k += 32) {
      const uint32_t item = k + lane;
      int pos = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        uint32_t val = __shfl_sync(kFull, incl, pos + step - 1);
        if (val <= item) pos += step;
      }
      const uint32_t s_incl = __shfl_sync(kFull, incl, pos);
      const uint32_t s_c = __shfl_sync(kFull, c, pos);
      const uint32_t s_j0 = __shfl_sync(kFull, j0, pos);
      const uint32_t s_h = __shfl_sync(kFull, h, pos);
      const int32_t s_u = __shfl_sync(kFull, u, pos);
      const int32_t s_v = __shfl_sync(kFull, v, pos);
      const uint32_t s_code = OPTS ? __shfl_sync(kFull, code, pos) : 0u;
      if (item < total) {
        const uint32_t j = s_j0 + (item - (s_incl - s_c));
        bool live;
        if (MASKED) {
          int32_t lo = a.xadj[s_u], hi = a.xadj[s_u + 1];
          while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (a.adj[mid] < s_v) lo = mid + 1; else hi = mid;
          }
          live = a.mask[(uint64_t)lo * a.R + j] != 0;
        } else if (OPTS) {
          live = lane_live_opt(__ldg(a.Xs + j), s_h, a.T32, a.all_live, a.weighted, s_code,
                               a.mix);
        } else {
          live = lane_live(__ldg(a.Xs + j), s_h, a.T32, a.all_live);
        }
        if (live) uf_unite(s_u, s_v, j, a.R, a.P, a.status, a.cap);
      }
    }
  }
}

cudaError_t launch_union(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                         const uint8_t *d_mask, cudaStream_t s) {
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
// Size memo (Section 3.3): every non-root slot gets its root (the component
// minimum) and each root slot accumulates -|component|. The label table is
// processed in tiles of 32 vertices x 32 lanes: the block loads a tile with
// sector-sized row reads, then warp w takes lane j0 + w of the 32 vertices,
// so the parent lookups of a warp hit one lane (vertices that share a parent,
// as in a giant component, coalesce into one request) and the root counters
// take one atomic per distinct root per warp instead of one per slot. Root
// slots are never written here except by those atomics.
constexpr uint32_t kCompV = 32;  // vertices per tile (one per warp lane)
constexpr uint32_t kCompL = 32;  // lanes per tile (four per warp of the block)

__global__ void __launch_bounds__(256) k_compress(int32_t *P, uint32_t n, uint32_t R,
                                                  int32_t *status, uint32_t cap) {
  __shared__ int32_t tile[kCompV][kCompL + 1];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint64_t tv = (n + kCompV - 1) / kCompV, tl = (R + kCompL - 1) / kCompL;
  const uint64_t ntiles = tv * tl;
  const bool vec = (R & 3u) == 0;  // rows start 16-byte aligned
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t v0 = (uint32_t)(t / tl) * kCompV, j0 = (uint32_t)(t % tl) * kCompL;
    {
      // thread: row tid / 8, lanes 4 * (tid % 8) .. + 3 of the tile
      const uint32_t rr = tid >> 3, c0 = (tid & 7u) * 4u;
      const uint32_t v = v0 + rr, j = j0 + c0;
      int32_t e[4] = {-1, -1, -1, -1};
      if (v < n) {
        const int32_t *row = P + (uint64_t)v * R;
        if (vec && j + 3 < R) {
          const int4 x4 = __ldcg(reinterpret_cast<const int4 *>(row + j));
          e[0] = x4.x; e[1] = x4.y; e[2] = x4.z; e[3] = x4.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (j + q < R) e[q] = __ldcg(row + j + q);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) tile[rr][c0 + q] = e[q];
    }
    __syncthreads();
    // warp w: tile lanes w, w + 8, w + 16, w + 24 of the 32 vertices; the
    // first parent loads of the four items are issued together
    const uint32_t v = v0 + lane;
    int32_t x[4], r[4];
    bool live[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x[q] = tile[lane][warp + 8u * q];
      r[q] = x[q];
      live[q] = x[q] >= 0;  // out-of-range slots were loaded as -1
    }
    int32_t y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      y[q] = live[q] ? __ldcg(P + (uint64_t)(uint32_t)r[q] * R + (j0 + warp + 8u * q)) : -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t j = j0 + warp + 8u * q;
      if (live[q] && y[q] >= 0) {  // parent is not the root: follow the chain
        r[q] = y[q];
        uint32_t it = 1;
        for (; it < cap; ++it) {
          const int32_t z = __ldcg(P + (uint64_t)(uint32_t)r[q] * R + j);
          if (z < 0) break;
          r[q] = z;
        }
        if (it == cap) {
          set_status(status, IM_ETIMEOUT);
          live[q] = false;
        } else if (it > 1) {
          // Full path compression: the chain's inner nodes (non-roots of the
          // same component) get the root too, so later walks through them
          // take one step. Their own slots are written with the same value
          // when their tiles come round, so no update is lost.
          int32_t z = x[q];  // the first parent; the walk stops at the root
          for (uint32_t k = 0; k < it && z != r[q]; ++k) {
            const int32_t nz = __ldcg(P + (uint64_t)(uint32_t)z * R + j);
            if (nz < 0) break;
            __stcg(P + (uint64_t)(uint32_t)z * R + j, r[q]);
            z = nz;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t j = j0 + warp + 8u * q;
      const uint32_t key = live[q] ? (uint32_t)r[q] : 0xffffffffu;
      const unsigned peers = __match_any_sync(kFull, key);
      if (live[q]) {
        if (lane == (uint32_t)(__ffs(peers) - 1))
          atomicAdd(P + (uint64_t)(uint32_t)r[q] * R + j, -(int32_t)__popc(peers));
        if (r[q] != x[q]) __stcg(P + (uint64_t)v * R + j, r[q]);
      }
    }
    __syncthreads();  // the tile is reloaded next iteration
  }
}

cudaError_t launch_compress(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                            cudaStream_t s) {
  const uint64_t ntiles = ((uint64_t)g->n + kCompV - 1) / kCompV * ((q.R + kCompL - 1) / kCompL);
  uint64_t blocks = ntiles;
  const uint64_t cap = (uint64_t)g->num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_compress<<<(unsigned)blocks, 256, 0, s>>>(ws->d_P, (uint32_t)g->n, q.R, ws->d_status,
                                              uf_budget((uint32_t)g->n));
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
