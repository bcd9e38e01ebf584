// Component kernels shared by the per-query launches (im_select.cu) and the
// batched launch (im_batch.cu): the fused hash-sample + union step over a
// group of 32 upper edges (Eq. 1-2, Algorithm 5's label merge done as
// union-find) and the size-memo tile (Section 3.3). COH selects coherent (L2)
// loads of data written earlier in the same launch.
#pragma once
#include "im_common.cuh"

namespace imgb {

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

template <bool COH>
static __device__ __forceinline__ uint32_t ld_lane(const uint32_t *p) {
  return COH ? __ldcg(p) : __ldg(p);
}

// One warp, upper edges [base, min(base + 32, end)): each edge's hash picks the
// candidate lanes (its lane bucket, or the run for its threshold code), the
// warp flattens the (edge, candidate lane) pairs with a prefix sum, and every
// live pair hooks the two components in that lane. s_boff: the bucket offsets
// (2^nb + 1 entries, shared memory). OPTS: the sampling options (per-edge
// threshold codes, mixed hash) are in play; the uniform-p path keeps its own
// instantiation.
template <bool MASKED, bool OPTS, bool COH>
static __device__ __forceinline__ void union_group(const UnionArgs &a, const uint32_t *s_boff,
                                            int64_t base, int64_t end) {
  const int lane = threadIdx.x & 31;
  const int64_t e = base + lane;
  const bool valid = e < end;
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
        live = lane_live_opt(ld_lane<COH>(a.Xs + j), s_h, a.T32, a.all_live, a.weighted, s_code,
                             a.mix);
      } else {
        live = lane_live(ld_lane<COH>(a.Xs + j), s_h, a.T32, a.all_live);
      }
      if (live) uf_unite(s_u, s_v, j, a.R, a.P, a.status, a.cap);
    }
  }
}

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

// Barrier of the 256 threads that work on one tile: the whole block (BAR 0),
// or named barrier BAR for thread group BAR - 1 of a larger block.
template <int BAR>
static __device__ __forceinline__ void group_sync() {
  if (BAR == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, 256;" ::"r"(BAR) : "memory");
}

// Tile t (32 vertices x 32 lanes) of the size memo, by 256 threads (tid in
// [0, 256), warp = tid / 32); tile: 32 x 33 ints of shared memory.
template <int BAR>
static __device__ __forceinline__ void compress_tile(int32_t *P, uint32_t n, uint32_t R, int32_t *status,
                                              uint32_t cap, uint64_t t,
                                              int32_t (*tile)[kCompL + 1], uint32_t tid) {
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const uint64_t tl = (R + kCompL - 1) / kCompL;
  const bool vec = (R & 3u) == 0;  // rows start 16-byte aligned
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
  group_sync<BAR>();
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
  group_sync<BAR>();  // the tile is reloaded next iteration
}

}  // namespace imgb
