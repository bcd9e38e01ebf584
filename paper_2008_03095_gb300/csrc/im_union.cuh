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
  const unsigned long long *gate;  // k_union returns at once while *gate == 0 (null: runs)
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

// The four slots of the size-memo tile at vertices v0.., lanes j0.. (32 x 32)
// that thread tid of a 256-thread group holds: row tid / 8, lanes
// 4 * (tid % 8) .. + 3; slots outside the table read as -1.
static __device__ __forceinline__ void compress_load(const int32_t *P, uint32_t n, uint32_t R,
                                                     uint32_t v0, uint32_t j0, uint32_t tid,
                                                     int32_t (&e)[4]) {
  const uint32_t v = v0 + (tid >> 3);
  const uint32_t j = j0 + (tid & 7u) * 4u;
#pragma unroll
  for (int q = 0; q < 4; ++q) e[q] = -1;
  if (v < n) {
    const int32_t *row = P + (uint64_t)v * R;
    if ((R & 3u) == 0 && j + 3 < R) {  // rows start 16-byte aligned
      const int4 x4 = __ldcg(reinterpret_cast<const int4 *>(row + j));
      e[0] = x4.x; e[1] = x4.y; e[2] = x4.z; e[3] = x4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (j + q < R) e[q] = __ldcg(row + j + q);
    }
  }
}

static __device__ __forceinline__ void compress_stage(const int32_t (&e)[4], uint32_t tid,
                                                      int32_t (*tile)[kCompL + 1]) {
  const uint32_t rr = tid >> 3, c0 = (tid & 7u) * 4u;
#pragma unroll
  for (int q = 0; q < 4; ++q) tile[rr][c0 + q] = e[q];
}

// The roots of four slots x[q] of one thread, at lanes jw + 8q (a parent, or
// negative for a root or a slot outside the table): r[q] = the root and
// live[q] set for every non-negative x[q]. The four chains advance together,
// one load of each per step, so they cost as many dependent loads as the
// longest. A chain longer than cap (longer than any chain of n vertices: a
// corrupt table) records IM_ETIMEOUT and leaves its slot not live.
static __device__ __forceinline__ void walk_roots(const int32_t *P, uint32_t R, int32_t *status,
                                                  uint32_t cap, uint32_t jw, const int32_t (&x)[4],
                                                  int32_t (&r)[4], bool (&live)[4]) {
  bool act[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q] = x[q];
    live[q] = x[q] >= 0;
    act[q] = live[q];
  }
  // r[q] holds a non-root vertex of the chain while act[q]; its slot is read
  // next, and a negative slot marks r[q] as the root
  for (uint32_t it = 0;; ++it) {
    int32_t z[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      z[q] = act[q] ? __ldcg(P + (uint64_t)(uint32_t)r[q] * R + (jw + 8u * q)) : -1;
    bool more = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (act[q] && z[q] >= 0) {
        r[q] = z[q];
        more = true;
      } else {
        act[q] = false;
      }
    }
    if (!more) break;
    if (it + 1 >= cap) {
      set_status(status, IM_ETIMEOUT);
#pragma unroll
      for (int q = 0; q < 4; ++q) live[q] = live[q] && !act[q];
      break;
    }
  }
}

// Root-count accumulators of one warp's four tile lanes, in shared memory
// (written by the warp's lane 0 only): in a giant component every tile of a
// lane adds to the same root slot, and those atomics pile onto one L2 slice.
// Each warp instead keeps, per lane, the count owed to the smallest root it
// has met, and pays it with one atomic when the root changes, when the warp
// moves to other lanes, or at the end (the root slot only decreases, so it
// reads negative throughout).
struct RootAcc {
  uint32_t root[4];  // 0xFFFFFFFF: none
  int32_t cnt[4];
};

static __device__ __forceinline__ void root_acc_clear(RootAcc *acc, uint32_t tid) {
  if ((tid & 31u) == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc->root[q] = 0xffffffffu;
      acc->cnt[q] = 0;
    }
  }
  __syncwarp();
}

// Pays the counts owed at tile lanes j0 + warp + 8q and clears them.
static __device__ __forceinline__ void root_acc_flush(int32_t *P, uint32_t R, uint32_t j0,
                                                      uint32_t tid, RootAcc *acc) {
  const uint32_t warp = (tid >> 5) & 7u;
  __syncwarp();
  if ((tid & 31u) == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (acc->cnt[q]) atomicAdd(P + (uint64_t)acc->root[q] * R + (j0 + warp + 8u * q), -acc->cnt[q]);
      acc->root[q] = 0xffffffffu;
      acc->cnt[q] = 0;
    }
  }
  __syncwarp();
}

// The tile at vertices v0.., lanes j0.., staged in shared memory, by 256
// threads, with the warp's root-count accumulators (acc, for these lanes):
// each non-root slot is pointed at its root and counted, into the
// accumulator when the root is the warp's accumulated one, else with one
// atomic per distinct root of the warp. Warp w takes tile lanes w, w + 8,
// w + 16, w + 24 of the 32 vertices (walk_roots). Where a sample holds a
// large component, its root recurs in nearly every tile of a lane. Ends with
// the group's barrier (the tile may be restaged after it).
template <int BAR>
static __device__ __forceinline__ void compress_walk_acc(int32_t *P, uint32_t R, int32_t *status,
                                                         uint32_t cap, uint32_t v0, uint32_t j0,
                                                         int32_t (*tile)[kCompL + 1], uint32_t tid,
                                                         RootAcc *acc) {
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const uint32_t v = v0 + lane;
  int32_t x[4], r[4];
  bool live[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = tile[lane][warp + 8u * q];
  walk_roots(P, R, status, cap, j0 + warp, x, r, live);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t j = j0 + warp + 8u * q;
    uint32_t ar = acc->root[q];  // read by every lane before lane 0 may write
    const uint32_t m = __reduce_min_sync(kFull, live[q] ? (uint32_t)r[q] : 0xffffffffu);
    if (m < ar) {  // a smaller root: pay the old one, follow the new one
      if (lane == 0) {
        if (acc->cnt[q]) atomicAdd(P + (uint64_t)ar * R + j, -acc->cnt[q]);
        acc->root[q] = m;
        acc->cnt[q] = 0;
      }
      ar = m;
    }
    const bool mine = live[q] && (uint32_t)r[q] == ar;
    const unsigned mm = __ballot_sync(kFull, mine);
    if (lane == 0 && mm) acc->cnt[q] += __popc(mm);
    const uint32_t key = (live[q] && !mine) ? (uint32_t)r[q] : 0xffffffffu;
    const unsigned peers = __match_any_sync(kFull, key);
    if (live[q]) {
      if (!mine && lane == (uint32_t)(__ffs(peers) - 1))
        atomicAdd(P + (uint64_t)(uint32_t)r[q] * R + j, -(int32_t)__popc(peers));
      if (r[q] != x[q]) __stcg(P + (uint64_t)v * R + j, r[q]);
    }
  }
  group_sync<BAR>();  // the tile is restaged next
}

// The accumulator walk on the tile's live slots only: the warp's four items
// (lanes w + 8q of the 32 vertices) usually hold few non-root slots, so the
// warp lists them (a ballot per item), and each thread takes one listed slot
// (passes of 32), walks it to its root, and the slots are counted by one
// match over (root, item): into the warp's accumulators where the root is
// the item's accumulated one, else one atomic per group. Same results as
// compress_walk_acc; ends with the group's barrier.
template <int BAR>
static __device__ __forceinline__ void compress_walk_acc_live(int32_t *P, uint32_t R,
                                                              int32_t *status, uint32_t cap,
                                                              uint32_t v0, uint32_t j0,
                                                              int32_t (*tile)[kCompL + 1],
                                                              uint32_t tid, RootAcc *acc) {
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  unsigned bal[4];
  uint32_t off[5];
  off[0] = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    bal[q] = __ballot_sync(kFull, tile[lane][warp + 8u * q] >= 0);
    off[q + 1] = off[q] + (uint32_t)__popc(bal[q]);
  }
  const uint32_t total = off[4];
  for (uint32_t base = 0; base < total; base += 32) {  // warp-uniform
    const uint32_t k = base + lane;
    const bool live0 = k < total;
    uint32_t q = 0, l = 0;
    int32_t x = -1;
    if (live0) {
      q = k >= off[2] ? (k >= off[3] ? 3u : 2u) : (k >= off[1] ? 1u : 0u);
      const unsigned bq = q == 0 ? bal[0] : q == 1 ? bal[1] : q == 2 ? bal[2] : bal[3];
      const uint32_t oq = q == 0 ? off[0] : q == 1 ? off[1] : q == 2 ? off[2] : off[3];
      l = __fns(bq, 0, (int)(k - oq + 1));  // the (k - oq)-th listed vertex of item q
      x = tile[l][warp + 8u * q];
    }
    const uint32_t j = j0 + warp + 8u * q;
    int32_t r = x;
    bool live = live0;
    for (uint32_t it = 0; live; ++it) {  // r is a non-root vertex of the chain
      const int32_t z = __ldcg(P + (uint64_t)(uint32_t)r * R + j);
      if (z < 0) break;
      r = z;
      if (it + 1 >= cap) {  // longer than any chain of n vertices: a corrupt table
        set_status(status, IM_ETIMEOUT);
        live = false;
      }
    }
    uint32_t ar[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) ar[qq] = acc->root[qq];  // every lane reads before lane 0 writes
    __syncwarp();
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const uint32_t m = __reduce_min_sync(kFull, (live && q == (uint32_t)qq) ? (uint32_t)r : 0xffffffffu);
      if (m < ar[qq]) {  // a smaller root: pay the old one, follow the new one
        if (lane == 0) {
          if (acc->cnt[qq]) atomicAdd(P + (uint64_t)ar[qq] * R + (j0 + warp + 8u * qq), -acc->cnt[qq]);
          acc->root[qq] = m;
          acc->cnt[qq] = 0;
        }
        ar[qq] = m;
      }
    }
    const uint32_t arq = q == 0 ? ar[0] : q == 1 ? ar[1] : q == 2 ? ar[2] : ar[3];
    const bool mine = live && (uint32_t)r == arq;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const unsigned mm = __ballot_sync(kFull, mine && q == (uint32_t)qq);
      if (lane == 0 && mm) acc->cnt[qq] += __popc(mm);
    }
    const unsigned long long key =
        (live && !mine) ? (((unsigned long long)(uint32_t)r << 2) | q) : ~0ull;
    const unsigned peers = __match_any_sync(kFull, key);
    if (live) {
      if (!mine && lane == (uint32_t)(__ffs(peers) - 1))
        atomicAdd(P + (uint64_t)(uint32_t)r * R + j, -(int32_t)__popc(peers));
      if (r != x) __stcg(P + (uint64_t)(v0 + l) * R + j, r);
    }
    __syncwarp();
  }
  group_sync<BAR>();  // the tile is restaged next
}

// The tile at vertices v0.., lanes j0.., by 256 threads, without
// accumulators: a thread's four chains are walked one after another, and a
// chain of two or more links is compressed (its inner vertices get the root
// too, so later walks through them take one step; their own slots are
// written with the same value when their tiles come round, so no update is
// lost). Each distinct root of a warp takes one atomic. Where samples hold
// no large component, chains are short and rarely shared: the walk with the
// least work per slot is the fastest.
template <int BAR>
static __device__ __forceinline__ void compress_walk(int32_t *P, uint32_t R, int32_t *status,
                                                     uint32_t cap, uint32_t v0, uint32_t j0,
                                                     int32_t (*tile)[kCompL + 1], uint32_t tid) {
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const uint32_t v = v0 + lane;
  int32_t x[4], r[4];
  bool live[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    x[q] = tile[lane][warp + 8u * q];
    r[q] = x[q];
    live[q] = x[q] >= 0;  // roots, and slots outside the table, are negative
  }
  // the first parent loads of the four items are issued together
  int32_t y[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    y[q] = live[q] ? __ldcg(P + (uint64_t)(uint32_t)r[q] * R + (j0 + warp + 8u * q)) : -1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t j = j0 + warp + 8u * q;
    if (live[q] && y[q] >= 0) {  // the parent is not the root: follow the chain
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
  group_sync<BAR>();  // the tile is restaged next
}

}  // namespace imgb
