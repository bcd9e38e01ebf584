// Internal declarations shared by the CUDA translation units of the library.
// Device helpers (edge hash of Eq. 1, live test of Eq. 2, union-find on the
// vertex-major label table) and the host-side handle structures.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/im.h"

namespace imgb {

constexpr int kMaxR = 65536;
constexpr int kMaxBucketBits = 12;      // at most 4096 lane buckets
constexpr int kSortSmemMax = 16384;     // lanes sorted in shared memory up to this padded count
// Budget of the union-find loops: a find follows distinct vertices of one
// acyclic chain and a hook retry happens only after another root was hooked in
// the same lane, so neither can legitimately exceed n steps.
__host__ __device__ __forceinline__ uint32_t uf_cap(uint32_t n) { return n + 64u; }
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ params
// Per-query sampling parameters (Eq. 2): live iff all_live or (X ^ h) < T32.
struct QueryParams {
  uint32_t R;
  uint32_t seed;
  uint64_t T;        // floor(p * 2^32) in [0, 2^32]
  uint32_t T32;      // T when T < 2^32
  int all_live;      // T == 2^32
  int none_live;     // T == 0
  int nb;            // lane-bucket bits: the top nb bits of X and h must agree for a live lane
  int weighted;      // per-edge threshold codes of the graph replace T (w(u,v) of Eq. 2)
  int mix;           // mixed hash: fmix32(X ^ h) is compared instead of X ^ h
};

// Threshold code of an always-live edge (w >= 1 - 2^-32).
constexpr uint32_t kCodeAll = 0xffffffffu;

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ uint32_t rotl32(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

// Eq. 1: MurmurHash3_x86_32 of the 8-byte key lo || hi (little-endian uint32
// halves, lo = min(u,v), hi = max(u,v)), seed 0: two 4-byte blocks, no tail,
// length 8, final avalanche.
__device__ __forceinline__ uint32_t edge_hash_ordered(uint32_t lo, uint32_t hi) {
  const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
  uint32_t h = 0u, k;
  k = lo * c1;
  k = rotl32(k, 15);
  k *= c2;
  h ^= k;
  h = rotl32(h, 13);
  h = h * 5u + 0xe6546b64u;
  k = hi * c1;
  k = rotl32(k, 15);
  k *= c2;
  h ^= k;
  h = rotl32(h, 13);
  h = h * 5u + 0xe6546b64u;
  h ^= 8u;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint32_t edge_hash(int32_t u, int32_t v) {
  return u < v ? edge_hash_ordered((uint32_t)u, (uint32_t)v)
               : edge_hash_ordered((uint32_t)v, (uint32_t)u);
}

// Eq. 2: sample r keeps arc {u,v} iff (X_r xor h) < T.
__device__ __forceinline__ bool lane_live(uint32_t x, uint32_t h, uint32_t T32, int all_live) {
  return all_live || ((x ^ h) < T32);
}

// Lanes are stored sorted by the top nb bits of X_r; every lane that can be
// live for hash h lies in bucket h >> (32 - nb).
__device__ __forceinline__ uint32_t lane_bucket(uint32_t v, int nb) {
  return nb ? (v >> (32 - nb)) : 0u;
}

// MurmurHash3's avalanche finalizer (fmix32), the mixing step of the
// mixed-hash sampler.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Live test under every sampling option: uniform T (T32 / all_live) or the
// edge's threshold code c (weighted), on X ^ h or, mixed, on fmix32(X ^ h).
__device__ __forceinline__ bool lane_live_opt(uint32_t x, uint32_t h, uint32_t T32, int all_live,
                                              int weighted, uint32_t c, int mix) {
  uint32_t z = x ^ h;
  if (mix) z = fmix32(z);
  if (weighted) return c == kCodeAll || z < c;
  return all_live || z < T32;
}

// Candidate lanes [j0, j1) of an edge with hash h: the lanes are sorted by the
// top nb bits of X (nb = kMaxBucketBits for weighted queries, 0 when mixed).
// Uniform T: the lanes of bucket h >> (32 - nb). Weighted, code c: a live
// lane has X ^ h <= c - 1, so the top clz(c - 1) bits of X equal those of h:
// with at most kMaxBucketBits of them, a contiguous run of buckets.
__device__ __forceinline__ void edge_lanes(uint32_t h, int nb, int weighted, uint32_t c, int mix,
                                           const uint32_t *boff, uint32_t &j0, uint32_t &j1) {
  if (mix || !weighted) {
    const uint32_t b = mix ? 0u : lane_bucket(h, nb);
    j0 = boff[b];
    j1 = boff[b + 1];
    return;
  }
  if (c == 0u) {  // never live
    j0 = j1 = 0u;
    return;
  }
  int eb = (c == kCodeAll) ? 0 : __clz(c - 1u);
  if (eb > nb) eb = nb;
  const int shift = nb - eb;
  const uint32_t lo = (eb ? (h >> (32 - eb)) : 0u) << shift;
  j0 = boff[lo];
  j1 = boff[lo + (1u << shift)];
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
  atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ union-find
// The label table P holds, per vertex v and (internal) lane j at P[v*R + j]:
//   P < 0  : v is a root; during hooking the value is -1, after the size pass
//            it is -(component size) (the size memo of Section 3.3 lives in
//            the root slots; non-root slots of a size table are unused anyway)
//   P >= 0 : parent of v (after the size pass: the root = the component minimum)
// Roots are only ever hooked under a smaller root, so the root of every tree
// is the minimum id in it and the final labels are the canonical min-id labels
// of Algorithm 5, independent of the order in which arcs are processed.

// Root of x in lane j with path halving (every store points x at an
// ancestor, so concurrent finds stay correct). Reads bypass L1 so that hooks
// made by other SMs are seen.
__device__ __forceinline__ int32_t uf_find(int32_t x, uint32_t j, uint32_t R, int32_t *P,
                                           int32_t *status, uint32_t cap) {
  for (uint32_t it = 0; it < cap; ++it) {
    int32_t y = __ldcg(P + (uint32_t)x * R + j);
    if (y < 0) return x;
    int32_t z = __ldcg(P + (uint32_t)y * R + j);
    if (z < 0) return y;
    __stcg(P + (uint32_t)x * R + j, z);
    x = z;
  }
  set_status(status, IM_ETIMEOUT);
  return x;
}

// Merge the components of a and b in lane j: hook the larger root under the
// smaller one with a compare-and-swap on the root slot (-1 = still a root).
__device__ __forceinline__ void uf_unite(int32_t a, int32_t b, uint32_t j, uint32_t R,
                                         int32_t *P, int32_t *status, uint32_t cap) {
  int32_t ra = uf_find(a, j, R, P, status, cap);
  int32_t rb = uf_find(b, j, R, P, status, cap);
  for (uint32_t it = 0; it < cap; ++it) {
    if (ra == rb) return;
    int32_t hi = ra > rb ? ra : rb;
    int32_t lo = ra > rb ? rb : ra;
    int32_t old = atomicCAS(P + (uint32_t)hi * R + j, -1, lo);
    if (old == -1) return;
    ra = uf_find(old, j, R, P, status, cap);
    rb = uf_find(lo, j, R, P, status, cap);
  }
  set_status(status, IM_ETIMEOUT);
}

}  // namespace imgb

// ------------------------------------------------------------------ handles
struct im_graph {
  int32_t n = 0;
  int64_t m = 0;          // undirected edges = arcs / 2
  int device = 0;
  int num_sms = 0;
  int l2_bytes = 0;       // device L2 size
  int32_t *d_xadj = nullptr;
  int32_t *d_adj = nullptr;
  int32_t *d_eu = nullptr;  // upper-triangle edge list, eu[e] < ev[e]
  int32_t *d_ev = nullptr;
  int64_t m_up = 0;
  uint32_t *d_code_up = nullptr;   // weighted graphs: threshold code per upper edge (eu/ev order)
  uint32_t *d_code_arc = nullptr;  // weighted graphs: threshold code per CSR arc (d_adj order)
  std::mutex mu;            // serializes blocking calls on the internal workspace
  im_workspace *ws = nullptr;
};

struct im_workspace {
  const im_graph *g = nullptr;
  int device = 0;
  int32_t R_max = 0;
  // select path
  int32_t *d_P = nullptr;       // n * R_max label/size table
  uint32_t *d_cov = nullptr;    // covered bitmap, n * R_max bits
  uint64_t *d_keys = nullptr;   // n CELF keys (gain << 32 | ~id)
  uint64_t *d_keyrange = nullptr;  // [min, max] of the keys
  uint32_t *d_pool = nullptr;   // CELF pool spill: 2 * kPool * R_max words
  uint8_t *d_chosen = nullptr;  // n flags: vertex already selected
  void *d_celf_ctl = nullptr;   // grid-shared CELF control block
  // lanes
  uint32_t *d_X = nullptr;      // R_max raw X_r
  uint32_t *d_Xs = nullptr;     // R_max X in internal lane order
  uint32_t *d_perm = nullptr;   // internal lane -> simulation index
  uint32_t *d_boff = nullptr;   // 2^kMaxBucketBits + 1 bucket offsets
  uint32_t *d_sortbuf = nullptr;  // lane sort scratch for large R
  // spread path
  uint32_t *d_V = nullptr;                                     // visited, n * W words
  uint32_t *d_F0 = nullptr, *d_F1 = nullptr, *d_F2 = nullptr;  // frontiers, n * W words each
  int32_t *d_L0 = nullptr, *d_L1 = nullptr, *d_L2 = nullptr;   // frontier lists (n)
  uint64_t *d_Q0 = nullptr, *d_Q1 = nullptr, *d_Q2 = nullptr;  // chunk lists (n + 2m/32)
  uint32_t *d_inlist = nullptr;                                // n level stamps
  uint32_t *d_cnt = nullptr;                                   // 2(n + 4) per-level counts
  unsigned long long *d_acc = nullptr;                         // sigma accumulator
  unsigned long long *d_stats = nullptr;                       // IM_NUM_STATS counters
  // status and blocking-call staging
  int32_t *d_status = nullptr;
  int32_t *d_seeds_out = nullptr;  // n
  uint64_t *d_sigma_out = nullptr; // n
  int32_t *d_seeds_in = nullptr;   // seed_in_cap
  int64_t seed_in_cap = 0;
  uint8_t *d_mask = nullptr;       // test-only explicit masks
  size_t mask_cap = 0;
};

namespace imgb {

// ------------------------------------------------------------------ test overrides
// Process-wide values set by im_debug_override (IM_OVR_* keys; 0 keeps the
// library's own choice). Read on the host when a kernel is launched.
int64_t override_value(int key);
// Every device allocation of the library goes through this gate, so that a
// test can make the k-th one fail (IM_OVR_FAIL_ALLOC) as cudaMalloc would.
cudaError_t dev_malloc(void **p, size_t bytes);
// Union-find walk budget of a launch (uf_cap, or a smaller test override).
uint32_t uf_budget(uint32_t n);

// Makes the graph's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// ------------------------------------------------------------------ API internals
// (defined in im_api.cu, used by the other host-side entry points)
int api_error(int code, const char *fmt, ...);           // sets im_last_error, returns code
int api_cuda_error(cudaError_t e, const char *what);     // IM_ENOMEM or IM_ECUDA
cudaStream_t api_stream();                               // the calling thread's stream
void api_count_launch();                                  // one more kernel in im_kernel_launches
// Query parameters of R, p, rng_seed under the IM_SAMPLE_* flags (IM_EINVAL on bad input).
int api_query_params(const im_graph *g, int32_t R, double p, uint32_t seed, uint32_t flags,
                     QueryParams *q);
// Workspaces and the kernel sequences of one query (queued on s, no sync).
int api_ws_create(const im_graph *g, int32_t R_max, im_workspace **out);
void api_ws_destroy(im_workspace *ws);
size_t api_ws_bytes(const im_graph *g, int32_t R_max);  // device bytes of a workspace
// After a query ended with IM_EINTERNAL: its first failed invariant check as
// text (read and cleared on s, which is synchronized).
std::string api_check_text(const im_workspace *ws, cudaStream_t s);
int api_ws_seed_capacity(im_workspace *ws, int64_t count);
int api_enqueue_select(const im_graph *g, const im_workspace *ws, int32_t K, const QueryParams &q,
                       int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s);
int api_enqueue_spread(const im_graph *g, const im_workspace *ws, const int32_t *d_seeds,
                       int32_t ns, const QueryParams &q, uint64_t *d_sigma, cudaStream_t s);

// ------------------------------------------------------------------ launchers
// All launchers queue work on `s` and return the launch error (if any).
cudaError_t launch_prep(const im_workspace *ws, const QueryParams &q, bool init_table,
                        bool zero_cov, cudaStream_t s);
// gate: a device word; the kernel returns at once while it is 0 (null: runs).
cudaError_t launch_union(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                         const uint8_t *d_mask, cudaStream_t s,
                         const unsigned long long *gate = nullptr);
cudaError_t launch_compress(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                            cudaStream_t s, const unsigned long long *gate = nullptr);
cudaError_t launch_gains(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                         cudaStream_t s);
cudaError_t launch_expand(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                          int32_t *d_labels, uint32_t *d_sizes, cudaStream_t s);
cudaError_t launch_gather_lanes(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                                const uint32_t *d_lanes, uint32_t nl, int32_t *d_labels,
                                uint32_t *d_sizes, cudaStream_t s);
cudaError_t launch_edge_hash(const int32_t *d_u, const int32_t *d_v, int64_t count,
                             uint32_t *d_h, cudaStream_t s);
cudaError_t launch_celf(const im_graph *g, const im_workspace *ws, const QueryParams &q, int K,
                        int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s);
// handover: the BFS may hand over (through ws->d_acc[1]): it then initialises
// the label table and the covered bitmap, and launch_union (gated by
// ws->d_acc + 1), launch_spread_mark and launch_spread_count must be queued
// behind it, in that order.
cudaError_t launch_spread(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                          const int32_t *d_seeds, int num_seeds, const uint8_t *d_mask,
                          uint64_t *d_sigma, bool handover, cudaStream_t s);
cudaError_t launch_spread_mark(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                               const int32_t *d_seeds, int num_seeds, cudaStream_t s);
cudaError_t launch_spread_count(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                                uint64_t *d_sigma, cudaStream_t s);
// FusedSampling variant: single-lane table reset and mg accumulation
cudaError_t launch_fs_init(const im_graph *g, int32_t *P1, cudaStream_t s);
cudaError_t launch_fs_accum(const im_graph *g, const int32_t *P1, unsigned long long *mg,
                            cudaStream_t s);
// graph construction (blocking helpers, return IM_* codes)
// h_w: per-arc probabilities (host, 2m) or null; validated by the caller.
int graph_build_device(im_graph *g, const int32_t *h_xadj, const int32_t *h_adj,
                       const double *h_w, char *err, size_t errlen);

// shared-memory need of the CELF kernel for a given R (pool in smem or spilled)
int celf_pool_size(uint32_t R);
size_t celf_ctl_bytes();
size_t lane_sort_smem(uint32_t R);

}  // namespace imgb
