// C ABI of the library (declared in include/im.h): argument validation,
// workspaces, stream handling and the kernel sequence of each query.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <queue>
#include <algorithm>
#include <utility>
#include <string>
#include <vector>

#include "im_common.cuh"

using namespace imgb;

// ------------------------------------------------------------------ static scratch
// Device scratch of im_estimate_spread_noalloc, sized for the IM_NOALLOC_*
// limits: the lane tables of the spread prologue and every buffer of the
// spread kernel, each at a 256-byte-aligned offset (NoallocLayout below).
namespace {
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct NoallocLayout {
  static constexpr size_t kN = IM_NOALLOC_MAX_N;
  static constexpr size_t kR = IM_NOALLOC_MAX_R;
  static constexpr size_t kW = (kR + 31) / 32;                // bitset words per vertex
  static constexpr size_t kQ = kN + IM_NOALLOC_MAX_EDGES / 16 + 1;  // work chunks per level
  static constexpr size_t X = 0;
  static constexpr size_t Xs = X + align256(4 * kR);
  static constexpr size_t perm = Xs + align256(4 * kR);
  static constexpr size_t boff = perm + align256(4 * kR);
  static constexpr size_t sortbuf = boff + align256(4 * ((1u << kMaxBucketBits) + 1));
  static constexpr size_t keyrange = sortbuf + align256(4);
  static constexpr size_t V = keyrange + align256(16);
  static constexpr size_t F0 = V + align256(4 * kN * kW);
  static constexpr size_t F1 = F0 + align256(4 * kN * kW);
  static constexpr size_t F2 = F1 + align256(4 * kN * kW);
  static constexpr size_t L0 = F2 + align256(4 * kN * kW);
  static constexpr size_t L1 = L0 + align256(4 * kN);
  static constexpr size_t L2 = L1 + align256(4 * kN);
  static constexpr size_t Q0 = L2 + align256(4 * kN);
  static constexpr size_t Q1 = Q0 + align256(8 * kQ);
  static constexpr size_t Q2 = Q1 + align256(8 * kQ);
  static constexpr size_t stamp = Q2 + align256(8 * kQ);
  static constexpr size_t cnt = stamp + align256(4 * kN);
  static constexpr size_t acc = cnt + align256(4 * 2 * (kN + 4));
  static constexpr size_t stats = acc + align256(8);
  static constexpr size_t status = stats + align256(8 * IM_NUM_STATS);
  static constexpr size_t seeds = status + align256(4);
  static constexpr size_t sigma = seeds + align256(4 * kN);
  static constexpr size_t bytes = sigma + align256(8);
};
static_assert(NoallocLayout::kR <= (size_t)kSortSmemMax, "lane sort must stay in shared memory");
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NoallocLayout::bytes];

// ------------------------------------------------------------------ test overrides
namespace {
std::atomic<int64_t> g_override[IM_NUM_OVERRIDES];
}  // namespace

namespace imgb {

int64_t override_value(int key) {
  return (key >= 0 && key < IM_NUM_OVERRIDES) ? g_override[key].load() : 0;
}

cudaError_t dev_malloc(void **p, size_t bytes) {
  // IM_OVR_FAIL_ALLOC counts down to the allocation that is made to fail
  int64_t k = g_override[IM_OVR_FAIL_ALLOC].load();
  while (k > 0) {
    if (g_override[IM_OVR_FAIL_ALLOC].compare_exchange_weak(k, k - 1)) {
      if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

uint32_t uf_budget(uint32_t n) {
  const uint32_t cap = uf_cap(n);
  const int64_t o = override_value(IM_OVR_UF_CAP);
  return (o > 0 && (uint64_t)o < cap) ? (uint32_t)o : cap;
}

}  // namespace imgb

namespace {

thread_local std::string t_err;
thread_local cudaStream_t t_stream = nullptr;

// ---- launch accounting and optional per-phase event timing
std::atomic<uint64_t> g_launches{0};
struct ProfRec {
  int phase;
  cudaEvent_t a, b;
};
thread_local bool t_prof_on = false;
thread_local std::vector<ProfRec> t_recs;
thread_local std::vector<cudaEvent_t> t_event_pool;

cudaEvent_t prof_event() {
  if (!t_event_pool.empty()) {
    cudaEvent_t e = t_event_pool.back();
    t_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch one kernel (through `launch`) for `phase`, bracketed by events on
// stream s when profiling is on.
template <class F>
cudaError_t timed(int phase, cudaStream_t s, F launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (t_prof_on) {
    a = prof_event();
    b = prof_event();
    if (a) cudaEventRecord(a, s);
  }
  cudaError_t e = launch();
  if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  if (t_prof_on && a && b) {
    cudaEventRecord(b, s);
    t_recs.push_back({phase, a, b});
  }
  return e;
}

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // clear a non-sticky error
  return fail(e == cudaErrorMemoryAllocation ? IM_ENOMEM : IM_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define API_CUDA(expr, what)                         \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

int make_params(const im_graph *g, int32_t R, double p, uint32_t seed, QueryParams *q) {
  if (R < 1 || R > kMaxR) return fail(IM_EINVAL, "R=%d outside [1, %d]", R, kMaxR);
  if (!(p >= 0.0 && p <= 1.0)) return fail(IM_EINVAL, "p outside [0, 1] or NaN");
  if (g && (uint64_t)g->n * (uint64_t)R >= (1ull << 32))
    return fail(IM_EINVAL, "n*R = %llu must be below 2^32",
                (unsigned long long)((uint64_t)g->n * (uint64_t)R));
  q->R = (uint32_t)R;
  q->seed = seed;
  q->T = (uint64_t)std::floor(p * 4294967296.0);
  q->all_live = q->T == (1ull << 32);
  q->none_live = q->T == 0;
  q->T32 = q->all_live ? 0u : (uint32_t)q->T;
  int nb = 0;
  if (!q->all_live && !q->none_live) {
    const uint64_t t1 = q->T - 1;  // live values are <= T-1 < 2^s
    const int s = t1 ? 64 - __builtin_clzll(t1) : 0;
    nb = 32 - s;
    if (nb > kMaxBucketBits) nb = kMaxBucketBits;
  }
  q->nb = nb;
  q->weighted = 0;
  q->mix = 0;
  return IM_OK;
}

constexpr uint32_t kSampleFlags = IM_SAMPLE_EDGE_WEIGHTS | IM_SAMPLE_MIXED_HASH;

// Parameters under the sampling options (flags: IM_SAMPLE_*). Weighted
// queries ignore p; their lanes are sorted by the top kMaxBucketBits bits of X
// so that every edge code finds its candidate lanes as one run (edge_lanes).
// The mixed hash cannot be bucketed: every lane is a candidate.
int make_params_ex(const im_graph *g, int32_t R, double p, uint32_t seed, uint32_t flags,
                   QueryParams *q) {
  if (flags & ~kSampleFlags) return fail(IM_EINVAL, "unknown sampling flags 0x%x", flags);
  const bool weighted = (flags & IM_SAMPLE_EDGE_WEIGHTS) != 0;
  if (weighted && !(g && g->d_code_arc))
    return fail(IM_EINVAL, "IM_SAMPLE_EDGE_WEIGHTS on a graph created without edge weights");
  int rc = make_params(g, R, weighted ? 0.5 : p, seed, q);
  if (rc != IM_OK) return rc;
  if (weighted) {
    q->weighted = 1;
    q->T = 0;
    q->T32 = 0;
    q->all_live = 0;
    q->none_live = 0;
    q->nb = kMaxBucketBits;
  }
  if (flags & IM_SAMPLE_MIXED_HASH) {
    q->mix = 1;
    q->nb = 0;
  }
  return IM_OK;
}

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  return dev_malloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

void ws_free(im_workspace *ws) {
  void *ptrs[] = {ws->d_P,      ws->d_cov,     ws->d_keys,      ws->d_keyrange, ws->d_pool,
                  ws->d_X,      ws->d_Xs,      ws->d_perm,      ws->d_boff,     ws->d_sortbuf,
                  ws->d_V,      ws->d_F0,      ws->d_F1,        ws->d_F2,       ws->d_L0,
                  ws->d_L1,     ws->d_L2,      ws->d_Q0,        ws->d_Q1,       ws->d_Q2,
                  ws->d_inlist, ws->d_cnt,     ws->d_acc,
                  ws->d_stats,  ws->d_status,  ws->d_seeds_out, ws->d_sigma_out,
                  ws->d_seeds_in, ws->d_mask,  ws->d_chosen,    ws->d_celf_ctl};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

int ws_create(const im_graph *g, int32_t R_max, im_workspace **out) {
  im_workspace *ws = new (std::nothrow) im_workspace();
  if (!ws) return fail(IM_ENOMEM, "host allocation failed");
  ws->g = g;
  ws->device = g->device;
  ws->R_max = R_max;
  const size_t n = (size_t)g->n;
  const size_t nR = n * (size_t)R_max;
  const size_t W = ((size_t)R_max + 31) / 32;
  cudaError_t e = cudaSuccess;
  size_t npow2 = 1;
  while (npow2 < (size_t)R_max) npow2 <<= 1;
#define WS_ALLOC(ptr, cnt)                 \
  if (e == cudaSuccess) e = dalloc(&ws->ptr, (cnt));
  WS_ALLOC(d_P, nR);
  WS_ALLOC(d_cov, (nR + 31) / 32);
  WS_ALLOC(d_keys, n);
  WS_ALLOC(d_keyrange, 2);
  WS_ALLOC(d_chosen, n);
  if (e == cudaSuccess) e = dev_malloc(&ws->d_celf_ctl, celf_ctl_bytes());
  WS_ALLOC(d_pool, (size_t)R_max * 8 > (size_t)160 * 1024 ? (size_t)2 * 8 * R_max : 1);
  WS_ALLOC(d_X, R_max);
  WS_ALLOC(d_Xs, R_max);
  WS_ALLOC(d_perm, R_max);
  WS_ALLOC(d_boff, (1u << kMaxBucketBits) + 1);
  WS_ALLOC(d_sortbuf, npow2 > (size_t)kSortSmemMax ? npow2 : 1);
  WS_ALLOC(d_V, n * W);
  WS_ALLOC(d_F0, n * W);
  WS_ALLOC(d_F1, n * W);
  WS_ALLOC(d_F2, n * W);
  WS_ALLOC(d_L0, n);
  WS_ALLOC(d_L1, n);
  WS_ALLOC(d_L2, n);
  WS_ALLOC(d_Q0, n + (size_t)g->m / 16 + 1);
  WS_ALLOC(d_Q1, n + (size_t)g->m / 16 + 1);
  WS_ALLOC(d_Q2, n + (size_t)g->m / 16 + 1);
  WS_ALLOC(d_inlist, n);
  WS_ALLOC(d_cnt, 2 * (n + 4));
  WS_ALLOC(d_acc, 7);  // spread: sigma, hand-over word, block counter; size-memo probe: 4
  WS_ALLOC(d_stats, IM_NUM_STATS);
  WS_ALLOC(d_status, 1);
  WS_ALLOC(d_seeds_out, n);
  WS_ALLOC(d_sigma_out, n);
#undef WS_ALLOC
  if (e == cudaSuccess) e = cudaMemset(ws->d_status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(ws->d_acc, 0, 7 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(ws->d_stats, 0, sizeof(unsigned long long) * IM_NUM_STATS);
  if (e != cudaSuccess) {
    ws_free(ws);
    delete ws;
    return cuda_fail(e, "workspace allocation");
  }
  *out = ws;
  return IM_OK;
}

int check_ws(const im_graph *g, const im_workspace *ws, int32_t R) {
  if (!g || !ws) return fail(IM_EINVAL, "null graph or workspace");
  if (ws->g != g) return fail(IM_EINVAL, "workspace belongs to another graph");
  if (R > ws->R_max) return fail(IM_EINVAL, "R=%d exceeds the workspace's R_max=%d", R, ws->R_max);
  return IM_OK;
}

// The kernel sequence of one select query (Algorithm 7).
int enqueue_select(const im_graph *g, const im_workspace *ws, int32_t K, const QueryParams &q,
                   const uint8_t *d_mask, int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s,
                   bool stop_after_tables) {
  QueryParams qq = q;
  if (d_mask) {  // explicit live mask: identity lane order, every lane a candidate
    qq.nb = 0;
    qq.none_live = 0;
  }
  API_CUDA(timed(IM_PHASE_PREP, s, [&] { return launch_prep(ws, qq, true, !stop_after_tables, s); }),
           "k_prep");
  if (!qq.none_live && g->m_up > 0) {
    API_CUDA(timed(IM_PHASE_UNION, s, [&] { return launch_union(g, ws, qq, d_mask, s); }),
             "k_union");
    API_CUDA(timed(IM_PHASE_COMPRESS, s, [&] { return launch_compress(g, ws, qq, s); }),
             "k_compress");
  }
  if (stop_after_tables) return IM_OK;
  API_CUDA(timed(IM_PHASE_GAINS, s, [&] { return launch_gains(g, ws, qq, s); }), "k_gains");
  API_CUDA(timed(IM_PHASE_CELF, s,
                 [&] { return launch_celf(g, ws, qq, K, d_seeds, d_sigma, s); }),
           "k_celf");
  return IM_OK;
}

// The spread (Algorithm 4 on the fixed samples): the BFS, and on tables larger
// than L2 the hand-over kernels behind it (they return at once unless the BFS
// handed over; see im_spread.cu).
int enqueue_spread(const im_graph *g, const im_workspace *ws, const int32_t *d_seeds, int32_t ns,
                   const QueryParams &q, const uint8_t *d_mask, uint64_t *d_sigma, cudaStream_t s) {
  QueryParams qq = q;
  if (d_mask) qq.nb = 0;
  // The hand-over pays when the table exceeds L2 and the BFS's cost per
  // vertex (its arcs, rescanned on about five levels at 65 ps per arc scan)
  // beats the components' (R slots at about 5.7 ps each): 112 m > n R.
  const uint64_t nR = (uint64_t)g->n * qq.R;
  const bool handover = ws->d_P && ws->d_cov && !qq.none_live && g->m_up > 0 &&
                        nR * sizeof(int32_t) > (uint64_t)g->l2_bytes &&
                        nR < 112ull * (uint64_t)g->m;
  API_CUDA(timed(IM_PHASE_SPREAD_PREP, s, [&] { return launch_prep(ws, qq, false, false, s); }),
           "k_prep");
  API_CUDA(timed(IM_PHASE_SPREAD, s,
                 [&] { return launch_spread(g, ws, qq, d_seeds, ns, d_mask, d_sigma, handover, s); }),
           "k_spread");
  if (handover) {  // each returns at once unless the BFS handed over
    const unsigned long long *gate = ws->d_acc + 1;
    API_CUDA(timed(IM_PHASE_SPREAD_UNION, s,
                   [&] { return launch_union(g, ws, qq, d_mask, s, gate); }),
             "k_union (spread)");
    API_CUDA(timed(IM_PHASE_SPREAD_MARK, s,
                   [&] { return launch_spread_mark(g, ws, qq, d_seeds, ns, s); }),
             "k_spread_mark");
    API_CUDA(timed(IM_PHASE_SPREAD_CC, s,
                   [&] { return launch_spread_count(g, ws, qq, d_sigma, s); }),
             "k_spread_count");
  }
  return IM_OK;
}

// Status word: read, clear, translate.
int take_status(const im_workspace *ws, cudaStream_t s) {
  int32_t st = 0;
  API_CUDA(cudaMemcpyAsync(&st, ws->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
           "status copy");
  API_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  if (st != 0) {
    API_CUDA(cudaMemsetAsync(ws->d_status, 0, sizeof(int32_t), s), "status clear");
    API_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    if (st == IM_EINTERNAL)
      return fail(st, "device-side invariant violated: %s", api_check_text(ws, s).c_str());
    const char *what = st == IM_ETIMEOUT ? "a device loop exceeded its iteration budget"
                       : st == IM_EINVAL ? "invalid seed id"
                                         : "device-side error";
    return fail(st, "%s", what);
  }
  return IM_OK;
}

// Internal workspace of a graph for blocking calls (grown on demand).
int internal_ws(im_graph *g, int32_t R, im_workspace **out) {
  if (g->ws && g->ws->R_max >= R) {
    *out = g->ws;
    return IM_OK;
  }
  if (g->ws) {
    ws_free(g->ws);
    delete g->ws;
    g->ws = nullptr;
  }
  int rc = ws_create(g, R, &g->ws);
  if (rc != IM_OK) return rc;
  *out = g->ws;
  return IM_OK;
}

int ensure_mask(im_workspace *ws, size_t bytes) {
  if (ws->mask_cap >= bytes) return IM_OK;
  if (ws->d_mask) cudaFree(ws->d_mask);
  ws->d_mask = nullptr;
  ws->mask_cap = 0;
  API_CUDA(dev_malloc(reinterpret_cast<void **>(&ws->d_mask), bytes ? bytes : 1),
           "cudaMalloc mask");
  ws->mask_cap = bytes;
  return IM_OK;
}

int ensure_seed_in(im_workspace *ws, int64_t count) {
  if (ws->seed_in_cap >= count && ws->d_seeds_in) return IM_OK;
  if (ws->d_seeds_in) cudaFree(ws->d_seeds_in);
  ws->d_seeds_in = nullptr;
  ws->seed_in_cap = 0;
  API_CUDA(dalloc(&ws->d_seeds_in, (size_t)(count > 0 ? count : 1)), "cudaMalloc seeds");
  ws->seed_in_cap = count > 0 ? count : 1;
  return IM_OK;
}

// FusedSampling (Section 4, Table 4): MixGreedy with the paper's fused hash
// sampling but none of its batching or memoization. Simulation r runs alone
// on a one-lane view of the workspace (its X_r, one lane bucket): the
// NewGreedy step hooks and compresses a single-lane label array per
// simulation and adds the component sizes into mg; the lazy greedy keeps a
// host priority queue ordered by (gain descending, id ascending) with
// MixGreedy's iteration stamps, and re-evaluates a stale top u by RandCas on
// the fixed samples: the spread of S + {u}, one single-lane BFS launch per
// simulation, minus sigma(S). Gains are exact integers, so the committed
// sequence is the naive greedy one (the same seeds and sigma*R as the default
// path).
int fused_sampling_select(im_graph *g, im_workspace *ws, int32_t K, const QueryParams &q,
                          int32_t *out_seeds, uint64_t *out_sigma, cudaStream_t s) {
  const uint32_t R = q.R;
  const size_t n = (size_t)g->n;
  // the lane randoms X_0..X_{R-1} in simulation order (ws->d_X)
  QueryParams qa = q;
  qa.nb = 0;
  API_CUDA(timed(IM_PHASE_PREP, s, [&] { return launch_prep(ws, qa, false, false, s); }),
           "k_prep");
  unsigned long long *d_mg = nullptr, *d_acc = nullptr;
  uint32_t *d_boff1 = nullptr;
  cudaError_t e = dev_malloc(reinterpret_cast<void **>(&d_mg), sizeof(unsigned long long) * n);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&d_acc), sizeof(uint64_t) * R);
  if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void **>(&d_boff1), 2 * sizeof(uint32_t));
  const uint32_t boff1[2] = {0u, 1u};  // one lane, one bucket
  if (e == cudaSuccess) e = cudaMemsetAsync(d_mg, 0, sizeof(unsigned long long) * n, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_boff1, boff1, sizeof(boff1), cudaMemcpyHostToDevice, s);
  auto release = [&] {
    if (d_mg) cudaFree(d_mg);
    if (d_acc) cudaFree(d_acc);
    if (d_boff1) cudaFree(d_boff1);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "FusedSampling buffers");
  }
  int rc = ensure_seed_in(ws, K + 1);
  if (rc != IM_OK) {
    release();
    return rc;
  }
  QueryParams q1 = q;  // one simulation: R = 1, one bucket
  q1.R = 1;
  q1.nb = 0;
  im_workspace v1 = *ws;  // one-lane view sharing the workspace's buffers
  v1.d_boff = d_boff1;
  v1.d_X = nullptr;
  v1.d_perm = nullptr;
  v1.d_sortbuf = nullptr;
  v1.d_keyrange = nullptr;
  int32_t *P1 = ws->d_P;  // the first n slots of the label table
  // ---- NewGreedy step, one simulation at a time
  for (uint32_t r = 0; r < R && e == cudaSuccess; ++r) {
    v1.d_Xs = ws->d_X + r;
    e = timed(IM_PHASE_PREP, s, [&] { return launch_fs_init(g, P1, s); });
    if (e == cudaSuccess && !q1.none_live && g->m_up > 0) {
      e = timed(IM_PHASE_UNION, s, [&] { return launch_union(g, &v1, q1, nullptr, s); });
      if (e == cudaSuccess)
        e = timed(IM_PHASE_COMPRESS, s, [&] { return launch_compress(g, &v1, q1, s); });
    }
    if (e == cudaSuccess)
      e = timed(IM_PHASE_GAINS, s, [&] { return launch_fs_accum(g, P1, d_mg, s); });
  }
  std::vector<unsigned long long> mg(n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mg.data(), d_mg, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "FusedSampling NewGreedy step");
  }
  rc = take_status(ws, s);
  if (rc != IM_OK) {
    release();
    return rc;
  }
  // ---- lazy greedy (CELF) with RandCas re-evaluations
  using Entry = std::pair<uint64_t, int64_t>;  // (gain, -id): the max is the largest gain, lowest id
  std::priority_queue<Entry> pq;
  std::vector<uint64_t> gain(n);
  std::vector<int32_t> iter(n, 0);
  std::vector<uint8_t> chosen(n, 0);
  for (size_t v = 0; v < n; ++v) {
    gain[v] = mg[v];
    pq.push(Entry(mg[v], -(int64_t)v));
  }
  std::vector<int32_t> S;
  std::vector<uint64_t> acc(R);
  uint64_t sigma = 0;
  while ((int32_t)S.size() < K && !pq.empty()) {
    const Entry top = pq.top();
    pq.pop();
    const int32_t u = (int32_t)(-top.second);
    if (chosen[u] || top.first != gain[u]) continue;  // a superseded entry
    if (iter[u] == (int32_t)S.size()) {
      chosen[u] = 1;
      S.push_back(u);
      sigma += gain[u];
      out_seeds[S.size() - 1] = u;
      out_sigma[S.size() - 1] = sigma;
      continue;
    }
    // RandCas(S + {u}) over the R fixed samples, one simulation per launch
    std::vector<int32_t> Su(S);
    Su.push_back(u);
    e = cudaMemcpyAsync(ws->d_seeds_in, Su.data(), sizeof(int32_t) * Su.size(),
                        cudaMemcpyHostToDevice, s);
    for (uint32_t r = 0; r < R && e == cudaSuccess; ++r) {
      v1.d_Xs = ws->d_X + r;
      e = timed(IM_PHASE_SPREAD, s, [&] {
        return launch_spread(g, &v1, q1, ws->d_seeds_in, (int)Su.size(), nullptr,
                             reinterpret_cast<uint64_t *>(d_acc) + r, false, s);
      });
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(uint64_t) * R, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(e, "FusedSampling RandCas");
    }
    uint64_t tot = 0;
    for (uint32_t r = 0; r < R; ++r) tot += acc[r];
    if (tot < sigma) {
      release();
      return fail(IM_EINTERNAL, "spread of S + {u} below spread of S");
    }
    gain[u] = tot - sigma;
    iter[u] = (int32_t)S.size();
    pq.push(Entry(gain[u], -(int64_t)u));
  }
  release();
  if ((int32_t)S.size() < K) return fail(IM_EINTERNAL, "priority queue ran dry");
  return take_status(ws, s);
}

}  // namespace

namespace imgb {

// The first failed internal invariant check of a query that ended with
// IM_EINTERNAL (work counters IM_STAT_CHECK_CODE/_V0/_V1), read and cleared
// on the query's stream, as text for the error message. Code 0 means that the
// failing step keeps no record (a prefix extraction of the lazy greedy).
std::string api_check_text(const im_workspace *ws, cudaStream_t s) {
  unsigned long long v[3] = {0ull, 0ull, 0ull};
  if (cudaMemcpyAsync(v, ws->d_stats + IM_STAT_CHECK_CODE, sizeof(v), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemsetAsync(ws->d_stats + IM_STAT_CHECK_CODE, 0, sizeof(v), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return "check record unreadable";
  char buf[160];
  if (v[0] == 0)
    std::snprintf(buf, sizeof(buf), "no check record (a prefix extraction step failed)");
  else
    std::snprintf(buf, sizeof(buf), "check %llu failed with 0x%llx, 0x%llx", v[0], v[1], v[2]);
  return buf;
}


int api_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

int api_cuda_error(cudaError_t e, const char *what) { return cuda_fail(e, what); }

cudaStream_t api_stream() { return t_stream; }

void api_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int api_query_params(const im_graph *g, int32_t R, double p, uint32_t seed, uint32_t flags,
                     QueryParams *q) {
  return make_params_ex(g, R, p, seed, flags, q);
}

int api_ws_create(const im_graph *g, int32_t R_max, im_workspace **out) {
  return ws_create(g, R_max, out);
}

void api_ws_destroy(im_workspace *ws) {
  ws_free(ws);
  delete ws;
}

// Mirrors ws_create's allocations (each rounded up to the allocator's 512 B).
size_t api_ws_bytes(const im_graph *g, int32_t R_max) {
  const size_t n = (size_t)g->n, nR = n * (size_t)R_max, W = ((size_t)R_max + 31) / 32;
  size_t npow2 = 1;
  while (npow2 < (size_t)R_max) npow2 <<= 1;
  const size_t q = n + (size_t)g->m / 16 + 1;
  const size_t parts[] = {4 * nR, 4 * ((nR + 31) / 32), 8 * n, 16, n, celf_ctl_bytes(),
                          (size_t)R_max * 8 > (size_t)160 * 1024 ? 4 * 2 * 8 * (size_t)R_max : 4,
                          4 * (size_t)R_max, 4 * (size_t)R_max, 4 * (size_t)R_max,
                          4 * ((1u << kMaxBucketBits) + 1),
                          npow2 > (size_t)kSortSmemMax ? 4 * npow2 : 4, 4 * n * W, 4 * n * W,
                          4 * n * W, 4 * n * W, 4 * n, 4 * n, 4 * n, 8 * q, 8 * q, 8 * q, 4 * n,
                          8 * (n + 4), 8, 8 * IM_NUM_STATS, 4, 4 * n, 8 * n};
  size_t b = 0;
  for (size_t x : parts) b += (x + 511) & ~(size_t)511;
  return b;
}

int api_ws_seed_capacity(im_workspace *ws, int64_t count) { return ensure_seed_in(ws, count); }

int api_enqueue_select(const im_graph *g, const im_workspace *ws, int32_t K, const QueryParams &q,
                       int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s) {
  return enqueue_select(g, ws, K, q, nullptr, d_seeds, d_sigma, s, false);
}

int api_enqueue_spread(const im_graph *g, const im_workspace *ws, const int32_t *d_seeds,
                       int32_t ns, const QueryParams &q, uint64_t *d_sigma, cudaStream_t s) {
  return enqueue_spread(g, ws, d_seeds, ns, q, nullptr, d_sigma, s);
}

}  // namespace imgb

namespace {

// Device address of g_noalloc_scratch per device, looked up once (with that
// device current) by the first im_estimate_spread_noalloc call on it.
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_base[kNoallocMaxDevices] = {};

int noalloc_base(int device, unsigned char **out) {
  if (device < 0 || device >= kNoallocMaxDevices)
    return fail(IM_EINVAL, "device %d outside the no-alloc table", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
    g_noalloc_base[device] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_base[device];
  return IM_OK;
}

// A workspace whose spread buffers all point into the static scratch; only
// the fields the spread prologue and kernel read are set.
im_workspace noalloc_workspace(const im_graph *g, int32_t R, unsigned char *b) {
  using L = NoallocLayout;
  im_workspace ws;
  ws.g = g;
  ws.device = g->device;
  ws.R_max = R;
  ws.d_X = reinterpret_cast<uint32_t *>(b + L::X);
  ws.d_Xs = reinterpret_cast<uint32_t *>(b + L::Xs);
  ws.d_perm = reinterpret_cast<uint32_t *>(b + L::perm);
  ws.d_boff = reinterpret_cast<uint32_t *>(b + L::boff);
  ws.d_sortbuf = reinterpret_cast<uint32_t *>(b + L::sortbuf);
  ws.d_keyrange = reinterpret_cast<uint64_t *>(b + L::keyrange);
  ws.d_V = reinterpret_cast<uint32_t *>(b + L::V);
  ws.d_F0 = reinterpret_cast<uint32_t *>(b + L::F0);
  ws.d_F1 = reinterpret_cast<uint32_t *>(b + L::F1);
  ws.d_F2 = reinterpret_cast<uint32_t *>(b + L::F2);
  ws.d_L0 = reinterpret_cast<int32_t *>(b + L::L0);
  ws.d_L1 = reinterpret_cast<int32_t *>(b + L::L1);
  ws.d_L2 = reinterpret_cast<int32_t *>(b + L::L2);
  ws.d_Q0 = reinterpret_cast<uint64_t *>(b + L::Q0);
  ws.d_Q1 = reinterpret_cast<uint64_t *>(b + L::Q1);
  ws.d_Q2 = reinterpret_cast<uint64_t *>(b + L::Q2);
  ws.d_inlist = reinterpret_cast<uint32_t *>(b + L::stamp);
  ws.d_cnt = reinterpret_cast<uint32_t *>(b + L::cnt);
  ws.d_acc = reinterpret_cast<unsigned long long *>(b + L::acc);
  ws.d_stats = reinterpret_cast<unsigned long long *>(b + L::stats);
  ws.d_status = reinterpret_cast<int32_t *>(b + L::status);
  ws.d_seeds_in = reinterpret_cast<int32_t *>(b + L::seeds);
  ws.seed_in_cap = (int64_t)L::kN;
  ws.d_sigma_out = reinterpret_cast<uint64_t *>(b + L::sigma);
  return ws;
}

}  // namespace

extern "C" {

const char *im_last_error(void) { return t_err.c_str(); }

int im_set_stream(void *cuda_stream) {
  t_stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return IM_OK;
}

int im_profile_enable(int on) {
  for (auto &r : t_recs) {
    t_event_pool.push_back(r.a);
    t_event_pool.push_back(r.b);
  }
  t_recs.clear();
  t_prof_on = on != 0;
  return IM_OK;
}

int im_profile_read(double *total_ms, int64_t *launches) {
  double ms[IM_NUM_PHASES] = {0};
  int64_t cnt[IM_NUM_PHASES] = {0};
  int rc = IM_OK;
  for (auto &r : t_recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && rc == IM_OK) rc = cuda_fail(e, "profile events");
    if (r.phase >= 0 && r.phase < IM_NUM_PHASES) {
      ms[r.phase] += t;
      cnt[r.phase] += 1;
    }
    t_event_pool.push_back(r.a);
    t_event_pool.push_back(r.b);
  }
  t_recs.clear();
  for (int i = 0; i < IM_NUM_PHASES; ++i) {
    if (total_ms) total_ms[i] = ms[i];
    if (launches) launches[i] = cnt[i];
  }
  return rc;
}

uint64_t im_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int im_debug_override(int32_t key, int64_t value) {
  if (key < 0 || key >= IM_NUM_OVERRIDES) return fail(IM_EINVAL, "unknown override key %d", key);
  if (key == IM_OVR_CELF_CLUSTER && !(value == 0 || value == -1 || value == 1 || value == 2 ||
                                      value == 4 || value == 8))
    return fail(IM_EINVAL, "cluster override %lld not in {0, -1, 1, 2, 4, 8}", (long long)value);
  if (key != IM_OVR_CELF_CLUSTER && value < 0)
    return fail(IM_EINVAL, "override %d must be >= 0", key);
  g_override[key].store(value);
  return IM_OK;
}

int im_sampling_threshold(double p, uint64_t *out_T) {
  if (!out_T) return fail(IM_EINVAL, "null output");
  QueryParams q;
  int rc = make_params(nullptr, 1, p, 0, &q);
  if (rc != IM_OK) return rc;
  *out_T = q.T;
  return IM_OK;
}

// Per-arc probabilities: each in [0, 1], and both orientations of an edge
// carry the same multiset of values (duplicate arcs may differ among
// themselves). Self-loops are ignored like their arcs.
static int check_weights(int32_t n, const int32_t *xadj, const int32_t *adj, const double *w) {
  const int64_t arcs = xadj[n];
  std::vector<std::pair<uint64_t, double>> fwd, bwd;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
      if (!(w[a] >= 0.0 && w[a] <= 1.0))
        return fail(IM_EINVAL, "edge weight of arc %lld outside [0, 1] or NaN", (long long)a);
      const int32_t v = adj[a];
      if (v < 0 || v >= n || v == u) continue;
      const uint64_t key = ((uint64_t)(uint32_t)(u < v ? u : v) << 32) | (uint32_t)(u < v ? v : u);
      (u < v ? fwd : bwd).emplace_back(key, w[a]);
    }
  (void)arcs;
  std::sort(fwd.begin(), fwd.end());
  std::sort(bwd.begin(), bwd.end());
  if (fwd != bwd) return fail(IM_EINVAL, "edge weights differ between the two arcs of an edge");
  return IM_OK;
}

static int graph_create_impl(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                             const double *w, im_graph **out);

int im_graph_create(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                    im_graph **out) {
  return graph_create_impl(n, m, xadj, adj, nullptr, out);
}

int im_graph_create_weighted(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                             const double *w, im_graph **out) {
  if (m > 0 && !w) return fail(IM_EINVAL, "null weights");
  return graph_create_impl(n, m, xadj, adj, w ? w : nullptr, out);
}

static int graph_create_impl(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                             const double *w, im_graph **out) {
  if (!out) return fail(IM_EINVAL, "null output handle");
  if (n < 1) return fail(IM_EINVAL, "n=%d must be >= 1", n);
  if (m < 0) return fail(IM_EINVAL, "m must be >= 0");
  if (2 * m >= (1ll << 31)) return fail(IM_EINVAL, "2m must be below 2^31");
  if (!xadj || (m > 0 && !adj)) return fail(IM_EINVAL, "null CSR array");
  if (xadj[0] != 0) return fail(IM_EINVAL, "xadj[0] must be 0");
  if ((int64_t)xadj[n] != 2 * m) return fail(IM_EINVAL, "xadj[n] must equal 2m");
  im_graph *g = new (std::nothrow) im_graph();
  if (!g) return fail(IM_ENOMEM, "host allocation failed");
  g->n = n;
  g->m = m;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->l2_bytes, cudaDevAttrL2CacheSize, g->device);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(e, "device query");
  }
  char err[256] = {0};
  const bool weighted = w != nullptr;
  if (weighted) {
    // the CSR shape is checked before the weights are indexed by it
    for (int32_t u = 0; u < n; ++u)
      if (xadj[u + 1] < xadj[u] || xadj[u] < 0 || (int64_t)xadj[u + 1] > 2 * m) {
        delete g;
        return fail(IM_EINVAL, "xadj is not non-decreasing within [0, 2m]");
      }
    const int wrc = check_weights(n, xadj, adj, w);
    if (wrc != IM_OK) {
      delete g;
      return wrc;
    }
  }
  int rc = graph_build_device(g, xadj, adj, w, err, sizeof(err));
  if (rc != IM_OK) {
    if (g->d_xadj) cudaFree(g->d_xadj);
    if (g->d_adj) cudaFree(g->d_adj);
    if (g->d_eu) cudaFree(g->d_eu);
    if (g->d_ev) cudaFree(g->d_ev);
    if (g->d_code_arc) cudaFree(g->d_code_arc);
    if (g->d_code_up) cudaFree(g->d_code_up);
    delete g;
    return fail(rc, "%s", err);
  }
  *out = g;
  return IM_OK;
}

int im_graph_destroy(im_graph *g) {
  if (!g) return fail(IM_EINVAL, "null graph");
  DeviceGuard dg(g->device);
  if (g->ws) {
    ws_free(g->ws);
    delete g->ws;
  }
  if (g->d_xadj) cudaFree(g->d_xadj);
  if (g->d_adj) cudaFree(g->d_adj);
  if (g->d_eu) cudaFree(g->d_eu);
  if (g->d_ev) cudaFree(g->d_ev);
  if (g->d_code_arc) cudaFree(g->d_code_arc);
  if (g->d_code_up) cudaFree(g->d_code_up);
  delete g;
  return IM_OK;
}

int im_graph_info(const im_graph *g, int32_t *n, int64_t *m) {
  if (!g) return fail(IM_EINVAL, "null graph");
  if (n) *n = g->n;
  if (m) *m = g->m;
  return IM_OK;
}

int im_workspace_create(const im_graph *g, int32_t R_max, im_workspace **out) {
  if (!g || !out) return fail(IM_EINVAL, "null argument");
  QueryParams q;
  int rc = make_params(g, R_max, 0.5, 0, &q);
  if (rc != IM_OK) return rc;
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(IM_ECUDA, "cannot select the graph's device");
  return ws_create(g, R_max, out);
}

int im_workspace_destroy(im_workspace *ws) {
  if (!ws) return fail(IM_EINVAL, "null workspace");
  DeviceGuard dg(ws->device);
  ws_free(ws);
  delete ws;
  return IM_OK;
}

int im_workspace_status(im_workspace *ws) {
  if (!ws) return fail(IM_EINVAL, "null workspace");
  DeviceGuard dg(ws->device);
  return take_status(ws, t_stream);
}

int im_workspace_stats(im_workspace *ws, int64_t *out) {
  if (!ws || !out) return fail(IM_EINVAL, "null argument");
  DeviceGuard dg(ws->device);
  unsigned long long h[IM_NUM_STATS];
  cudaStream_t s = t_stream;
  API_CUDA(cudaMemcpyAsync(h, ws->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s), "stats copy");
  API_CUDA(cudaMemsetAsync(ws->d_stats, 0, sizeof(h), s), "stats clear");
  API_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  for (int i = 0; i < IM_NUM_STATS; ++i) out[i] = (int64_t)h[i];
  return IM_OK;
}

int im_select_seeds_ex_async(const im_graph *g, im_workspace *ws, int32_t K, int32_t R, double p,
                             uint32_t rng_seed, uint32_t flags, int32_t *d_seeds,
                             uint64_t *d_sigma_R) {
  int rc = check_ws(g, ws, R);
  if (rc != IM_OK) return rc;
  if (K < 0 || K > g->n) return fail(IM_EINVAL, "K=%d outside [0, n=%d]", K, g->n);
  if (K > 0 && (!d_seeds || !d_sigma_R)) return fail(IM_EINVAL, "null output");
  if (flags & IM_ALGO_FUSED_SAMPLING)
    return fail(IM_EINVAL, "IM_ALGO_FUSED_SAMPLING is blocking only (im_select_seeds_ex)");
  QueryParams q;
  rc = make_params_ex(g, R, p, rng_seed, flags, &q);
  if (rc != IM_OK) return rc;
  if (K == 0) return IM_OK;
  DeviceGuard dg(g->device);
  return enqueue_select(g, ws, K, q, nullptr, d_seeds, d_sigma_R, t_stream, false);
}

int im_select_seeds_async(const im_graph *g, im_workspace *ws, int32_t K, int32_t R, double p,
                          uint32_t rng_seed, int32_t *d_seeds, uint64_t *d_sigma_R) {
  return im_select_seeds_ex_async(g, ws, K, R, p, rng_seed, 0u, d_seeds, d_sigma_R);
}

int im_estimate_spread_ex_async(const im_graph *g, im_workspace *ws, const int32_t *d_seeds,
                                int32_t num_seeds, int32_t R, double p, uint32_t rng_seed,
                                uint32_t flags, uint64_t *d_sigma_R) {
  int rc = check_ws(g, ws, R);
  if (rc != IM_OK) return rc;
  if (num_seeds < 0) return fail(IM_EINVAL, "num_seeds < 0");
  if (!d_sigma_R || (num_seeds > 0 && !d_seeds)) return fail(IM_EINVAL, "null argument");
  QueryParams q;
  rc = make_params_ex(g, R, p, rng_seed, flags, &q);
  if (rc != IM_OK) return rc;
  DeviceGuard dg(g->device);
  return enqueue_spread(g, ws, d_seeds, num_seeds, q, nullptr, d_sigma_R, t_stream);
}

int im_estimate_spread_async(const im_graph *g, im_workspace *ws, const int32_t *d_seeds,
                             int32_t num_seeds, int32_t R, double p, uint32_t rng_seed,
                             uint64_t *d_sigma_R) {
  return im_estimate_spread_ex_async(g, ws, d_seeds, num_seeds, R, p, rng_seed, 0u, d_sigma_R);
}

int im_select_seeds_ex(const im_graph *g_, int32_t K, int32_t R, double p, uint32_t rng_seed,
                       uint32_t flags, int32_t *out_seeds, uint64_t *out_sigma_R) {
  if (!g_) return fail(IM_EINVAL, "null graph");
  im_graph *g = const_cast<im_graph *>(g_);
  if (K < 0 || K > g->n) return fail(IM_EINVAL, "K=%d outside [0, n=%d]", K, g->n);
  if (K > 0 && (!out_seeds || !out_sigma_R)) return fail(IM_EINVAL, "null output");
  QueryParams q;
  int rc = make_params_ex(g, R, p, rng_seed, flags & ~(uint32_t)IM_ALGO_FUSED_SAMPLING, &q);
  if (rc != IM_OK) return rc;
  if (K == 0) return IM_OK;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  if (flags & IM_ALGO_FUSED_SAMPLING)
    return fused_sampling_select(g, ws, K, q, out_seeds, out_sigma_R, s);
  rc = enqueue_select(g, ws, K, q, nullptr, ws->d_seeds_out, ws->d_sigma_out, s, false);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(out_seeds, ws->d_seeds_out, sizeof(int32_t) * K,
                           cudaMemcpyDeviceToHost, s), "copy seeds");
  API_CUDA(cudaMemcpyAsync(out_sigma_R, ws->d_sigma_out, sizeof(uint64_t) * K,
                           cudaMemcpyDeviceToHost, s), "copy sigma");
  return take_status(ws, s);
}

int im_select_seeds(const im_graph *g, int32_t K, int32_t R, double p, uint32_t rng_seed,
                    int32_t *out_seeds, uint64_t *out_sigma_R) {
  return im_select_seeds_ex(g, K, R, p, rng_seed, 0u, out_seeds, out_sigma_R);
}

int im_estimate_spread_ex(const im_graph *g_, const int32_t *seeds, int32_t num_seeds, int32_t R,
                          double p, uint32_t rng_seed, uint32_t flags, uint64_t *out_sigma_R) {
  if (!g_) return fail(IM_EINVAL, "null graph");
  im_graph *g = const_cast<im_graph *>(g_);
  if (num_seeds < 0) return fail(IM_EINVAL, "num_seeds < 0");
  if (!out_sigma_R || (num_seeds > 0 && !seeds)) return fail(IM_EINVAL, "null argument");
  for (int32_t i = 0; i < num_seeds; ++i)
    if (seeds[i] < 0 || seeds[i] >= g->n) return fail(IM_EINVAL, "seed id %d out of range", seeds[i]);
  QueryParams q;
  int rc = make_params_ex(g, R, p, rng_seed, flags, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  rc = ensure_seed_in(ws, num_seeds);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  if (num_seeds > 0)
    API_CUDA(cudaMemcpyAsync(ws->d_seeds_in, seeds, sizeof(int32_t) * num_seeds,
                             cudaMemcpyHostToDevice, s), "copy seeds");
  rc = enqueue_spread(g, ws, ws->d_seeds_in, num_seeds, q, nullptr, ws->d_sigma_out, s);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(out_sigma_R, ws->d_sigma_out, sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, s), "copy sigma");
  return take_status(ws, s);
}

int im_estimate_spread(const im_graph *g, const int32_t *seeds, int32_t num_seeds, int32_t R,
                       double p, uint32_t rng_seed, uint64_t *out_sigma_R) {
  return im_estimate_spread_ex(g, seeds, num_seeds, R, p, rng_seed, 0u, out_sigma_R);
}

// Same kernels and launches as im_estimate_spread; every device buffer is a
// slice of g_noalloc_scratch, so nothing is allocated or freed here.
int im_estimate_spread_noalloc(const im_graph *g, const int32_t *seeds, int32_t num_seeds,
                               int32_t R, double p, uint32_t rng_seed, uint64_t *out_sigma_R) {
  if (!g) return fail(IM_EINVAL, "null graph");
  if (num_seeds < 0) return fail(IM_EINVAL, "num_seeds < 0");
  if (!out_sigma_R || (num_seeds > 0 && !seeds)) return fail(IM_EINVAL, "null argument");
  if (g->n > IM_NOALLOC_MAX_N)
    return fail(IM_EINVAL, "n=%d exceeds IM_NOALLOC_MAX_N=%d", g->n, IM_NOALLOC_MAX_N);
  if (g->m > IM_NOALLOC_MAX_EDGES)
    return fail(IM_EINVAL, "m=%lld exceeds IM_NOALLOC_MAX_EDGES=%d", (long long)g->m,
                IM_NOALLOC_MAX_EDGES);
  if (R > IM_NOALLOC_MAX_R)
    return fail(IM_EINVAL, "R=%d exceeds IM_NOALLOC_MAX_R=%d", R, IM_NOALLOC_MAX_R);
  if (num_seeds > IM_NOALLOC_MAX_N)
    return fail(IM_EINVAL, "num_seeds=%d exceeds IM_NOALLOC_MAX_N=%d", num_seeds, IM_NOALLOC_MAX_N);
  for (int32_t i = 0; i < num_seeds; ++i)
    if (seeds[i] < 0 || seeds[i] >= g->n) return fail(IM_EINVAL, "seed id %d out of range", seeds[i]);
  QueryParams q;
  int rc = make_params(g, R, p, rng_seed, &q);
  if (rc != IM_OK) return rc;
  DeviceGuard dg(g->device);
  unsigned char *base = nullptr;
  rc = noalloc_base(g->device, &base);
  if (rc != IM_OK) return rc;
  const im_workspace ws = noalloc_workspace(g, R, base);
  cudaStream_t s = t_stream;
  // The status word must start at zero; the spread kernel clears its own
  // frontier, visited and counter buffers.
  API_CUDA(cudaMemsetAsync(ws.d_status, 0, sizeof(int32_t), s), "clear status");
  if (num_seeds > 0)
    API_CUDA(cudaMemcpyAsync(ws.d_seeds_in, seeds, sizeof(int32_t) * num_seeds,
                             cudaMemcpyHostToDevice, s), "copy seeds");
  rc = enqueue_spread(g, &ws, ws.d_seeds_in, num_seeds, q, nullptr, ws.d_sigma_out, s);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(out_sigma_R, ws.d_sigma_out, sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, s), "copy sigma");
  return take_status(&ws, s);
}

// ------------------------------------------------------------------ test hooks

static int debug_tables(const im_graph *g_, int32_t R, double p, uint32_t rng_seed,
                        const uint8_t *h_mask, int32_t *out_labels, uint32_t *out_sizes,
                        uint32_t flags = 0u) {
  if (!g_) return fail(IM_EINVAL, "null graph");
  im_graph *g = const_cast<im_graph *>(g_);
  QueryParams q;
  int rc = make_params_ex(g, R, p, rng_seed, flags, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  const uint8_t *d_mask = nullptr;
  if (h_mask) {
    const size_t bytes = (size_t)2 * g->m * R;
    rc = ensure_mask(ws, bytes);
    if (rc != IM_OK) return rc;
    API_CUDA(cudaMemcpyAsync(ws->d_mask, h_mask, bytes, cudaMemcpyHostToDevice, s), "copy mask");
    d_mask = ws->d_mask;
  }
  rc = enqueue_select(g, ws, 0, q, d_mask, nullptr, nullptr, s, true);
  if (rc != IM_OK) return rc;
  const size_t nR = (size_t)g->n * R;
  int32_t *d_lab = nullptr;
  uint32_t *d_siz = nullptr;
  if (out_labels) API_CUDA(dalloc(&d_lab, nR), "cudaMalloc labels");
  if (out_sizes) {
    cudaError_t e = dalloc(&d_siz, nR);
    if (e != cudaSuccess) {
      if (d_lab) cudaFree(d_lab);
      return cuda_fail(e, "cudaMalloc sizes");
    }
  }
  cudaError_t e = launch_expand(g, ws, q, d_lab, d_siz, s);
  if (e == cudaSuccess && d_lab)
    e = cudaMemcpyAsync(out_labels, d_lab, sizeof(int32_t) * nR, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && d_siz)
    e = cudaMemcpyAsync(out_sizes, d_siz, sizeof(uint32_t) * nR, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_lab) cudaFree(d_lab);
  if (d_siz) cudaFree(d_siz);
  if (e != cudaSuccess) return cuda_fail(e, "debug tables");
  return take_status(ws, s);
}

int im_debug_tables_ex(const im_graph *g, int32_t R, double p, uint32_t rng_seed, uint32_t flags,
                       int32_t *out_labels, uint32_t *out_sizes) {
  if (!out_labels && !out_sizes) return fail(IM_EINVAL, "null outputs");
  return debug_tables(g, R, p, rng_seed, nullptr, out_labels, out_sizes, flags);
}

int im_debug_labels(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                    int32_t *out_labels) {
  if (!out_labels) return fail(IM_EINVAL, "null output");
  return debug_tables(g, R, p, rng_seed, nullptr, out_labels, nullptr);
}

int im_debug_tables_lanes(const im_graph *g_, int32_t R, double p, uint32_t rng_seed,
                          const int32_t *lanes, int32_t num_lanes, int32_t *out_labels,
                          uint32_t *out_sizes) {
  if (!g_) return fail(IM_EINVAL, "null graph");
  if (num_lanes < 1 || !lanes || !out_labels || !out_sizes) return fail(IM_EINVAL, "null argument");
  for (int32_t k = 0; k < num_lanes; ++k)
    if (lanes[k] < 0 || lanes[k] >= R) return fail(IM_EINVAL, "simulation %d outside [0, R)", lanes[k]);
  im_graph *g = const_cast<im_graph *>(g_);
  QueryParams q;
  int rc = make_params(g, R, p, rng_seed, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  rc = enqueue_select(g, ws, 0, q, nullptr, nullptr, nullptr, s, true);
  if (rc != IM_OK) return rc;
  // internal lane of each requested simulation index (perm: lane -> simulation)
  std::vector<uint32_t> perm(R), inv(R), sel(num_lanes);
  API_CUDA(cudaMemcpyAsync(perm.data(), ws->d_perm, sizeof(uint32_t) * R, cudaMemcpyDeviceToHost, s),
           "copy lane order");
  API_CUDA(cudaStreamSynchronize(s), "stream synchronize");
  for (int32_t j = 0; j < R; ++j) inv[perm[j]] = (uint32_t)j;
  for (int32_t k = 0; k < num_lanes; ++k) sel[k] = inv[lanes[k]];
  const size_t cnt = (size_t)g->n * num_lanes;
  uint32_t *d_sel = nullptr;
  int32_t *d_lab = nullptr;
  uint32_t *d_siz = nullptr;
  cudaError_t e = dalloc(&d_sel, (size_t)num_lanes);
  if (e == cudaSuccess) e = dalloc(&d_lab, cnt);
  if (e == cudaSuccess) e = dalloc(&d_siz, cnt);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_sel, sel.data(), sizeof(uint32_t) * num_lanes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_gather_lanes(g, ws, q, d_sel, (uint32_t)num_lanes, d_lab, d_siz, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_labels, d_lab, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_sizes, d_siz, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (d_sel) cudaFree(d_sel);
  if (d_lab) cudaFree(d_lab);
  if (d_siz) cudaFree(d_siz);
  if (e != cudaSuccess) return cuda_fail(e, "debug tables on selected simulations");
  return take_status(ws, s);
}

int im_debug_first_gains(const im_graph *g_, int32_t R, double p, uint32_t rng_seed,
                         uint64_t *out_mg) {
  if (!g_ || !out_mg) return fail(IM_EINVAL, "null argument");
  im_graph *g = const_cast<im_graph *>(g_);
  QueryParams q;
  int rc = make_params(g, R, p, rng_seed, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  rc = enqueue_select(g, ws, 0, q, nullptr, nullptr, nullptr, s, true);
  if (rc != IM_OK) return rc;
  API_CUDA(timed(IM_PHASE_GAINS, s, [&] { return launch_gains(g, ws, q, s); }), "k_gains");
  std::vector<uint64_t> keys((size_t)g->n);
  API_CUDA(cudaMemcpyAsync(keys.data(), ws->d_keys, sizeof(uint64_t) * g->n,
                           cudaMemcpyDeviceToHost, s), "copy keys");
  rc = take_status(ws, s);
  if (rc != IM_OK) return rc;
  for (int32_t v = 0; v < g->n; ++v) out_mg[v] = keys[(size_t)v] >> 32;  // key = mg << 32 | ~v
  return IM_OK;
}

int im_debug_sizes(const im_graph *g, int32_t R, double p, uint32_t rng_seed,
                   uint32_t *out_sizes) {
  if (!out_sizes) return fail(IM_EINVAL, "null output");
  return debug_tables(g, R, p, rng_seed, nullptr, nullptr, out_sizes);
}

int im_debug_lane_randoms(int32_t R, uint32_t rng_seed, uint32_t *out_X) {
  if (!out_X) return fail(IM_EINVAL, "null output");
  QueryParams q;
  int rc = make_params(nullptr, R, 0.5, rng_seed, &q);
  if (rc != IM_OK) return rc;
  im_graph g;
  g.n = 1;
  API_CUDA(cudaGetDevice(&g.device), "device");
  API_CUDA(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, g.device), "attr");
  im_workspace *ws = nullptr;
  rc = ws_create(&g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  cudaError_t e = launch_prep(ws, q, false, false, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_X, ws->d_X, sizeof(uint32_t) * R, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  ws_free(ws);
  delete ws;
  if (e != cudaSuccess) return cuda_fail(e, "lane randoms");
  return IM_OK;
}

int im_debug_edge_hash(const int32_t *u, const int32_t *v, int64_t count, uint32_t *out_h) {
  if (count < 0 || (count > 0 && (!u || !v || !out_h))) return fail(IM_EINVAL, "bad arguments");
  if (count == 0) return IM_OK;
  int32_t *du = nullptr, *dv = nullptr;
  uint32_t *dh = nullptr;
  cudaStream_t s = t_stream;
  cudaError_t e = dalloc(&du, count);
  if (e == cudaSuccess) e = dalloc(&dv, count);
  if (e == cudaSuccess) e = dalloc(&dh, count);
  if (e == cudaSuccess) e = cudaMemcpyAsync(du, u, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v, sizeof(int32_t) * count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_edge_hash(du, dv, count, dh, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_h, dh, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (du) cudaFree(du);
  if (dv) cudaFree(dv);
  if (dh) cudaFree(dh);
  if (e != cudaSuccess) return cuda_fail(e, "edge hash");
  return IM_OK;
}

int im_debug_select_seeds_masked(const im_graph *g_, int32_t K, int32_t R, const uint8_t *mask,
                                 int32_t *out_seeds, uint64_t *out_sigma_R,
                                 int32_t *out_labels, uint32_t *out_sizes) {
  if (!g_ || !mask) return fail(IM_EINVAL, "null argument");
  im_graph *g = const_cast<im_graph *>(g_);
  if (K < 0 || K > g->n) return fail(IM_EINVAL, "K outside [0, n]");
  if (K > 0 && (!out_seeds || !out_sigma_R)) return fail(IM_EINVAL, "null output");
  if (out_labels || out_sizes) {
    int rc = debug_tables(g, R, 0.5, 0, mask, out_labels, out_sizes);
    if (rc != IM_OK) return rc;
  }
  if (K == 0) return IM_OK;
  QueryParams q;
  int rc = make_params(g, R, 0.5, 0, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  const size_t bytes = (size_t)2 * g->m * R;
  rc = ensure_mask(ws, bytes);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(ws->d_mask, mask, bytes, cudaMemcpyHostToDevice, s), "copy mask");
  rc = enqueue_select(g, ws, K, q, ws->d_mask, ws->d_seeds_out, ws->d_sigma_out, s, false);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(out_seeds, ws->d_seeds_out, sizeof(int32_t) * K,
                           cudaMemcpyDeviceToHost, s), "copy seeds");
  API_CUDA(cudaMemcpyAsync(out_sigma_R, ws->d_sigma_out, sizeof(uint64_t) * K,
                           cudaMemcpyDeviceToHost, s), "copy sigma");
  return take_status(ws, s);
}

int im_debug_estimate_spread_masked(const im_graph *g_, const int32_t *seeds, int32_t num_seeds,
                                    int32_t R, const uint8_t *mask, uint64_t *out_sigma_R) {
  if (!g_ || !mask || !out_sigma_R || num_seeds < 0 || (num_seeds > 0 && !seeds))
    return fail(IM_EINVAL, "bad arguments");
  im_graph *g = const_cast<im_graph *>(g_);
  for (int32_t i = 0; i < num_seeds; ++i)
    if (seeds[i] < 0 || seeds[i] >= g->n) return fail(IM_EINVAL, "seed id out of range");
  QueryParams q;
  int rc = make_params(g, R, 0.5, 0, &q);
  if (rc != IM_OK) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  im_workspace *ws = nullptr;
  rc = internal_ws(g, R, &ws);
  if (rc != IM_OK) return rc;
  rc = ensure_seed_in(ws, num_seeds);
  if (rc != IM_OK) return rc;
  cudaStream_t s = t_stream;
  const size_t bytes = (size_t)2 * g->m * R;
  rc = ensure_mask(ws, bytes);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(ws->d_mask, mask, bytes, cudaMemcpyHostToDevice, s), "copy mask");
  if (num_seeds > 0)
    API_CUDA(cudaMemcpyAsync(ws->d_seeds_in, seeds, sizeof(int32_t) * num_seeds,
                             cudaMemcpyHostToDevice, s), "copy seeds");
  rc = enqueue_spread(g, ws, ws->d_seeds_in, num_seeds, q, ws->d_mask, ws->d_sigma_out, s);
  if (rc != IM_OK) return rc;
  API_CUDA(cudaMemcpyAsync(out_sigma_R, ws->d_sigma_out, sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, s), "copy sigma");
  return take_status(ws, s);
}

}  // extern "C"
