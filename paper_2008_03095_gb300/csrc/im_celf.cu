// On-device lazy greedy (CELF) seed selection over the memoized samples
// (Algorithm 7 lines 3-18; CELF of Section 2.2), one persistent 1024-thread
// block per query.
//
// Keys pack (gain << 32) | (0xffffffff - v): a larger key means a larger gain
// and, on equal gains, a smaller vertex id, so the key order is exactly the
// greedy tie-break of the oracle. Gains are integers sigma*R, so keys are
// exact and unique.
//
// State:
//   keys[n]    initial upper bounds (the NewGreedy-step gains mg_v) in global
//              memory; C, a prefix of at most kCap candidates extracted from it
//              in key order, lives in shared memory with its current bounds.
//   sig_out    the largest key of any vertex outside C (0 if none).
//   pool       up to B candidates evaluated exactly against the current seed
//              set: per lane, the component root and the (not yet covered)
//              component size, kept in shared memory.
// Round: take the top-B keys of C into the pool and evaluate them (the
// segmented reduce of Algorithm 7 lines 14-16). While the best pool gain beats
// every other bound (C's largest and sig_out), commit it (lines 11-12): mark
// its components covered in the per-sample bitmap and subtract, from every
// other pool member, the lanes it shares a component with -- so pool gains stay
// exact and several seeds can be committed per round. Remaining pool members
// return to C with their exact gains as new bounds (submodularity keeps them
// valid). If everything in C falls below sig_out, C is written back and the
// next prefix is extracted. The committed sequence equals naive greedy with
// lowest-id tie-break: a committed key is exact and exceeds every bound, and
// bounds dominate true gains.
#include "im_common.cuh"

namespace imgb {

constexpr int kCelfThreads = 1024;
constexpr int kCelfWarps = kCelfThreads / 32;
constexpr int kCap = 4096;     // candidate prefix capacity
constexpr int kTarget = 2048;  // prefix size aimed for per extraction
constexpr int kPoolMax = 32;
constexpr size_t kPoolSmemBudget = 160 * 1024;
constexpr uint32_t kRoundCap = 1u << 22;

int celf_pool_size(uint32_t R) {
  const size_t per = (size_t)R * 8;
  size_t b = kPoolSmemBudget / per;
  if (b > (size_t)kPoolMax) b = kPoolMax;
  if (b == 0) return 8;  // pool spilled to global memory
  return (int)b;
}

static bool celf_pool_in_smem(uint32_t R) { return (size_t)R * 8 <= kPoolSmemBudget; }

struct CelfArgs {
  const int32_t *P;
  uint32_t *cov;
  uint64_t *keys;
  const uint64_t *keyrange;
  uint32_t n, R;
  int K;
  int B;
  int pool_smem;
  uint32_t *g_pool;
  int32_t *out_seeds;
  uint64_t *out_sigma;
  int32_t *status;
};

struct CelfSmem {
  uint64_t C[kCap];
  uint64_t bmin[256];
  uint64_t bmax[256];
  uint32_t hist[256];
  uint64_t red[kCelfWarps];
  uint32_t redc[kCelfWarps];
  int32_t pid[kPoolMax];
  int32_t pslot[kPoolMax];
  uint32_t pgain[kPoolMax];
  int32_t pactive[kPoolMax];
  uint32_t nC;
  uint32_t npool;
  uint64_t sel_t, sel_A, sel_B;
  uint32_t sel_above;
  int sel_done;
  uint64_t best_key;
  int best_w;
};

__device__ __forceinline__ uint64_t make_key(uint32_t gain, int32_t v) {
  return ((uint64_t)gain << 32) | (uint64_t)(0xffffffffu - (uint32_t)v);
}
__device__ __forceinline__ int32_t key_vertex(uint64_t k) {
  return (int32_t)(0xffffffffu - (uint32_t)k);
}

__device__ uint64_t block_max_u64(uint64_t v, CelfSmem &s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    uint64_t o = __shfl_xor_sync(kFull, v, d);
    v = o > v ? o : v;
  }
  if (lane == 0) s.red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = s.red[lane];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      uint64_t o = __shfl_xor_sync(kFull, v, d);
      v = o > v ? o : v;
    }
    if (lane == 0) s.red[0] = v;
  }
  __syncthreads();
  v = s.red[0];
  __syncthreads();
  return v;
}

__device__ uint64_t block_min_u64(uint64_t v, CelfSmem &s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    uint64_t o = __shfl_xor_sync(kFull, v, d);
    v = o < v ? o : v;
  }
  if (lane == 0) s.red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = s.red[lane];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      uint64_t o = __shfl_xor_sync(kFull, v, d);
      v = o < v ? o : v;
    }
    if (lane == 0) s.red[0] = v;
  }
  __syncthreads();
  v = s.red[0];
  __syncthreads();
  return v;
}

__device__ uint32_t block_sum_u32(uint32_t v, CelfSmem &s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  if (lane == 0) s.redc[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = s.redc[lane];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    if (lane == 0) s.redc[0] = v;
  }
  __syncthreads();
  v = s.redc[0];
  __syncthreads();
  return v;
}

// Radix-style threshold search. Valid keys: nonzero and (if bounded) < hi.
// A, B, nvalid: minimum, maximum and count of the valid keys. Returns t such
// that the valid keys >= t number between min(target, nvalid) and cap. Each
// pass histograms the 8 bits below the highest bit in which the current range
// [A, B] differs, then either stops at the bucket where the count crosses the
// target or narrows the range to that bucket.
__device__ uint64_t select_threshold(const uint64_t *keys, uint32_t cnt, bool bounded,
                                     uint64_t hi, uint64_t A, uint64_t B, uint32_t nvalid,
                                     uint32_t target, uint32_t cap, CelfSmem &s,
                                     int32_t *status) {
  if (nvalid <= cap) return A;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t above = 0;
  for (int pass = 0; pass < 66; ++pass) {
    if (A == B) return A;
    const int hb = 63 - __clzll((long long)(A ^ B));
    const int shift = hb >= 7 ? hb - 7 : 0;
    const uint64_t base = A >> shift;
    for (int i = tid; i < 256; i += blockDim.x) {
      s.hist[i] = 0;
      s.bmin[i] = ~0ull;
      s.bmax[i] = 0ull;
    }
    __syncthreads();
    for (uint32_t i = tid; i < cnt; i += blockDim.x) {
      const uint64_t k = keys[i];
      if (k == 0 || (bounded && k >= hi) || k < A || k > B) continue;
      const uint32_t d = (uint32_t)((k >> shift) - base);
      atomicAdd(&s.hist[d], 1u);
      atomicMin((unsigned long long *)&s.bmin[d], (unsigned long long)k);
      atomicMax((unsigned long long *)&s.bmax[d], (unsigned long long)k);
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t c8[8];
      uint32_t lsum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c8[i] = s.hist[255 - 8 * lane - i];
        lsum += c8[i];
      }
      uint32_t incl = lsum;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
      }
      const uint32_t excl = incl - lsum;
      const unsigned ball = __ballot_sync(kFull, above + incl >= target);
      const int L = ball ? __ffs(ball) - 1 : -1;
      if (L < 0 && lane == 0) {  // cannot happen: the range holds >= target keys
        s.sel_done = 1;
        s.sel_t = A;
        set_status(status, IM_EINTERNAL);
      }
      if (lane == L) {
        uint32_t cum = above + excl;
        int d = 255 - 8 * lane;
        for (int i = 0; i < 8; ++i) {
          d = 255 - 8 * lane - i;
          if (cum + c8[i] >= target) break;
          cum += c8[i];
        }
        if (cum + s.hist[d] <= cap) {
          s.sel_done = 1;
          s.sel_t = s.bmin[d];
        } else {
          s.sel_done = 0;
          s.sel_A = s.bmin[d];
          s.sel_B = s.bmax[d];
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
  set_status(status, IM_EINTERNAL);
  return A;
}

__global__ void __launch_bounds__(kCelfThreads, 1) k_celf(CelfArgs a) {
  __shared__ CelfSmem s;
  extern __shared__ uint32_t dyn[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t R = a.R;
  const int B = a.B;
  uint32_t *proot = a.pool_smem ? dyn : a.g_pool;
  uint32_t *pcont = proot + (size_t)B * R;

  int nsel = 0;
  uint64_t sigma = 0;  // meaningful in thread 0
  bool bounded = false;
  uint64_t hi = 0;
  uint64_t sig_out = 0;
  bool need_extract = true;
  if (tid == 0) s.nC = 0;
  __syncthreads();

  for (uint32_t round = 0; nsel < a.K; ++round) {
    if (round >= kRoundCap) {
      if (tid == 0) set_status(a.status, IM_ETIMEOUT);
      break;
    }
    // ---------------------------------------------------------- extraction
    if (need_extract) {
      const uint32_t nC = s.nC;
      for (uint32_t i = tid; i < nC; i += blockDim.x) {
        const uint64_t k = s.C[i];
        if (k) a.keys[key_vertex(k)] = k;
      }
      __syncthreads();
      uint64_t A, Bk;
      uint32_t nvalid;
      if (!bounded) {
        A = a.keyrange[0];
        Bk = a.keyrange[1];
        nvalid = a.n;
      } else {
        uint64_t mn = ~0ull, mx = 0ull;
        uint32_t c = 0;
        for (uint32_t i = tid; i < a.n; i += blockDim.x) {
          const uint64_t k = a.keys[i];
          if (k == 0 || k >= hi) continue;
          mn = k < mn ? k : mn;
          mx = k > mx ? k : mx;
          ++c;
        }
        A = block_min_u64(mn, s);
        Bk = block_max_u64(mx, s);
        nvalid = block_sum_u32(c, s);
      }
      if (nvalid == 0) {  // no vertex left anywhere: cannot happen with K <= n
        if (tid == 0) set_status(a.status, IM_EINTERNAL);
        break;
      }
      const uint64_t t = select_threshold(a.keys, a.n, bounded, hi, A, Bk, nvalid, kTarget,
                                          kCap, s, a.status);
      if (tid == 0) s.nC = 0;
      __syncthreads();
      uint64_t below = 0;
      for (uint32_t i = tid; i < a.n; i += blockDim.x) {
        const uint64_t k = a.keys[i];
        if (k == 0 || (bounded && k >= hi)) continue;
        if (k >= t) {
          const uint32_t pos = atomicAdd(&s.nC, 1u);
          if (pos < (uint32_t)kCap) s.C[pos] = k;
        } else if (k > below) {
          below = k;
        }
      }
      sig_out = block_max_u64(below, s);  // includes a barrier
      if (s.nC > (uint32_t)kCap) {
        if (tid == 0) set_status(a.status, IM_EINTERNAL);
        break;
      }
      bounded = true;
      hi = t;
      need_extract = false;
    }

    // ---------------------------------------------------------- pool = top-B of C
    const uint32_t nC = s.nC;
    uint64_t mn = ~0ull, mx = 0ull;
    uint32_t c = 0;
    for (uint32_t i = tid; i < nC; i += blockDim.x) {
      const uint64_t k = s.C[i];
      if (!k) continue;
      mn = k < mn ? k : mn;
      mx = k > mx ? k : mx;
      ++c;
    }
    const uint64_t cA = block_min_u64(mn, s);
    const uint64_t cB = block_max_u64(mx, s);
    const uint32_t cvalid = block_sum_u32(c, s);
    uint64_t kc = 0;
    if (tid == 0) s.npool = 0;
    __syncthreads();
    if (cvalid > 0) {
      const uint64_t tB =
          select_threshold(s.C, nC, false, 0, cA, cB, cvalid, (uint32_t)B, (uint32_t)B, s, a.status);
      uint64_t below = 0;
      for (uint32_t i = tid; i < nC; i += blockDim.x) {
        const uint64_t k = s.C[i];
        if (!k) continue;
        if (k >= tB) {
          const uint32_t p = atomicAdd(&s.npool, 1u);
          if (p < (uint32_t)B) {
            s.pid[p] = key_vertex(k);
            s.pslot[p] = (int32_t)i;
            s.pactive[p] = 1;
            s.C[i] = 0;
          }
        } else if (k > below) {
          below = k;
        }
      }
      kc = block_max_u64(below, s);
    }
    const uint32_t npool = s.npool < (uint32_t)B ? s.npool : (uint32_t)B;
    const uint64_t top_out = kc > sig_out ? kc : sig_out;

    // ---------------------------------------------------------- exact gains
    // g(u | S) = sum_r [component of u in r not covered] * |C_r(u)|
    if ((uint32_t)warp < npool) {
      const int32_t u = s.pid[warp];
      uint32_t *rr = proot + (size_t)warp * R;
      uint32_t *cc = pcont + (size_t)warp * R;
      const int32_t *row = a.P + (size_t)u * R;
      for (uint32_t j = lane; j < R; j += 32) rr[j] = (uint32_t)__ldg(row + j);
      uint32_t g = 0;
      for (uint32_t j = lane; j < R; j += 32) {
        const int32_t x = (int32_t)rr[j];
        uint32_t root, sz;
        bool maybe_cov;
        if (x < 0) {
          root = (uint32_t)u;
          sz = (uint32_t)(-x);
          maybe_cov = x != -1;  // a singleton {u} is covered only if u is a seed
        } else {
          root = (uint32_t)x;
          sz = (uint32_t)(-__ldg(a.P + (size_t)x * R + j));
          maybe_cov = true;
        }
        uint32_t cv = sz;
        if (maybe_cov) {
          const uint32_t bit = root * R + j;
          if ((__ldcg(a.cov + (bit >> 5)) >> (bit & 31)) & 1u) cv = 0;
        }
        rr[j] = root;
        cc[j] = cv;
        g += cv;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) g += __shfl_xor_sync(kFull, g, d);
      if (lane == 0) s.pgain[warp] = g;
    }
    __syncthreads();

    // ---------------------------------------------------------- commits
    uint64_t bk = 0;
    for (;;) {
      if (warp == 0) {
        uint64_t k = 0;
        if ((uint32_t)lane < npool && s.pactive[lane]) k = make_key(s.pgain[lane], s.pid[lane]);
        uint64_t best = k;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          uint64_t o = __shfl_xor_sync(kFull, best, d);
          best = o > best ? o : best;
        }
        const unsigned b = __ballot_sync(kFull, k != 0 && k == best);
        if (lane == 0) {
          s.best_key = best;
          s.best_w = b ? __ffs(b) - 1 : -1;
        }
      }
      __syncthreads();
      bk = s.best_key;
      const int bw = s.best_w;
      if (bk == 0 || bk < top_out) break;
      if (tid == 0) {
        sigma += s.pgain[bw];
        a.out_seeds[nsel] = s.pid[bw];
        a.out_sigma[nsel] = sigma;
        s.pactive[bw] = 0;
      }
      ++nsel;
      const uint32_t *rb = proot + (size_t)bw * R;
      const uint32_t *cb = pcont + (size_t)bw * R;
      for (uint32_t j = tid; j < R; j += blockDim.x) {
        if (cb[j]) {
          const uint32_t bit = rb[j] * R + j;
          atomicOr(a.cov + (bit >> 5), 1u << (bit & 31));
        }
      }
      __syncthreads();
      if (nsel >= a.K) break;
      if ((uint32_t)warp < npool && s.pactive[warp]) {
        const uint32_t *rr = proot + (size_t)warp * R;
        uint32_t *cc = pcont + (size_t)warp * R;
        uint32_t d = 0;
        for (uint32_t j = lane; j < R; j += 32) {
          const uint32_t cv = cc[j];
          if (cv && rr[j] == rb[j]) {
            d += cv;
            cc[j] = 0;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
        if (lane == 0) s.pgain[warp] -= d;
      }
      __syncthreads();
    }
    if (nsel >= a.K) break;
    // ---------------------------------------------------------- back to C
    if (warp == 0 && (uint32_t)lane < npool && s.pactive[lane])
      s.C[s.pslot[lane]] = make_key(s.pgain[lane], s.pid[lane]);
    __threadfence();
    __syncthreads();
    if (bk == 0 && kc == 0 && sig_out == 0) {
      if (tid == 0) set_status(a.status, IM_EINTERNAL);
      break;
    }
    need_extract = sig_out > kc;
  }
}

cudaError_t launch_celf(const im_graph *g, const im_workspace *ws, const QueryParams &q, int K,
                        int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  CelfArgs a;
  a.P = ws->d_P;
  a.cov = ws->d_cov;
  a.keys = ws->d_keys;
  a.keyrange = ws->d_keyrange;
  a.n = (uint32_t)g->n;
  a.R = q.R;
  a.K = K;
  a.B = celf_pool_size(q.R);
  a.pool_smem = celf_pool_in_smem(q.R) ? 1 : 0;
  a.g_pool = ws->d_pool;
  a.out_seeds = d_seeds;
  a.out_sigma = d_sigma;
  a.status = ws->d_status;
  const size_t dyn = a.pool_smem ? (size_t)2 * a.B * q.R * sizeof(uint32_t) : 0;
  cudaError_t e = cudaFuncSetAttribute(k_celf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPoolSmemBudget);
  if (e != cudaSuccess) return e;
  k_celf<<<1, kCelfThreads, dyn, s>>>(a);
  return cudaGetLastError();
}

}  // namespace imgb
