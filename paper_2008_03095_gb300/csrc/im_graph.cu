// Device CSR store (Section 3.4): validation of a symmetric CSR and the
// upper-triangle edge list {u < v} consumed by the component kernel.
#include <algorithm>
#include <cmath>
#include <utility>
#include <cstdio>
#include <cstring>
#include <vector>

#include "im_common.cuh"

namespace imgb {

enum : uint32_t {
  kBadXadj = 1u,
  kBadId = 2u,
  kUnsorted = 4u,
  kAsym = 8u,
};

__global__ void k_check_xadj(const int32_t *xadj, int32_t n, int64_t arcs, uint32_t *flags) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = xadj[u], b = xadj[u + 1];
    if (a > b || a < 0 || (int64_t)b > arcs) atomicOr(flags, kBadXadj);
  }
}

// warp per vertex: neighbour ids in range, lists non-decreasing
__global__ void k_check_arcs(const int32_t *xadj, const int32_t *adj, int32_t n,
                             uint32_t *flags) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < n; u += nw) {
    const int32_t beg = xadj[u], end = xadj[u + 1];
    uint32_t f = 0;
    for (int32_t a = beg + lane; a < end; a += 32) {
      const int32_t v = adj[a];
      if (v < 0 || v >= n) f |= kBadId;
      if (a > beg && adj[a - 1] > v) f |= kUnsorted;
    }
    f = __reduce_or_sync(kFull, f);
    if (lane == 0 && f) atomicOr(flags, f);
  }
}

// warp per vertex: every arc (u,v) has its reverse (binary search in v's
// sorted list); count upper neighbours v > u
__global__ void k_check_sym(const int32_t *xadj, const int32_t *adj, int32_t n, uint32_t *flags,
                            int32_t *upcount) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < n; u += nw) {
    const int32_t beg = xadj[u], end = xadj[u + 1];
    uint32_t f = 0, up = 0;
    for (int32_t a = beg + lane; a < end; a += 32) {
      const int32_t v = adj[a];
      if (v > u) ++up;
      if (v == u) continue;
      int32_t lo = xadj[v], hi = xadj[v + 1];
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (adj[mid] < (int32_t)u) lo = mid + 1; else hi = mid;
      }
      if (lo >= xadj[v + 1] || adj[lo] != (int32_t)u) f |= kAsym;
    }
    f = __reduce_or_sync(kFull, f);
    up = __reduce_add_sync(kFull, up);
    if (lane == 0) {
      if (f) atomicOr(flags, f);
      upcount[u] = (int32_t)up;
    }
  }
}

// warp per vertex: the upper neighbours of u are the sorted suffix v > u
// (weighted graphs: the threshold code of each upper arc goes along)
__global__ void k_scatter_upper(const int32_t *xadj, const int32_t *adj, int32_t n,
                                const int32_t *upoff, int32_t *eu, int32_t *ev,
                                const uint32_t *code_arc, uint32_t *code_up) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = gw; u < n; u += nw) {
    const int32_t end = xadj[u + 1];
    int32_t lo = xadj[u], hi = end;
    while (lo < hi) {
      const int32_t mid = (lo + hi) >> 1;
      if (adj[mid] <= (int32_t)u) lo = mid + 1; else hi = mid;
    }
    const int32_t o = upoff[u];
    for (int32_t a = lo + lane; a < end; a += 32) {
      eu[o + (a - lo)] = (int32_t)u;
      ev[o + (a - lo)] = adj[a];
      if (code_up) code_up[o + (a - lo)] = code_arc[a];
    }
  }
}

static int fail(char *err, size_t len, int code, const char *msg) {
  std::snprintf(err, len, "%s", msg);
  return code;
}

#define GB_CUDA(expr, what)                                                          \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cudaGetLastError();                                                            \
      std::snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e_));            \
      rc = (e_ == cudaErrorMemoryAllocation) ? IM_ENOMEM : IM_ECUDA;                 \
      goto done;                                                                     \
    }                                                                                \
  } while (0)

// Threshold code of an edge probability w in [0, 1]: T = floor(w * 2^32) of
// Eq. 2, with the largest 32-bit code standing for an always-live edge.
static uint32_t edge_code(double w) {
  const double t = std::floor(w * 4294967296.0);
  return t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
}

int graph_build_device(im_graph *g, const int32_t *h_xadj, const int32_t *h_adj,
                       const double *h_w, char *err, size_t errlen) {
  int rc = IM_OK;
  const int32_t n = g->n;
  const int64_t arcs = 2 * g->m;
  uint32_t *d_flags = nullptr;
  int32_t *d_up = nullptr;
  uint32_t flags = 0;
  std::vector<int32_t> up, off;
  int64_t m_up = 0;
  const int wblocks = g->num_sms * 8;  // 256-thread blocks, warp per vertex
  GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_xadj), sizeof(int32_t) * (size_t)(n + 1)), "cudaMalloc xadj");
  GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_adj), sizeof(int32_t) * (size_t)(arcs > 0 ? arcs : 1)), "cudaMalloc adj");
  GB_CUDA(dev_malloc(reinterpret_cast<void **>(&d_flags), sizeof(uint32_t)), "cudaMalloc flags");
  GB_CUDA(dev_malloc(reinterpret_cast<void **>(&d_up), sizeof(int32_t) * (size_t)n), "cudaMalloc counts");
  GB_CUDA(cudaMemcpy(g->d_xadj, h_xadj, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice),
          "copy xadj");
  if (arcs > 0)
    GB_CUDA(cudaMemcpy(g->d_adj, h_adj, sizeof(int32_t) * (size_t)arcs, cudaMemcpyHostToDevice),
            "copy adj");
  GB_CUDA(cudaMemset(d_flags, 0, sizeof(uint32_t)), "memset");
  k_check_xadj<<<g->num_sms * 4, 256>>>(g->d_xadj, n, arcs, d_flags);
  GB_CUDA(cudaGetLastError(), "k_check_xadj");
  GB_CUDA(cudaMemcpy(&flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost), "flags");
  if (flags & kBadXadj) {
    rc = fail(err, errlen, IM_EINVAL, "xadj is not non-decreasing within [0, 2m]");
    goto done;
  }
  k_check_arcs<<<wblocks, 256>>>(g->d_xadj, g->d_adj, n, d_flags);
  GB_CUDA(cudaGetLastError(), "k_check_arcs");
  GB_CUDA(cudaMemcpy(&flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost), "flags");
  if (flags & kBadId) {
    rc = fail(err, errlen, IM_EINVAL, "neighbour id out of range [0, n)");
    goto done;
  }
  if (h_w) {  // per-arc threshold codes, in the device's arc order
    std::vector<uint32_t> codes((size_t)arcs);
    for (int64_t a = 0; a < arcs; ++a) codes[(size_t)a] = edge_code(h_w[a]);
    if (flags & kUnsorted) {  // neighbour lists get sorted below: carry the codes along
      std::vector<std::pair<int32_t, uint32_t>> pr;
      for (int32_t u = 0; u < n; ++u) {
        pr.clear();
        for (int32_t a = h_xadj[u]; a < h_xadj[u + 1]; ++a) pr.emplace_back(h_adj[a], codes[a]);
        std::sort(pr.begin(), pr.end());
        for (size_t k = 0; k < pr.size(); ++k) codes[(size_t)h_xadj[u] + k] = pr[k].second;
      }
    }
    GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_code_arc),
                       sizeof(uint32_t) * (size_t)(arcs > 0 ? arcs : 1)), "cudaMalloc codes");
    if (arcs > 0)
      GB_CUDA(cudaMemcpy(g->d_code_arc, codes.data(), sizeof(uint32_t) * (size_t)arcs,
                         cudaMemcpyHostToDevice), "copy codes");
  }
  if (flags & kUnsorted) {  // sort every neighbour list once, on the host
    std::vector<int32_t> sorted(h_adj, h_adj + arcs);
    for (int32_t u = 0; u < n; ++u) std::sort(sorted.begin() + h_xadj[u], sorted.begin() + h_xadj[u + 1]);
    GB_CUDA(cudaMemcpy(g->d_adj, sorted.data(), sizeof(int32_t) * (size_t)arcs,
                       cudaMemcpyHostToDevice), "copy sorted adj");
  }
  k_check_sym<<<wblocks, 256>>>(g->d_xadj, g->d_adj, n, d_flags, d_up);
  GB_CUDA(cudaGetLastError(), "k_check_sym");
  GB_CUDA(cudaMemcpy(&flags, d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost), "flags");
  if (flags & kAsym) {
    rc = fail(err, errlen, IM_EINVAL, "CSR is not symmetric: an arc (u,v) has no reverse arc");
    goto done;
  }
  up.resize(n);
  off.resize(n);
  GB_CUDA(cudaMemcpy(up.data(), d_up, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost),
          "copy counts");
  for (int32_t u = 0; u < n; ++u) {
    off[u] = (int32_t)m_up;
    m_up += up[u];
  }
  g->m_up = m_up;
  if (m_up > 0) {
    GB_CUDA(cudaMemcpy(d_up, off.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice),
            "copy offsets");
    GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_eu), sizeof(int32_t) * (size_t)m_up), "cudaMalloc eu");
    GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_ev), sizeof(int32_t) * (size_t)m_up), "cudaMalloc ev");
    if (h_w)
      GB_CUDA(dev_malloc(reinterpret_cast<void **>(&g->d_code_up), sizeof(uint32_t) * (size_t)m_up),
              "cudaMalloc upper codes");
    k_scatter_upper<<<wblocks, 256>>>(g->d_xadj, g->d_adj, n, d_up, g->d_eu, g->d_ev,
                                      g->d_code_arc, g->d_code_up);
    GB_CUDA(cudaGetLastError(), "k_scatter_upper");
  }
  GB_CUDA(cudaDeviceSynchronize(), "graph build");
done:
  if (d_flags) cudaFree(d_flags);
  if (d_up) cudaFree(d_up);
  return rc;
}

}  // namespace imgb
