// Kernels of the FusedSampling variant (Section 4, Table 4: fused hash
// sampling without memoization or batched simulations): one simulation at a
// time, a single-lane label array P1[n] is reset, hooked by the component
// kernel on that one lane, compressed, and its component sizes are added to
// the first-seed gains mg_v (Algorithm 1's NewGreedy step, simulation by
// simulation). The other kernels of the variant are the library's own
// union, size-memo and spread kernels run on a one-lane view.
#include "im_common.cuh"

namespace imgb {

__global__ void k_fs_init(int32_t *P1, uint32_t n) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    P1[v] = -1;
}

// mg[v] += |component of v| of this simulation: after the size pass a root
// slot holds -(size) and every other slot its root.
__global__ void k_fs_accum(const int32_t *P1, uint32_t n, unsigned long long *mg) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t x = P1[v];
    const int32_t sz = x < 0 ? -x : -P1[x];
    mg[v] += (unsigned long long)(uint32_t)sz;
  }
}

static unsigned fs_blocks(const im_graph *g) {
  uint64_t b = ((uint64_t)g->n + 255) / 256;
  const uint64_t cap = (uint64_t)g->num_sms * 8;
  return (unsigned)(b < cap ? (b ? b : 1) : cap);
}

cudaError_t launch_fs_init(const im_graph *g, int32_t *P1, cudaStream_t s) {
  k_fs_init<<<fs_blocks(g), 256, 0, s>>>(P1, (uint32_t)g->n);
  return cudaGetLastError();
}

cudaError_t launch_fs_accum(const im_graph *g, const int32_t *P1, unsigned long long *mg,
                            cudaStream_t s) {
  k_fs_accum<<<fs_blocks(g), 256, 0, s>>>(P1, (uint32_t)g->n, mg);
  return cudaGetLastError();
}

}  // namespace imgb
