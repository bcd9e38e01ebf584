// Spread of a seed set on the fixed hash samples: sigmaR(S) = sum_r
// |union_{s in S} C_r(s)| (Algorithm 4 evaluated on the samples of Eq. 2).
//
// Bit-parallel multi-source BFS over all R samples at once: every vertex has an
// R-bit visited mask V and a frontier mask F (bit j = internal lane j). One
// level expands every frontier vertex u: for each neighbour v the edge hash
// selects the lane bucket that can be live (the same bucket test as the
// component kernel), the live bits of that bucket are built word by word, and
// v gains F[u] & live & ~V[v] (atomicOr on V[v] decides who won each bit).
// Newly set bits form v's next frontier mask and are counted into sigmaR.
// Levels are separated by grid-wide barriers of one cooperative launch.
#include <cooperative_groups.h>

#include "im_common.cuh"

namespace cg = cooperative_groups;

namespace imgb {

struct SpreadArgs {
  const int32_t *xadj, *adj;
  uint32_t n, R, W;
  const uint32_t *Xs, *boff;
  int nb;
  uint32_t T32;
  int all_live;
  const uint8_t *mask;  // explicit-mask test mode: mask[arc * R + j]
  const int32_t *seeds;
  int num_seeds;
  uint32_t *V, *F0, *F1;
  int32_t *L0, *L1;
  uint32_t *inlist;
  uint32_t *cnt;  // [2] frontier sizes
  unsigned long long *acc;
  uint64_t *out;
  int32_t *status;
};

__global__ void __launch_bounds__(512) k_spread(SpreadArgs a) {
  cg::grid_group grid = cg::this_grid();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const uint64_t gwarp = tid >> 5, nwarps = nthr >> 5;
  const uint32_t W = a.W;
  const uint64_t nW = (uint64_t)a.n * W;

  for (uint64_t i = tid; i < nW; i += nthr) {
    a.V[i] = 0u;
    a.F0[i] = 0u;
    a.F1[i] = 0u;
  }
  for (uint64_t i = tid; i < a.n; i += nthr) a.inlist[i] = 0u;
  if (tid < 2) a.cnt[tid] = 0u;
  if (tid == 0) *a.acc = 0ull;
  grid.sync();

  // sources: deduplicated seed set, all R lanes reached
  for (uint64_t i = tid; i < (uint64_t)a.num_seeds; i += nthr) {
    const int32_t s = a.seeds[i];
    if (s < 0 || (uint32_t)s >= a.n) {
      set_status(a.status, IM_EINVAL);
      continue;
    }
    if (atomicCAS(a.inlist + s, 0u, 1u) == 0u) a.L0[atomicAdd(a.cnt, 1u)] = s;
  }
  grid.sync();
  const uint32_t c0 = __ldcg(a.cnt);
  const uint32_t lastmask = (a.R & 31u) ? ((1u << (a.R & 31u)) - 1u) : 0xffffffffu;
  for (uint64_t i = tid; i < (uint64_t)c0 * W; i += nthr) {
    const uint32_t k = (uint32_t)(i / W), w = (uint32_t)(i % W);
    const uint32_t m = (w == W - 1) ? lastmask : 0xffffffffu;
    const uint64_t o = (uint64_t)a.L0[k] * W + w;
    a.V[o] = m;
    a.F0[o] = m;
  }
  for (uint64_t i = tid; i < c0; i += nthr) a.inlist[a.L0[i]] = 0u;
  unsigned long long local = 0;
  if (tid == 0) local = (unsigned long long)c0 * a.R;
  grid.sync();

  int32_t *Lc = a.L0, *Ln = a.L1;
  uint32_t *Fc = a.F0, *Fn = a.F1;
  int par = 0;
  uint32_t level = 0;
  for (; level <= a.n + 1; ++level) {
    const uint32_t cc = __ldcg(a.cnt + par);
    if (cc == 0) break;
    for (uint64_t i = gwarp; i < cc; i += nwarps) {
      const int32_t u = Lc[i];
      const int32_t beg = a.xadj[u], end = a.xadj[u + 1];
      const uint32_t *fu = Fc + (uint64_t)u * W;
      for (int32_t e = beg + lane; e < end; e += 32) {
        const int32_t v = a.adj[e];
        if (v == u) continue;
        uint32_t j0, j1, h = 0;
        if (a.mask) {
          j0 = 0;
          j1 = a.R;
        } else {
          h = edge_hash(u, v);
          const uint32_t b = lane_bucket(h, a.nb);
          j0 = __ldg(a.boff + b);
          j1 = __ldg(a.boff + b + 1);
        }
        if (j0 >= j1) continue;
        for (uint32_t w = j0 >> 5; w <= (j1 - 1) >> 5; ++w) {
          const uint32_t f = __ldcg(fu + w);
          if (!f) continue;
          const uint32_t lo = j0 > (w << 5) ? j0 : (w << 5);
          const uint32_t hi = j1 < (w << 5) + 32 ? j1 : (w << 5) + 32;
          uint32_t live = 0;
          for (uint32_t j = lo; j < hi; ++j) {
            bool l;
            if (a.mask) l = a.mask[(uint64_t)e * a.R + j] != 0;
            else l = lane_live(__ldg(a.Xs + j), h, a.T32, a.all_live);
            live |= (uint32_t)l << (j & 31);
          }
          uint32_t nb = f & live;
          if (!nb) continue;
          const uint64_t o = (uint64_t)v * W + w;
          nb &= ~__ldcg(a.V + o);
          if (!nb) continue;
          const uint32_t old = atomicOr(a.V + o, nb);
          const uint32_t gained = nb & ~old;
          if (!gained) continue;
          atomicOr(Fn + o, gained);
          local += __popc(gained);
          if (atomicCAS(a.inlist + v, 0u, 1u) == 0u) Ln[atomicAdd(a.cnt + (par ^ 1), 1u)] = v;
        }
      }
    }
    grid.sync();
    const uint32_t cn = __ldcg(a.cnt + (par ^ 1));
    for (uint64_t i = tid; i < (uint64_t)cc * W; i += nthr)
      Fc[(uint64_t)Lc[i / W] * W + (i % W)] = 0u;
    for (uint64_t i = tid; i < cn; i += nthr) a.inlist[Ln[i]] = 0u;
    if (tid == 0) a.cnt[par] = 0u;
    grid.sync();
    int32_t *tl = Lc;
    Lc = Ln;
    Ln = tl;
    uint32_t *tf = Fc;
    Fc = Fn;
    Fn = tf;
    par ^= 1;
  }
  if (level > a.n + 1 && tid == 0) set_status(a.status, IM_ETIMEOUT);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) local += __shfl_xor_sync(kFull, local, d);
  if (lane == 0 && local) atomicAdd(a.acc, local);
  grid.sync();
  if (tid == 0) *a.out = (uint64_t)__ldcg(a.acc);
}

cudaError_t launch_spread(const im_graph *g, const im_workspace *ws, const QueryParams &q,
                          const int32_t *d_seeds, int num_seeds, const uint8_t *d_mask,
                          uint64_t *d_sigma, cudaStream_t s) {
  SpreadArgs a;
  a.xadj = g->d_xadj;
  a.adj = g->d_adj;
  a.n = (uint32_t)g->n;
  a.R = q.R;
  a.W = (q.R + 31) / 32;
  a.Xs = ws->d_Xs;
  a.boff = ws->d_boff;
  a.nb = d_mask ? 0 : q.nb;
  a.T32 = q.T32;
  a.all_live = q.all_live;
  a.mask = d_mask;
  a.seeds = d_seeds;
  a.num_seeds = num_seeds;
  a.V = ws->d_V;
  a.F0 = ws->d_F0;
  a.F1 = ws->d_F1;
  a.L0 = ws->d_L0;
  a.L1 = ws->d_L1;
  a.inlist = ws->d_inlist;
  a.cnt = ws->d_cnt;
  a.acc = ws->d_acc;
  a.out = d_sigma;
  a.status = ws->d_status;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread, 512, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (per_sm > 2) per_sm = 2;
  dim3 grid(g->num_sms * per_sm), block(512);
  void *args[] = {&a};
  return cudaLaunchCooperativeKernel((const void *)k_spread, grid, block, args, 0, s);
}

}  // namespace imgb
