// On-device lazy greedy (CELF) seed selection over the memoized samples
// (Algorithm 7; CELF of Section 2.2): one cooperative launch of 1024-thread
// blocks (one per SM for graphs above 65536 vertices, a quarter of the SMs
// below, where only the bulk refresh needs the grid). Block 0 drives the lazy
// greedy; all blocks join for the grid-wide steps (prefix extraction and bulk
// gain refresh).
//
// Keys pack (gain << 32) | (0xffffffff - v): a larger key means a larger gain
// and, on equal gains, a smaller vertex id, so the key order is exactly the
// greedy tie-break of the oracle. Gains are integers sigma*R, so keys are
// exact and unique.
//
// State:
//   keys[n]    upper bounds of every vertex (initially the NewGreedy-step
//              gains mg_v) in global memory; C, a prefix of at most kCap
//              candidates extracted from it in key order, lives in the
//              driver's shared memory, sorted descending, with current bounds.
//   sig_out    the largest key of any vertex outside C (0 if none).
//   pool       the first B entries of C, evaluated exactly against the current
//              seed set: per lane, the component root and the not yet covered
//              component size, kept in shared memory.
// Round (driver): evaluate the pool (the segmented reduce of marginal gains over
// the R samples in Algorithm 7). While the best pool gain beats every other
// bound (the head of the rest of C and sig_out), commit it and subtract, from every
// other pool member, the lanes it shares a component with -- pool gains stay
// exact, so several seeds can be committed per round. The round's seeds mark
// their components covered in the per-sample bitmap; surviving pool members
// are merged back into C with their exact gains as new bounds (submodularity
// keeps them valid). The committed sequence equals naive greedy with lowest-id
// tie-break: a committed key is exact and exceeds every bound.
// Grid steps:
//   extraction  when the head of C falls below sig_out, C is written back and
//               all blocks find the next prefix (histogram threshold search
//               over the bounds, then compaction).
//   refresh     when many candidates were evaluated without a commit (a large
//               component just got covered, so many bounds are loose), all
//               blocks recompute every exact gain against the current seed set
//               (a full NewGreedy step on the memoized samples) and the prefix
//               is extracted again from these exact keys.
#include "im_celf.cuh"

namespace imgb {

size_t celf_ctl_bytes() { return sizeof(CelfCtl); }

// Above this many vertices the lazy greedy's bulk refresh runs as a launch of
// its own (k_celf_refresh).
constexpr uint32_t kExtRefreshMinN = 1u << 20;
int celf_pool_size(uint32_t R) {
  const size_t per = (size_t)R * 8;
  size_t b = kPoolSmemBudget / per;
  if (b > (size_t)kPoolMax) b = kPoolMax;
  if (b == 0) return 8;  // pool spilled to global memory
  return (int)b;
}
static bool celf_pool_in_smem(uint32_t R) { return (size_t)R * 8 <= kPoolSmemBudget; }

template <bool POOL_SMEM>
__global__ void __launch_bounds__(kCelfThreads, 1) k_celf(CelfArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ CelfSmem s;
  extern __shared__ uint32_t dyn[];
  const int tid = threadIdx.x;
  const bool driver = blockIdx.x == 0;
  // Helpers: the other blocks of the driver's cluster (none when the launch
  // has no cluster shape, or clusters of one block; the driver then evaluates
  // every item itself).
  const bool helper = !driver && grid.cluster_rank() == 0 && cg::this_cluster().num_blocks() > 1;
  const uint32_t gtid = blockIdx.x * blockDim.x + tid;
  const uint32_t gthreads = gridDim.x * blockDim.x;
  const uint32_t R = a.R;
  uint32_t *proot = POOL_SMEM ? dyn : a.g_pool;
  uint32_t *pcont = proot + (size_t)a.B * R;
  CelfCtl *ctl = a.ctl;
  const bool local_extract = a.n <= kLocalN;
  // A resuming launch runs only after a launch that stopped for an external
  // refresh (the same word in every thread: the previous launch wrote it).
  if (a.resume && __ldcg(&ctl->ext_state) != 1) return;

  Driver d;
  bool bounded = false;
  uint64_t hi = 0;
  uint64_t A0 = a.keyrange[0], B0 = a.keyrange[1];
  uint32_t pass_id = 0, extracts = 0, refreshes = 0;
  int cmd = kCmdExtract;
  uint32_t outer = 0;
  if (!a.resume) {
    for (uint32_t i = gtid; i < 3 * kBins; i += gthreads) (&ctl->hist[0][0])[i] = 0u;
    for (uint32_t i = gtid; i < a.n; i += gthreads) a.chosen[i] = 0;
    if (gtid == 0) {
      ctl->kmin = ~0ull;
      ctl->kmax = 0ull;
      ctl->kcount = 0u;
      ctl->nC = 0u;
      ctl->sig_out = 0ull;
      ctl->cmd = 0;
      ctl->ext_state = 0;
    }
  } else {  // the state left by the stopped launch; the keys are refreshed
    d.nsel = __ldcg(&ctl->s_nsel);
    d.sigma = __ldcg(&ctl->s_sigma);
    d.rounds = __ldcg(&ctl->s_rounds);
    d.evals = __ldcg(&ctl->s_evals);
    d.lb = __ldcg(&ctl->s_lb);
    for (int i = 0; i < 4; ++i) d.cyc[i] = __ldcg(&ctl->s_cyc[i]);
    for (int i = 0; i < 2; ++i) d.fine[i] = __ldcg(&ctl->s_fine[i]);
    outer = __ldcg(&ctl->s_outer);
    extracts = __ldcg(&ctl->s_extracts);
    refreshes = __ldcg(&ctl->s_refreshes) + 1;
    pass_id = __ldcg(&ctl->s_pass);
    A0 = __ldcg(&ctl->kmin);
    B0 = __ldcg(&ctl->kmax);
  }
  grid.sync();
  if (a.resume && gtid == 0) {  // every thread has read the state
    ctl->ext_state = 0;
    ctl->kmin = ~0ull;
    ctl->kmax = 0ull;
    ctl->kcount = 0u;
  }

  bool stopped = false;
  for (; outer < a.round_cap; ++outer) {
    const long long t0 = clock64();
    if (cmd == kCmdRefresh && a.ext_left > 0) {
      // Stop for the refresh kernel queued behind this launch: the driver's
      // state goes to the control block, the key statistics start empty.
      if (gtid == 0) {
        ctl->s_nsel = d.nsel;
        ctl->s_sigma = d.sigma;
        ctl->s_rounds = d.rounds;
        ctl->s_evals = d.evals;
        ctl->s_lb = d.lb;
        for (int i = 0; i < 4; ++i) ctl->s_cyc[i] = d.cyc[i];
        for (int i = 0; i < 2; ++i) ctl->s_fine[i] = d.fine[i];
        ctl->s_outer = outer;
        ctl->s_extracts = extracts;
        ctl->s_refreshes = refreshes;
        ctl->s_pass = pass_id;
        ctl->kmin = ~0ull;
        ctl->kmax = 0ull;
        ctl->kcount = 0u;
        __threadfence();
        ctl->ext_state = 1;
      }
      stopped = true;
      break;
    }
    if (cmd == kCmdRefresh) {
      grid_refresh(a, __ldcg(&ctl->refresh_lb));
      grid.sync();
      A0 = __ldcg(&ctl->kmin);
      B0 = __ldcg(&ctl->kmax);
      bounded = false;
      hi = 0;
      ++refreshes;
    }
    // ---------------------------------------------------------- extraction
    bool ok = true;
    if (local_extract) {
      if (driver) {
        uint64_t A = A0, B = B0;
        if (bounded) {
          uint64_t mn = ~0ull, mx = 0ull;
          for (uint32_t i = tid; i < a.n; i += blockDim.x) {
            const uint64_t k = __ldcg(a.keys + i);
            if (k == 0 || k >= hi) continue;
            mn = umin64(mn, k);
            mx = umax64(mx, k);
          }
          A = block_reduce_u64(mn, false, s);
          B = block_reduce_u64(mx, true, s);
        }
        if (B == 0 || A > B) {  // no vertex left anywhere: cannot happen with K <= n
          ok = false;
        } else {
          const uint64_t t = block_select(a, bounded, hi, A, B, kTarget, kCap, s);
          uint64_t so = 0;
          d.nC = block_compact(a, bounded, hi, t, s, so);
          d.sig_out = so;
          hi = t;
        }
        if (tid == 0) {  // accumulators of the next grid step
          ctl->kmin = ~0ull;
          ctl->kmax = 0ull;
          ctl->kcount = 0u;
        }
      }
    } else {
      uint64_t A = A0, B = B0;
      if (bounded) {
        grid_key_stats(a, hi);
        grid.sync();
        A = __ldcg(&ctl->kmin);
        B = __ldcg(&ctl->kmax);
      }
      if (B == 0 || A > B) {  // no vertex left anywhere: cannot happen with K <= n
        if (gtid == 0) set_status(a.status, IM_EINTERNAL);
        break;
      }
      const uint64_t t = grid_select(a, grid, bounded, hi, A, B, kTarget, kCap, s, pass_id);
      grid_compact(a, bounded, hi, t);
      grid.sync();
      hi = t;
      if (driver) {
        const uint32_t nC = __ldcg(&ctl->nC);
        d.nC = nC;
        d.sig_out = __ldcg(&ctl->sig_out);
        if (nC <= (uint32_t)kCap)
          for (uint32_t i = tid; i < nC; i += blockDim.x) s.C[i] = __ldcg(&ctl->C[i]);
        __syncthreads();
        if (tid == 0) {  // accumulators for the next extraction
          ctl->nC = 0u;
          ctl->sig_out = 0ull;
          ctl->kmin = ~0ull;
          ctl->kmax = 0ull;
          ctl->kcount = 0u;
        }
      }
    }
    bounded = true;
    ++extracts;
    // ---------------------------------------------------------- rounds (driver)
    if (driver) {
      if (!ok || d.nC > (uint32_t)kCap || d.nC == 0) {
        if (tid == 0) set_status(a.status, IM_EINTERNAL);
        cmd = kCmdFail;
        if (POOL_SMEM) {  // the helpers wait for the driver's first announcement
          if (tid == 0) s.ccmd = kCmdFail;
          cg::this_cluster().sync();
        }
      } else {
        d.head = 0;
        sort_desc(s, d.nC);
        d.cyc[0] += (unsigned long long)(clock64() - t0);
        cmd = drive_rounds<POOL_SMEM, false>(a, s, proot, pcont, d);
        if (cmd == kCmdExtract) {  // write the bounds of C back before the next search
          for (uint32_t i = d.head + tid; i < d.nC; i += blockDim.x) {
            const uint64_t k = s.C[i];
            a.keys[key_vertex(k)] = k;
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        ctl->cmd = cmd;
        ctl->refresh_lb = d.lb;
      }
    } else if (POOL_SMEM && helper) {
      helper_rounds(a, s, dyn);
    }
    grid.sync();
    cmd = __ldcg(&ctl->cmd);
    if (cmd == kCmdDone || cmd == kCmdFail) break;
  }
  if (stopped) return;  // the resuming launch reports the counters
  if (outer >= a.round_cap && gtid == 0) set_status(a.status, IM_ETIMEOUT);
  if (driver && tid == 0 && a.stats) {
    atomicAdd(a.stats + 0, (unsigned long long)d.rounds);
    atomicAdd(a.stats + 1, (unsigned long long)d.evals);
    atomicAdd(a.stats + 2, (unsigned long long)extracts);
    for (int i = 0; i < 4; ++i) atomicAdd(a.stats + 4 + i, d.cyc[i]);
    atomicAdd(a.stats + 8, (unsigned long long)refreshes);
    atomicAdd(a.stats + 9, d.fine[0]);
    atomicAdd(a.stats + 10, d.fine[1]);
  }
}

// The refresh as a streaming launch of its own, between a launch that stopped
// for it and the one that resumes (the same result as grid_refresh): a warp
// takes 32 vertices (one flag and key per lane), and every one whose bound
// reaches the driver's lb is re-evaluated against the current seed set with
// lane j on thread j mod 32, sixteen slots per thread in flight (a whole
// 512-lane row at once; consecutive lanes keep the gathers of a shared root
// in one request). Measured on the 4M-vertex graph, lazy greedy per
// selection: 4.97 ms at sixteen slots and four blocks per SM (64 registers),
// 5.4 ms at eight slots and eight blocks, 5.5 ms at sixteen and six, 8.0 ms
// with 16-byte row loads, 6.9 ms with the refresh inside the cooperative
// launch (one 1024-thread block per SM). Chosen vertices get 0; the key range
// and count of the valid keys go to the control block.
__global__ void __launch_bounds__(256, 4) k_celf_refresh(CelfArgs a) {
  CelfCtl *ctl = a.ctl;
  if (__ldcg(&ctl->ext_state) != 1) return;
  const uint32_t lb = __ldcg(&ctl->refresh_lb);
  const int lane = threadIdx.x & 31;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t R = a.R;
  uint64_t mn = ~0ull, mx = 0ull;
  uint32_t c = 0, evaluated = 0;
  // a warp takes 32 vertices at a time: one flag and one key per lane, then
  // the qualifying vertices one after another, each row read at once
  for (uint32_t base = gwarp * 32; base < a.n; base += nwarps * 32) {
    const uint32_t v0 = base + lane;
    uint64_t key = 0;
    bool eval = false;
    if (v0 < a.n && !__ldcg(a.chosen + v0)) {
      key = __ldcg(a.keys + v0);
      eval = (uint32_t)(key >> 32) >= lb;
    }
    unsigned todo = __ballot_sync(kFull, eval);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t v = base + (uint32_t)src;
      const int32_t *row = a.P + (size_t)v * R;
      uint32_t g = 0;
      auto slot = [&](int32_t x, uint32_t j) {
        const uint32_t root = x < 0 ? v : (uint32_t)x;
        const uint32_t sz = x < 0 ? (uint32_t)(-x) : (uint32_t)(-__ldg(a.P + (size_t)x * R + j));
        const uint32_t bit = root * R + j;
        const uint32_t cw = (x != -1) ? __ldcg(a.cov + (bit >> 5)) : 0u;
        return ((cw >> (bit & 31)) & 1u) ? 0u : sz;
      };
#pragma unroll 16
      for (uint32_t j = lane; j < R; j += 32) g += slot(__ldg(row + j), j);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) g += __shfl_xor_sync(kFull, g, d);
      if (lane == src) key = make_key(g, (int32_t)v);
      ++evaluated;
    }
    if (v0 < a.n) {
      if (eval || key == 0) a.keys[v0] = key;  // chosen vertices get 0
      if (key) {
        mn = umin64(mn, key);
        mx = umax64(mx, key);
        ++c;
      }
    }
  }
  mn = warp_min_u64(mn);
  mx = warp_max_u64(mx);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
  if (lane == 0 && c) {
    atomicMin(&ctl->kmin, (unsigned long long)mn);
    atomicMax(&ctl->kmax, (unsigned long long)mx);
    atomicAdd(&ctl->kcount, c);
  }
  if (lane == 0 && evaluated && a.stats)
    atomicAdd(a.stats + IM_STAT_CELF_REFRESHED, (unsigned long long)evaluated);
}

// One cooperative lazy-greedy launch with arguments a.
static cudaError_t launch_celf_once(const im_graph *g, CelfArgs a, cudaStream_t s) {
  const size_t dyn = a.pool_smem ? (size_t)2 * a.B * a.R * sizeof(uint32_t) : 0;
  const void *fn = a.pool_smem ? (const void *)k_celf<true> : (const void *)k_celf<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPoolSmemBudget);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCelfThreads, dyn);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // With the single-block extraction the other blocks only join the bulk
  // refresh, so a quarter of the SMs suffices and the rest stay free for
  // queries running concurrently on other streams; the grid-wide extraction
  // of larger graphs takes every SM.
  int nblocks = (uint32_t)g->n <= kLocalN ? (g->num_sms + 3) / 4 : g->num_sms;
  if (nblocks > g->num_sms * per_sm) nblocks = g->num_sms * per_sm;
  void *args[] = {&a};
  // Cluster size of the shared-memory pool launch: kEvalCluster, or a test
  // override (-1: a plain cooperative launch with no cluster attribute). The
  // kernel reads the cluster shape it actually received, so every shape
  // evaluates every (candidate, lane) item.
  const int64_t c_ovr = override_value(IM_OVR_CELF_CLUSTER);
  if (!a.pool_smem || c_ovr == -1) {
    dim3 grid(nblocks), block(kCelfThreads);
    return cudaLaunchCooperativeKernel(fn, grid, block, args, dyn, s);
  }
  const int csize = c_ovr > 0 ? (int)c_ovr : kEvalCluster;
  // Shared-memory pool: clusters of csize blocks (the driver's cluster
  // evaluates each round's pool together), as many as can be co-resident.
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)csize;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kCelfThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cfg.gridDim = dim3((unsigned)csize);
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, fn, &cfg);
  if (e != cudaSuccess) return e;
  if (max_clusters < 1) return cudaErrorInvalidConfiguration;
  int nclusters = (nblocks + csize - 1) / csize;
  if (nclusters > max_clusters) nclusters = max_clusters;
  cfg.gridDim = dim3((unsigned)(nclusters * csize));
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_celf(const im_graph *g, const im_workspace *ws, const QueryParams &q, int K,
                        int32_t *d_seeds, uint64_t *d_sigma, cudaStream_t s) {
  if (K <= 0) return cudaSuccess;
  CelfArgs a;
  a.P = ws->d_P;
  a.cov = ws->d_cov;
  a.keys = ws->d_keys;
  a.keyrange = ws->d_keyrange;
  a.chosen = ws->d_chosen;
  a.ctl = reinterpret_cast<CelfCtl *>(ws->d_celf_ctl);
  a.n = (uint32_t)g->n;
  a.R = q.R;
  a.K = K;
  a.B = celf_pool_size(q.R);
  a.pool_smem = celf_pool_in_smem(q.R) ? 1 : 0;
  // Refresh after 8 exact evaluations without a commit (one pool round that
  // committed nothing): the refresh re-evaluates only the vertices whose bound
  // reaches the best exact gain already known, so it is cheap next to a run
  // of pool rounds. Swept over {8, 16, 32, 64, 128, 256, 1024, 4096, 16384}
  // and the earlier max(n/64, 4B) on every workload: 8 was never slower and
  // up to 1.3x faster than 64, which was 1.2-5x faster than the rest (the
  // 4M-vertex graph: 34.6 -> 6.9 ms), with identical seeds throughout.
  uint32_t ra = 8;
  const int64_t ra_ovr = override_value(IM_OVR_CELF_REFRESH_AFTER);
  if (ra_ovr > 0) ra = ra_ovr < (int64_t)UINT32_MAX ? (uint32_t)ra_ovr : UINT32_MAX;
  a.refresh_after = ra;
  a.magic_R = q.R == 1 ? 0u : (uint32_t)(((1ull << 32) + q.R - 1) / q.R);
  // Every round evaluates at least one candidate, fewer than refresh_after
  // evaluations separate two commits or a commit and a refresh, and the
  // round after a refresh commits (its keys are exact); every grid step is
  // followed by at least one round.
  a.round_cap = (uint32_t)(K + 2) * (ra + 8) + 1024;
  const int64_t rc_ovr = override_value(IM_OVR_CELF_ROUND_CAP);
  if (rc_ovr > 0 && (uint64_t)rc_ovr < a.round_cap) a.round_cap = (uint32_t)rc_ovr;
  a.g_pool = ws->d_pool;
  a.out_seeds = d_seeds;
  a.out_sigma = d_sigma;
  a.status = ws->d_status;
  a.stats = ws->d_stats;
  a.resume = 0;
  a.ext_left = 0;
  // Large graphs: the bulk refresh runs as a streaming launch of its own
  // (k_celf_refresh) between a lazy-greedy launch that stops for it and one
  // that resumes; two such pairs are queued (each returns at once unless the
  // launch before it stopped), and any later refresh runs inside the launch.
  int ext = (uint32_t)g->n > kExtRefreshMinN ? 1 : 0;
  const int64_t x_ovr = override_value(IM_OVR_CELF_EXT_REFRESH);
  if (x_ovr == 1) ext = 1;
  if (x_ovr == 2) ext = 0;
  if (!ext) return launch_celf_once(g, a, s);
  constexpr int kExtPairs = 2;
  const void *rfn = (const void *)k_celf_refresh;
  int rper_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper_sm, rfn, 256, 0);
  if (e != cudaSuccess) return e;
  if (rper_sm < 1) rper_sm = 1;
  uint64_t rblocks = ((uint64_t)g->n + 255) / 256;  // a warp per 32 vertices
  if (rblocks > (uint64_t)g->num_sms * rper_sm) rblocks = (uint64_t)g->num_sms * rper_sm;
  a.ext_left = kExtPairs;
  e = launch_celf_once(g, a, s);
  for (int k = 0; k < kExtPairs && e == cudaSuccess; ++k) {
    {
      void *rargs[] = {&a};
      e = cudaLaunchKernel(rfn, dim3((unsigned)rblocks), dim3(256), rargs, 0, s);
    }
    if (e != cudaSuccess) break;
    api_count_launch();
    a.resume = 1;
    a.ext_left = kExtPairs - 1 - k;
    e = launch_celf_once(g, a, s);
    if (e == cudaSuccess) api_count_launch();
  }
  return e;
}

}  // namespace imgb
