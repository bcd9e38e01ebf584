// Lane randoms of a query (Section 3.1: one uniform random value X_r per
// simulation, the first R outputs of MT19937) and the lane order by their
// top bits, shared by the query kernels and the batched launch.
#pragma once
#include "im_common.cuh"

namespace imgb {

// ------------------------------------------------------------------ MT19937
// Matsumoto & Nishimura (1998), 32-bit: n = 624, m = 397, matrix 0x9908b0df,
// tempering (11, 7 0x9d2c5680, 15 0xefc60000, 18), init multiplier 1812433253.
// The state refresh ("twist") is done by one block in four dependency-safe
// phases: entries [0,227) read only old state, [227,454) and [454,623) read
// entries refreshed by the previous phase, and entry 623 reads entry 0.
static __device__ __forceinline__ uint32_t mt_next_word(uint32_t cur, uint32_t nxt, uint32_t far) {
  uint32_t y = (cur & 0x80000000u) | (nxt & 0x7fffffffu);
  return far ^ (y >> 1) ^ ((y & 1u) ? 0x9908b0dfu : 0u);
}

static __device__ void mt_twist(uint32_t *mt) {
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

static __device__ __forceinline__ uint32_t mt_temper(uint32_t y) {
  y ^= y >> 11;
  y ^= (y << 7) & 0x9d2c5680u;
  y ^= (y << 15) & 0xefc60000u;
  y ^= y >> 18;
  return y;
}

// Ascending bitonic sort of npow2 keys (shared or global memory) by one block.
static __device__ void block_bitonic_sort(uint32_t *a, int npow2) {
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

// Lane randoms and lane order of one query, by one block: X_0..X_{R-1} =
// the first R outputs of MT19937(seed) (simulation order), the lanes sorted by
// (top nb bits of X, simulation index) into perm / Xs, and boff[b] = the first
// internal lane of bucket b (2^nb + 1 entries). keys: npow2(R) words of sort
// scratch (shared memory when it fits, else sortbuf). keyrange (optional) is
// reset for the first-gain key range.
static __device__ void draw_lanes(uint32_t seed, uint32_t R, int nb, uint32_t *X, uint32_t *Xs,
                           uint32_t *perm, uint32_t *boff, uint32_t *s_sort, uint32_t *sortbuf,
                           uint64_t *keyrange) {
  __shared__ uint32_t mt[624];
  const int t = threadIdx.x;
  if (t == 0) {  // the seeding recurrence is sequential; keep it in a register
    uint32_t x = seed;
    mt[0] = x;
    for (int i = 1; i < 624; ++i) {
      x = 1812433253u * (x ^ (x >> 30)) + (uint32_t)i;
      mt[i] = x;
    }
  }
  __syncthreads();
  for (uint32_t base = 0; base < R; base += 624) {
    mt_twist(mt);
    for (uint32_t i = t; i < 624 && base + i < R; i += blockDim.x) X[base + i] = mt_temper(mt[i]);
    __syncthreads();
  }
  // Lane order: sort keys (bucket << 16 | r); a stable, deterministic order.
  int npow2 = 1;
  while (npow2 < (int)R) npow2 <<= 1;
  uint32_t *keys = (npow2 <= kSortSmemMax) ? s_sort : sortbuf;
  for (int i = t; i < npow2; i += blockDim.x)
    keys[i] = (i < (int)R) ? ((lane_bucket(X[i], nb) << 16) | (uint32_t)i) : 0xffffffffu;
  __syncthreads();
  if (nb > 0) block_bitonic_sort(keys, npow2);
  for (uint32_t j = t; j < R; j += blockDim.x) {
    const uint32_t r = keys[j] & 0xffffu;
    perm[j] = r;
    Xs[j] = X[r];
  }
  // boff[b] = first internal lane whose bucket is >= b
  const uint32_t nbk = 1u << nb;
  for (uint32_t b = t; b <= nbk; b += blockDim.x) {
    uint32_t lo = 0, hi = R;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if ((keys[mid] >> 16) < b) lo = mid + 1; else hi = mid;
    }
    boff[b] = lo;
  }
  if (t == 0 && keyrange) {
    keyrange[0] = ~0ull;
    keyrange[1] = 0ull;
  }
}

}  // namespace imgb
