// Plain CPU oracle for fused-sampling influence maximization
// (Goktürk & Kaya, "Boosting Parallel Influence-Maximization Kernels for
// Undirected Networks with Fusing and Vectorization", arXiv 2008.03095).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
// this file: only the test suite, the package smoke check and the benchmark's
// CPU-baseline leg use it. It shares no code, header, table or constant
// generator with the CUDA library; it is a slow, literal restatement of the
// method's definitions, single-threaded by default, in the paper's order and
// notation.
//
// What it computes (all integer, exact):
//   * h(u,v): MurmurHash3_x86_32 of the 8-byte key min(u,v) || max(u,v),
//     little-endian uint32 halves, seed 0 (Section 3.1, Eq. 1).
//   * X_r: the first R outputs of std::mt19937(rng_seed) (Section 3.1: one
//     uniform random value per simulation; generator choice is our reading).
//   * T = floor(p * 2^32); arc {u,v} is live in simulation r iff
//     (uint64)(X_r XOR h(u,v)) < T (Section 3.1, Eq. 2 with h_max = 2^32 and
//     the strict unsigned comparison as our reading of the live test).
//   * Component labels: for each simulation, the connected components of the
//     live-edge subgraph, each vertex labelled with the minimum vertex id of
//     its component -- the fixpoint of the label propagation of Algorithm 5.
//     Computed here by breadth-first search from every unvisited vertex in
//     increasing id order, so the BFS root is the component minimum.
//   * Component-size memo: size[l*R + r] = #{v : l_v[r] = l} (Section 3.3).
//   * Seeds: greedy over the R fixed samples (Algorithm 1 restricted to the
//     memoized samples, which Algorithm 7 reaches through CELF): at step k,
//     g(v | S) = sum_r [component of v in r contains no seed] * |C_r(v)|,
//     choose argmax with ties to the lowest vertex id, sigmaR_k = sigmaR_{k-1}
//     + g(s_k | S). The first step is the NewGreedy step of Algorithm 5.
//   * Spread: sigmaR(S) = sum_r |union_{s in S} C_r(s)| by per-simulation BFS
//     from S over live arcs (Algorithm 4 evaluated on the fixed samples).
// A second sampler takes an explicit per-arc, per-simulation live mask instead
// of the hash, so that the worked example of Figures 3-4 and brute-force
// enumerations over all live-edge subsets can be fed in directly.
//
// Built with -fopenmp (oracle/_build/liboracle_omp.so, the all-core CPU
// baseline and the writer of stored expected values for the largest graphs),
// the simulations of the label pass and the vertices of each greedy step are
// split over threads. Nothing else changes: every simulation is still labelled
// by the same BFS, and a greedy step still takes the largest gain with the
// lowest id among equal gains (each thread keeps its own first maximum, and the
// thread maxima are compared in id order), so both builds return identical
// results; only the order of integer additions differs.

#include <algorithm>
#include <cmath>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <cstdint>
#include <cstring>
#include <random>
#include <vector>

namespace {

// ---------------------------------------------------------------- validation
// CSR rules: n >= 1, m >= 0, xadj[0] = 0, xadj non-decreasing, xadj[n] = 2m,
// every neighbour id in [0, n), and every arc (u,v) has a reverse arc (v,u).
bool csr_ok(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj) {
  if (n < 1 || m < 0) return false;
  if (xadj[0] != 0) return false;
  if ((int64_t)xadj[n] != 2 * m) return false;
  for (int32_t u = 0; u < n; ++u)
    if (xadj[u + 1] < xadj[u]) return false;
  for (int64_t a = 0; a < 2 * m; ++a)
    if (adj[a] < 0 || adj[a] >= n) return false;
  // Reverse-arc lookup on a sorted copy of every neighbour list.
  std::vector<int32_t> sorted(adj, adj + 2 * m);
  for (int32_t u = 0; u < n; ++u) std::sort(sorted.begin() + xadj[u], sorted.begin() + xadj[u + 1]);
  for (int32_t u = 0; u < n; ++u) {
    for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
      int32_t v = adj[a];
      if (!std::binary_search(sorted.begin() + xadj[v], sorted.begin() + xadj[v + 1], u))
        return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------- Murmur3
// MurmurHash3_x86_32 as published by Austin Appleby (public domain):
// 4-byte blocks mixed into the state, a 1-3 byte tail, length xor, fmix32.
uint32_t rotl(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

// The avalanche finalizer of MurmurHash3 (fmix32).
uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

uint32_t murmur3_x86_32(const uint8_t *data, int len, uint32_t seed) {
  const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
  uint32_t h = seed;
  int nblocks = len / 4;
  for (int i = 0; i < nblocks; ++i) {
    uint32_t k = (uint32_t)data[4 * i] | ((uint32_t)data[4 * i + 1] << 8) |
                 ((uint32_t)data[4 * i + 2] << 16) | ((uint32_t)data[4 * i + 3] << 24);
    k *= c1;
    k = rotl(k, 15);
    k *= c2;
    h ^= k;
    h = rotl(h, 13);
    h = h * 5 + 0xe6546b64u;
  }
  const uint8_t *tail = data + 4 * nblocks;
  uint32_t k = 0;
  switch (len & 3) {
    case 3: k ^= (uint32_t)tail[2] << 16; [[fallthrough]];
    case 2: k ^= (uint32_t)tail[1] << 8; [[fallthrough]];
    case 1:
      k ^= (uint32_t)tail[0];
      k *= c1;
      k = rotl(k, 15);
      k *= c2;
      h ^= k;
  }
  h ^= (uint32_t)len;
  return fmix32(h);
}

// Eq. 1: h(u,v) = Murmur3(min(u,v) || max(u,v)).
uint32_t edge_hash(int32_t u, int32_t v) {
  uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
  uint8_t key[8];
  for (int i = 0; i < 4; ++i) key[i] = (uint8_t)(a >> (8 * i));
  for (int i = 0; i < 4; ++i) key[4 + i] = (uint8_t)(b >> (8 * i));
  return murmur3_x86_32(key, 8, 0u);
}

// T = floor(p * 2^32): multiplying by a power of two is exact in binary64.
uint64_t threshold(double p) { return (uint64_t)std::floor(p * 4294967296.0); }

// ---------------------------------------------------------------- samplers
// Hash sampler (Eq. 2): live iff (X_r xor h(u,v)) < T.
struct HashSampler {
  std::vector<uint32_t> X;
  uint64_t T;
  HashSampler(int32_t R, double p, uint32_t seed) : X(R), T(threshold(p)) {
    std::mt19937 gen(seed);
    for (int32_t r = 0; r < R; ++r) X[r] = (uint32_t)gen();
  }
  bool live(int64_t /*arc*/, int32_t u, int32_t v, int32_t r) const {
    return (uint64_t)(X[r] ^ edge_hash(u, v)) < T;
  }
};

// Per-edge probabilities w(u,v) (the w_{u,v} of Algorithm 2 and Eq. 2 in place
// of one uniform p): T_e = floor(w * 2^32) as a 32-bit code c_e; the largest
// code 2^32 - 1 stands for "always live", so w >= 1 - 2^-32 is certain (the
// one reading a 32-bit code forces; every other threshold is exact).
uint32_t edge_code(double w) {
  const uint64_t T = threshold(w);
  return T >= 0xffffffffull ? 0xffffffffu : (uint32_t)T;
}

// Hash sampler with options:
//   codes  per-arc codes c_a (arc = CSR position) or null for the uniform T
//   mix    the mixed variant: the XOR of X_r and h goes through fmix32 before
//          the comparison, so that two edges are co-live with probability
//          about p^2 whatever their hashes (with the plain XOR, edges whose
//          hashes differ above T's magnitude are never co-live in a sample)
struct HashSamplerEx {
  std::vector<uint32_t> X;
  uint64_t T;
  const uint32_t *codes;
  bool mix;
  HashSamplerEx(int32_t R, double p, uint32_t seed, const uint32_t *c, bool m)
      : X(R), T(threshold(p)), codes(c), mix(m) {
    std::mt19937 gen(seed);
    for (int32_t r = 0; r < R; ++r) X[r] = (uint32_t)gen();
  }
  bool live(int64_t a, int32_t u, int32_t v, int32_t r) const {
    uint32_t z = X[r] ^ edge_hash(u, v);
    if (mix) z = fmix32(z);
    if (codes) return codes[a] == 0xffffffffu || z < codes[a];
    return (uint64_t)z < T;
  }
};

// Weights: one per CSR arc, in [0, 1] (NaN rejected), equal on both arcs of
// an edge. Fills the per-arc codes.
bool weights_ok(int32_t n, const int32_t *xadj, const int32_t *adj, const double *w,
                std::vector<uint32_t> &codes) {
  const int64_t arcs = xadj[n];
  codes.resize(arcs);
  for (int64_t a = 0; a < arcs; ++a) {
    if (!(w[a] >= 0.0 && w[a] <= 1.0)) return false;
    codes[a] = edge_code(w[a]);
  }
  for (int32_t u = 0; u < n; ++u)
    for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
      const int32_t v = adj[a];
      bool found = false;
      for (int32_t b = xadj[v]; b < xadj[v + 1]; ++b)
        if (adj[b] == u && w[b] == w[a]) { found = true; break; }
      if (!found) return false;
    }
  return true;
}

// Explicit sampler: live[a * R + r] != 0 for arc a (CSR position) in sample r.
struct MaskSampler {
  const uint8_t *mask;
  int32_t R;
  bool live(int64_t a, int32_t, int32_t, int32_t r) const { return mask[a * R + r] != 0; }
};

// Mask must agree on both orientations of an edge, else "undirected" breaks.
bool mask_symmetric(int32_t n, const int32_t *xadj, const int32_t *adj, const uint8_t *mask,
                    int32_t R) {
  for (int32_t u = 0; u < n; ++u)
    for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
      int32_t v = adj[a];
      int32_t back = -1;
      for (int32_t b = xadj[v]; b < xadj[v + 1]; ++b)
        if (adj[b] == u) { back = b; break; }
      for (int32_t r = 0; r < R; ++r)
        if ((mask[(int64_t)a * R + r] != 0) != (mask[(int64_t)back * R + r] != 0)) return false;
    }
  return true;
}

// ---------------------------------------------------------------- labels
// One simulation r: BFS from every unvisited vertex in increasing id order over
// live arcs; the root (= smallest id of the component) labels every vertex.
template <class S>
void label_one_sample(int32_t n, const int32_t *xadj, const int32_t *adj, const S &smp, int32_t r,
                      std::vector<int32_t> &lab, std::vector<uint32_t> &cnt,
                      std::vector<int32_t> &queue) {
  for (int32_t v = 0; v < n; ++v) lab[v] = -1;
  for (int32_t v = 0; v < n; ++v) cnt[v] = 0;
  for (int32_t root = 0; root < n; ++root) {
    if (lab[root] != -1) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = root;
    lab[root] = root;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
        int32_t v = adj[a];
        if (v == u || lab[v] != -1) continue;
        if (!smp.live(a, u, v, r)) continue;
        lab[v] = root;
        queue[tail++] = v;
      }
    }
    cnt[root] = (uint32_t)tail;
  }
}

// Full n x R label and size tables, vertex-major (the R entries of v are
// contiguous, Section 3.3).
template <class S>
void all_labels(int32_t n, const int32_t *xadj, const int32_t *adj, int32_t R, const S &smp,
                int32_t *labels, uint32_t *sizes) {
#pragma omp parallel
  {
    std::vector<int32_t> lab(n), queue(n);
    std::vector<uint32_t> cnt(n);
#pragma omp for schedule(dynamic, 1)
    for (int32_t r = 0; r < R; ++r) {
      label_one_sample(n, xadj, adj, smp, r, lab, cnt, queue);
      for (int32_t v = 0; v < n; ++v) {
        labels[(int64_t)v * R + r] = lab[v];
        sizes[(int64_t)v * R + r] = cnt[v];
      }
    }
  }
}

// ---------------------------------------------------------------- greedy
// Greedy seed selection over the memoized samples with a covered table
// cov[l*R + r] = 1 once component l of sample r holds a seed.
void greedy(int32_t n, int32_t R, const int32_t *labels, const uint32_t *sizes, int32_t K,
            int32_t *seeds, uint64_t *sigma) {
  std::vector<uint8_t> cov((size_t)n * R, 0), chosen(n, 0);
  uint64_t total = 0;
  for (int32_t k = 0; k < K; ++k) {
    int64_t best = -1;
    uint64_t best_gain = 0;
#pragma omp parallel
    {
      // each thread scans a contiguous id range in increasing order
      int64_t tbest = -1;
      uint64_t tgain = 0;
#pragma omp for schedule(static)
      for (int32_t v = 0; v < n; ++v) {
        if (chosen[v]) continue;
        uint64_t g = 0;
        for (int32_t r = 0; r < R; ++r) {
          int64_t l = labels[(int64_t)v * R + r];
          if (!cov[l * R + r]) g += sizes[l * R + r];
        }
        if (tbest < 0 || g > tgain) {  // strict: lowest id wins ties
          tbest = v;
          tgain = g;
        }
      }
#pragma omp critical
      if (tbest >= 0 && (best < 0 || tgain > best_gain || (tgain == best_gain && tbest < best))) {
        best = tbest;
        best_gain = tgain;
      }
    }
    int32_t s = (int32_t)best;
    chosen[s] = 1;
    for (int32_t r = 0; r < R; ++r) cov[(int64_t)labels[(int64_t)s * R + r] * R + r] = 1;
    total += best_gain;
    seeds[k] = s;
    sigma[k] = total;
  }
}

// ---------------------------------------------------------------- spread
// sigmaR(S) = sum over samples of the number of vertices reachable from S.
template <class S>
uint64_t spread(int32_t n, const int32_t *xadj, const int32_t *adj, int32_t R, const S &smp,
                const int32_t *seeds, int32_t ns) {
  std::vector<uint8_t> seen(n);
  std::vector<int32_t> queue(n);
  uint64_t total = 0;
  for (int32_t r = 0; r < R; ++r) {
    std::fill(seen.begin(), seen.end(), 0);
    int64_t head = 0, tail = 0;
    for (int32_t i = 0; i < ns; ++i)
      if (!seen[seeds[i]]) {
        seen[seeds[i]] = 1;
        queue[tail++] = seeds[i];
      }
    while (head < tail) {
      int32_t u = queue[head++];
      for (int32_t a = xadj[u]; a < xadj[u + 1]; ++a) {
        int32_t v = adj[a];
        if (v == u || seen[v]) continue;
        if (!smp.live(a, u, v, r)) continue;
        seen[v] = 1;
        queue[tail++] = v;
      }
    }
    total += (uint64_t)tail;
  }
  return total;
}

bool seeds_ok(int32_t n, const int32_t *seeds, int32_t ns) {
  if (ns < 0) return false;
  for (int32_t i = 0; i < ns; ++i)
    if (seeds[i] < 0 || seeds[i] >= n) return false;
  return true;
}

bool query_ok(int32_t n, int32_t R, double p) {
  if (R < 1 || R > 65536) return false;
  if (!(p >= 0.0 && p <= 1.0)) return false;
  if ((uint64_t)n * (uint64_t)R >= (1ull << 32)) return false;
  return true;
}

}  // namespace

// ---------------------------------------------------------------- C entry points
// Return 0 on success, -1 on invalid input. Arrays are caller-owned host memory.
extern "C" {

uint32_t orc_murmur3_x86_32(const uint8_t *key, int32_t len, uint32_t seed) {
  return murmur3_x86_32(key, len, seed);
}

uint32_t orc_edge_hash(int32_t u, int32_t v) { return edge_hash(u, v); }

void orc_mt19937(uint32_t seed, int64_t count, uint32_t *out) {
  std::mt19937 gen(seed);
  for (int64_t i = 0; i < count; ++i) out[i] = (uint32_t)gen();
}

uint64_t orc_threshold(double p) { return threshold(p); }

// Threads a parallel region of this build uses (1 without OpenMP).
int32_t orc_max_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

int32_t orc_live(int32_t u, int32_t v, uint32_t x, double p) {
  return (uint64_t)(x ^ edge_hash(u, v)) < threshold(p) ? 1 : 0;
}

int32_t orc_validate_csr(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj) {
  return csr_ok(n, m, xadj, adj) ? 0 : -1;
}

int32_t orc_labels(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj, int32_t R,
                   double p, uint32_t seed, int32_t *labels, uint32_t *sizes) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, p)) return -1;
  HashSampler smp(R, p, seed);
  all_labels(n, xadj, adj, R, smp, labels, sizes);
  return 0;
}

// Labels of a subset of simulations: out[v * nl + i] is the label of v in
// simulation lanes[i] (X drawn from the full stream of R values).
int32_t orc_labels_lanes(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj, int32_t R,
                         double p, uint32_t seed, int32_t nl, const int32_t *lanes,
                         int32_t *labels, uint32_t *sizes) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, p) || nl < 0) return -1;
  for (int32_t i = 0; i < nl; ++i)
    if (lanes[i] < 0 || lanes[i] >= R) return -1;
  HashSampler smp(R, p, seed);
  std::vector<int32_t> lab(n), queue(n);
  std::vector<uint32_t> cnt(n);
  for (int32_t i = 0; i < nl; ++i) {
    label_one_sample(n, xadj, adj, smp, lanes[i], lab, cnt, queue);
    for (int32_t v = 0; v < n; ++v) {
      labels[(int64_t)v * nl + i] = lab[v];
      if (sizes) sizes[(int64_t)v * nl + i] = cnt[v];
    }
  }
  return 0;
}

int32_t orc_select_seeds(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj, int32_t K,
                         int32_t R, double p, uint32_t seed, int32_t *seeds, uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, p) || K < 0 || K > n) return -1;
  HashSampler smp(R, p, seed);
  std::vector<int32_t> labels((size_t)n * R);
  std::vector<uint32_t> sizes((size_t)n * R);
  all_labels(n, xadj, adj, R, smp, labels.data(), sizes.data());
  greedy(n, R, labels.data(), sizes.data(), K, seeds, sigma);
  return 0;
}

int32_t orc_estimate_spread(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                            const int32_t *seeds, int32_t ns, int32_t R, double p, uint32_t seed,
                            uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, p) || !seeds_ok(n, seeds, ns)) return -1;
  HashSampler smp(R, p, seed);
  *sigma = spread(n, xadj, adj, R, smp, seeds, ns);
  return 0;
}

// ----- sampling options: per-arc weights (w: 2m doubles, or null for the
// uniform p) and the mixed hash (mix != 0)
int32_t orc_labels_ex(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj, int32_t R,
                      double p, uint32_t seed, const double *w, int32_t mix, int32_t *labels,
                      uint32_t *sizes) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, w ? 0.5 : p)) return -1;
  std::vector<uint32_t> codes;
  if (w && !weights_ok(n, xadj, adj, w, codes)) return -1;
  HashSamplerEx smp(R, w ? 0.0 : p, seed, w ? codes.data() : nullptr, mix != 0);
  all_labels(n, xadj, adj, R, smp, labels, sizes);
  return 0;
}

int32_t orc_select_seeds_ex(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                            int32_t K, int32_t R, double p, uint32_t seed, const double *w,
                            int32_t mix, int32_t *seeds, uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, w ? 0.5 : p) || K < 0 || K > n) return -1;
  std::vector<uint32_t> codes;
  if (w && !weights_ok(n, xadj, adj, w, codes)) return -1;
  HashSamplerEx smp(R, w ? 0.0 : p, seed, w ? codes.data() : nullptr, mix != 0);
  std::vector<int32_t> labels((size_t)n * R);
  std::vector<uint32_t> sizes((size_t)n * R);
  all_labels(n, xadj, adj, R, smp, labels.data(), sizes.data());
  greedy(n, R, labels.data(), sizes.data(), K, seeds, sigma);
  return 0;
}

int32_t orc_estimate_spread_ex(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                               const int32_t *seeds, int32_t ns, int32_t R, double p,
                               uint32_t seed, const double *w, int32_t mix, uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || !query_ok(n, R, w ? 0.5 : p) || !seeds_ok(n, seeds, ns))
    return -1;
  std::vector<uint32_t> codes;
  if (w && !weights_ok(n, xadj, adj, w, codes)) return -1;
  HashSamplerEx smp(R, w ? 0.0 : p, seed, w ? codes.data() : nullptr, mix != 0);
  *sigma = spread(n, xadj, adj, R, smp, seeds, ns);
  return 0;
}

// Live test of one arc under the options: the code of weight w when use_w,
// else the uniform p; the mixed hash when mix.
int32_t orc_live_ex(int32_t u, int32_t v, uint32_t x, double p, double w, int32_t use_w,
                    int32_t mix) {
  uint32_t z = x ^ edge_hash(u, v);
  if (mix) z = fmix32(z);
  if (use_w) {
    const uint32_t c = edge_code(w);
    return (c == 0xffffffffu || z < c) ? 1 : 0;
  }
  return (uint64_t)z < threshold(p) ? 1 : 0;
}

uint32_t orc_fmix32(uint32_t h) { return fmix32(h); }

uint32_t orc_edge_code(double w) { return edge_code(w); }

// Greedy from caller-provided label/size tables (n x R, vertex-major).
int32_t orc_greedy_from_tables(int32_t n, int32_t R, const int32_t *labels, const uint32_t *sizes,
                               int32_t K, int32_t *seeds, uint64_t *sigma) {
  if (n < 1 || R < 1 || K < 0 || K > n) return -1;
  greedy(n, R, labels, sizes, K, seeds, sigma);
  return 0;
}

// Marginal gains g(v | S) for every v (0 for v in S) from label/size tables.
int32_t orc_marginal_gains(int32_t n, int32_t R, const int32_t *labels, const uint32_t *sizes,
                           const int32_t *S, int32_t ns, uint64_t *gains) {
  if (n < 1 || R < 1 || !seeds_ok(n, S, ns)) return -1;
  std::vector<uint8_t> cov((size_t)n * R, 0), in_s(n, 0);
  for (int32_t i = 0; i < ns; ++i) {
    in_s[S[i]] = 1;
    for (int32_t r = 0; r < R; ++r) cov[(int64_t)labels[(int64_t)S[i] * R + r] * R + r] = 1;
  }
  for (int32_t v = 0; v < n; ++v) {
    uint64_t g = 0;
    if (!in_s[v])
      for (int32_t r = 0; r < R; ++r) {
        int64_t l = labels[(int64_t)v * R + r];
        if (!cov[l * R + r]) g += sizes[l * R + r];
      }
    gains[v] = g;
  }
  return 0;
}

// ----- explicit-mask sampler variants (mask[a * R + r], a = CSR arc index)
int32_t orc_labels_masked(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj, int32_t R,
                          const uint8_t *mask, int32_t *labels, uint32_t *sizes) {
  if (!csr_ok(n, m, xadj, adj) || R < 1 || !mask_symmetric(n, xadj, adj, mask, R)) return -1;
  MaskSampler smp{mask, R};
  all_labels(n, xadj, adj, R, smp, labels, sizes);
  return 0;
}

int32_t orc_select_seeds_masked(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                                int32_t K, int32_t R, const uint8_t *mask, int32_t *seeds,
                                uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || R < 1 || K < 0 || K > n ||
      !mask_symmetric(n, xadj, adj, mask, R))
    return -1;
  MaskSampler smp{mask, R};
  std::vector<int32_t> labels((size_t)n * R);
  std::vector<uint32_t> sizes((size_t)n * R);
  all_labels(n, xadj, adj, R, smp, labels.data(), sizes.data());
  greedy(n, R, labels.data(), sizes.data(), K, seeds, sigma);
  return 0;
}

int32_t orc_estimate_spread_masked(int32_t n, int64_t m, const int32_t *xadj, const int32_t *adj,
                                   const int32_t *seeds, int32_t ns, int32_t R,
                                   const uint8_t *mask, uint64_t *sigma) {
  if (!csr_ok(n, m, xadj, adj) || R < 1 || !seeds_ok(n, seeds, ns) ||
      !mask_symmetric(n, xadj, adj, mask, R))
    return -1;
  MaskSampler smp{mask, R};
  *sigma = spread(n, xadj, adj, R, smp, seeds, ns);
  return 0;
}

}  // extern "C"
