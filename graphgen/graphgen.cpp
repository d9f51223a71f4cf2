// Seeded synthetic graph generators and a canonical CSR builder.
//
// This module only makes inputs.  It holds none of the colouring method's
// arithmetic: no degree thresholds, no priorities, no colours.  Both the CPU
// oracle and the CUDA path receive the CSR arrays it writes.
//
// Every generator is a pure function of its parameters and seed: random draws
// come from a counter-based generator (SplitMix64: Steele, Lea & Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014), so the
// result does not depend on the number of worker threads.  The CSR it builds is
// canonical: undirected, symmetric, no self-loops, no duplicate edges, each
// row sorted ascending, int64 row offsets and int32 column ids (the graph model
// of the paper's Section 2.1).
//
// Families (recipes follow the paper's workload classes, Section 6):
//   ER     G(n, m) with exactly m distinct undirected edges
//   R-MAT  2x2 stochastic Kronecker sampler (a, b, c, d), edge factor ef
//   BA     Barabasi-Albert preferential attachment, seed clique K_{m+1}
//   grid   2D k1 x k2 (4-neighbour) and 3D k1 x k2 x k3 (6-neighbour)
//   any of them relabelled by a seeded Fisher-Yates permutation
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// k-th draw (k >= 0) of stream `stream` under `seed`.
inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t k) {
  uint64_t base = mix64(seed * kGamma + stream * 0xd1b54a32d192ed03ULL + 0x632be59bd9b4e019ULL);
  return mix64(base + (k + 1) * kGamma);
}

// Uniform integer in [0, bound) by 128-bit multiply-shift (Lemire); bias is
// below 2^-32 for the bounds used here, which is fine for input synthesis.
inline uint64_t below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

int num_threads() {
  const char* env = std::getenv("GRAPHGEN_THREADS");
  if (env) {
    int t = std::atoi(env);
    if (t > 0) return t;
  }
  unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 1 : (int)std::min(h, 64u);
}

template <class F>
void parallel_for(int64_t begin, int64_t end, F&& fn) {
  int64_t total = end - begin;
  if (total <= 0) return;
  int T = num_threads();
  if (total < 65536 || T == 1) {
    fn(begin, end);
    return;
  }
  std::vector<std::thread> pool;
  int64_t chunk = (total + T - 1) / T;
  for (int t = 0; t < T; ++t) {
    int64_t b = begin + t * chunk, e = std::min(end, b + chunk);
    if (b >= e) break;
    pool.emplace_back([&fn, b, e] { fn(b, e); });
  }
  for (auto& th : pool) th.join();
}

// Dynamic scheduling for uneven work (row sorts where hubs are long).
template <class F>
void parallel_dynamic(int64_t count, int64_t grain, F&& fn) {
  if (count <= 0) return;
  int T = num_threads();
  if (count < 4 * grain || T == 1) {
    fn((int64_t)0, count);
    return;
  }
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t)
    pool.emplace_back([&] {
      for (;;) {
        int64_t b = next.fetch_add(grain);
        if (b >= count) break;
        fn(b, std::min(count, b + grain));
      }
    });
  for (auto& th : pool) th.join();
}

struct Csr {
  int64_t n = 0;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col_idx;
};

// Canonical CSR from an undirected edge list (self-loops and duplicates
// dropped, both directions stored, rows sorted).
int build_csr(int64_t n, int64_t M, const uint32_t* src, const uint32_t* dst, Csr* out) {
  if (n < 0 || n > (int64_t)INT32_MAX) return 1;
  std::vector<uint32_t> deg(n, 0);
  int bad = 0;
  parallel_for(0, M, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      uint32_t u = src[i], v = dst[i];
      if ((int64_t)u >= n || (int64_t)v >= n) {
        __atomic_store_n(&bad, 1, __ATOMIC_RELAXED);
        continue;
      }
      if (u == v) continue;
      __atomic_fetch_add(&deg[u], 1u, __ATOMIC_RELAXED);
      __atomic_fetch_add(&deg[v], 1u, __ATOMIC_RELAXED);
    }
  });
  if (bad) return 2;
  std::vector<int64_t> off(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
  std::vector<int32_t> tmp(off[n]);
  {
    std::vector<int64_t> cur(off.begin(), off.end() - 1);
    parallel_for(0, M, [&](int64_t b, int64_t e) {
      for (int64_t i = b; i < e; ++i) {
        uint32_t u = src[i], v = dst[i];
        if (u == v) continue;
        tmp[__atomic_fetch_add(&cur[u], (int64_t)1, __ATOMIC_RELAXED)] = (int32_t)v;
        tmp[__atomic_fetch_add(&cur[v], (int64_t)1, __ATOMIC_RELAXED)] = (int32_t)u;
      }
    });
  }
  std::vector<int64_t> uniq(n, 0);
  parallel_dynamic(n, 4096, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v) {
      int32_t* s = tmp.data() + off[v];
      int32_t* t = tmp.data() + off[v + 1];
      std::sort(s, t);
      uniq[v] = std::unique(s, t) - s;
    }
  });
  out->n = n;
  out->row_ptr.assign(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) out->row_ptr[v + 1] = out->row_ptr[v] + uniq[v];
  out->col_idx.resize(out->row_ptr[n]);
  parallel_for(0, n, [&](int64_t b, int64_t e) {
    for (int64_t v = b; v < e; ++v)
      std::memcpy(out->col_idx.data() + out->row_ptr[v], tmp.data() + off[v], uniq[v] * sizeof(int32_t));
  });
  return 0;
}

// Relabel vertex v -> perm[v] with a seeded Fisher-Yates shuffle, rebuild CSR.
int permute_csr(const Csr& g, uint64_t seed, Csr* out) {
  int64_t n = g.n;
  std::vector<uint32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)below(draw(seed, 7, (uint64_t)i), (uint64_t)(i + 1));
    std::swap(perm[i], perm[j]);
  }
  int64_t M = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t k = g.row_ptr[v]; k < g.row_ptr[v + 1]; ++k)
      if (g.col_idx[k] > v) ++M;
  std::vector<uint32_t> s(M), t(M);
  int64_t i = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t k = g.row_ptr[v]; k < g.row_ptr[v + 1]; ++k)
      if (g.col_idx[k] > v) {
        s[i] = perm[v];
        t[i] = perm[g.col_idx[k]];
        ++i;
      }
  return build_csr(n, M, s.data(), t.data(), out);
}

int gen_er(int64_t n, int64_t m, uint64_t seed, Csr* out) {
  if (n < 0 || m < 0) return 1;
  if (n < 2) {
    if (m > 0) return 1;
    return build_csr(n, 0, nullptr, nullptr, out);
  }
  if ((unsigned __int128)m > (unsigned __int128)n * (n - 1) / 2) return 1;
  // Accept candidates in stream order; keep the first m distinct pairs.
  uint64_t cap = 16;
  while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
  std::vector<uint64_t> table(cap, ~0ULL);
  std::vector<uint32_t> s, t;
  s.reserve(m);
  t.reserve(m);
  for (uint64_t k = 0; (int64_t)s.size() < m; ++k) {
    uint64_t r = draw(seed, 1, k);
    // two 32-bit halves scaled into [0, n) by multiply-shift
    uint64_t u = ((r & 0xffffffffULL) * (uint64_t)n) >> 32;
    uint64_t v = ((r >> 32) * (uint64_t)n) >> 32;
    if (u == v) continue;
    if (u > v) std::swap(u, v);
    uint64_t key = (u << 32) | v;
    uint64_t h = mix64(key) & (cap - 1);
    bool dup = false;
    while (table[h] != ~0ULL) {
      if (table[h] == key) {
        dup = true;
        break;
      }
      h = (h + 1) & (cap - 1);
    }
    if (dup) continue;
    table[h] = key;
    s.push_back((uint32_t)u);
    t.push_back((uint32_t)v);
  }
  return build_csr(n, m, s.data(), t.data(), out);
}

int gen_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed, Csr* out) {
  if (scale < 1 || scale > 30 || edge_factor < 0) return 1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
  const int64_t n = (int64_t)1 << scale;
  const int64_t M = edge_factor * n;
  const uint64_t two32 = 1ULL << 32;
  const uint64_t ta = (uint64_t)(a * (double)two32);
  const uint64_t tab = (uint64_t)((a + b) * (double)two32);
  const uint64_t tabc = (uint64_t)((a + b + c) * (double)two32);
  const int64_t words = (scale + 1) / 2;  // two 32-bit draws per 64-bit word
  std::vector<uint32_t> s(M), t(M);
  parallel_for(0, M, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      uint32_t u = 0, v = 0;
      uint64_t w = 0;
      for (int lev = 0; lev < scale; ++lev) {
        if ((lev & 1) == 0) w = draw(seed, 2, (uint64_t)(i * words + lev / 2));
        uint64_t r = (lev & 1) ? (w >> 32) : (w & 0xffffffffULL);
        uint32_t bu, bv;
        if (r < ta) {
          bu = 0; bv = 0;
        } else if (r < tab) {
          bu = 0; bv = 1;
        } else if (r < tabc) {
          bu = 1; bv = 0;
        } else {
          bu = 1; bv = 1;
        }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
      }
      s[i] = u;
      t[i] = v;
    }
  });
  return build_csr(n, M, s.data(), t.data(), out);
}

// Barabasi-Albert: start from the clique K_{m+1}; each later vertex links to m
// distinct earlier vertices drawn with probability proportional to degree
// (uniform pick from the endpoint list).
int gen_ba(int64_t n, int64_t m, uint64_t seed, Csr* out) {
  if (n < 0 || m < 1) return 1;
  int64_t core = std::min(n, m + 1);
  std::vector<uint32_t> s, t, ends;
  for (int64_t u = 0; u < core; ++u)
    for (int64_t v = u + 1; v < core; ++v) {
      s.push_back((uint32_t)u);
      t.push_back((uint32_t)v);
      ends.push_back((uint32_t)u);
      ends.push_back((uint32_t)v);
    }
  uint64_t k = 0;
  std::vector<uint32_t> picked;
  for (int64_t v = core; v < n; ++v) {
    picked.clear();
    while ((int64_t)picked.size() < m) {
      uint32_t w = ends[below(draw(seed, 3, k++), (uint64_t)ends.size())];
      if (std::find(picked.begin(), picked.end(), w) == picked.end()) picked.push_back(w);
    }
    for (uint32_t w : picked) {
      s.push_back((uint32_t)v);
      t.push_back(w);
      ends.push_back((uint32_t)v);
      ends.push_back(w);
    }
  }
  return build_csr(n, (int64_t)s.size(), s.data(), t.data(), out);
}

int gen_grid(int64_t k1, int64_t k2, int64_t k3, Csr* out) {
  if (k1 < 1 || k2 < 1 || k3 < 1) return 1;
  int64_t n = k1 * k2 * k3;
  if (n > (int64_t)INT32_MAX) return 1;
  int64_t M = (k1 - 1) * k2 * k3 + k1 * (k2 - 1) * k3 + k1 * k2 * (k3 - 1);
  std::vector<uint32_t> s(M), t(M);
  int64_t i = 0;
  for (int64_t z = 0; z < k3; ++z)
    for (int64_t y = 0; y < k2; ++y)
      for (int64_t x = 0; x < k1; ++x) {
        int64_t v = (z * k2 + y) * k1 + x;
        if (x + 1 < k1) { s[i] = (uint32_t)v; t[i] = (uint32_t)(v + 1); ++i; }
        if (y + 1 < k2) { s[i] = (uint32_t)v; t[i] = (uint32_t)(v + k1); ++i; }
        if (z + 1 < k3) { s[i] = (uint32_t)v; t[i] = (uint32_t)(v + k1 * k2); ++i; }
      }
  return build_csr(n, M, s.data(), t.data(), out);
}

}  // namespace

extern "C" {

typedef struct gg_graph gg_graph;
struct gg_graph {
  Csr csr;
};

int64_t gg_n(const gg_graph* g) { return g ? g->csr.n : -1; }
int64_t gg_nnz(const gg_graph* g) { return g ? g->csr.row_ptr.back() : -1; }

// Copy the CSR into caller buffers of n+1 int64 and nnz int32 entries.
int gg_export(const gg_graph* g, int64_t* row_ptr, int32_t* col_idx) {
  if (!g) return 1;
  std::memcpy(row_ptr, g->csr.row_ptr.data(), (g->csr.n + 1) * sizeof(int64_t));
  std::memcpy(col_idx, g->csr.col_idx.data(), g->csr.col_idx.size() * sizeof(int32_t));
  return 0;
}

void gg_free(gg_graph* g) { delete g; }

static gg_graph* finish(int rc, gg_graph* g) {
  if (rc != 0) {
    delete g;
    return nullptr;
  }
  return g;
}

gg_graph* gg_from_edges(int64_t n, int64_t M, const uint32_t* src, const uint32_t* dst) {
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return nullptr;
  return finish(build_csr(n, M, src, dst, &g->csr), g);
}

gg_graph* gg_er(int64_t n, int64_t m, uint64_t seed) {
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return nullptr;
  return finish(gen_er(n, m, seed, &g->csr), g);
}

gg_graph* gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed) {
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return nullptr;
  return finish(gen_rmat(scale, edge_factor, a, b, c, seed, &g->csr), g);
}

gg_graph* gg_ba(int64_t n, int64_t m, uint64_t seed) {
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return nullptr;
  return finish(gen_ba(n, m, seed, &g->csr), g);
}

gg_graph* gg_grid(int64_t k1, int64_t k2, int64_t k3) {
  gg_graph* g = new (std::nothrow) gg_graph();
  if (!g) return nullptr;
  return finish(gen_grid(k1, k2, k3, &g->csr), g);
}

// Returns a new graph: `g` relabelled by a seeded permutation (g unchanged).
gg_graph* gg_permute(const gg_graph* g, uint64_t seed) {
  if (!g) return nullptr;
  gg_graph* h = new (std::nothrow) gg_graph();
  if (!h) return nullptr;
  return finish(permute_csr(g->csr, seed, &h->csr), h);
}

// Uniform 64-bit draw k of stream s (exposed so that Python-side recipes,
// such as the per-graph sizes of a batched workload, use the same generator).
uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t k) { return draw(seed, stream, k); }

// Recipe of a batched workload: graph g has n log-uniform in [n_lo, n_hi]
// (from draw 2g of stream 11) and family draw(2g+1) % 3: 0 = Erdos-Renyi with
// m = 4n (average degree 8), 1 = Barabasi-Albert with m = 4, 2 = 2D grid with
// k = ceil(sqrt(n)) per side.
void gg_batch_recipe(int64_t count, int64_t n_lo, int64_t n_hi, uint64_t seed, int32_t* fam, int64_t* n) {
  const double lo = std::log(static_cast<double>(n_lo)), hi = std::log(static_cast<double>(n_hi));
  for (int64_t g = 0; g < count; ++g) {
    const double u = static_cast<double>(draw(seed, 11, 2 * g) >> 11) / 9007199254740992.0;
    n[g] = static_cast<int64_t>(std::llround(std::exp(lo + u * (hi - lo))));
    fam[g] = static_cast<int32_t>(draw(seed, 11, 2 * g + 1) % 3);
  }
}

// The whole batched workload generated in parallel (graphs over threads) and
// packed as the disjoint union: graph g is generated with seed `seed + g`.
gg_graph* gg_batch(int64_t count, int64_t n_lo, int64_t n_hi, uint64_t seed, int64_t* graph_off) {
  std::vector<int32_t> fam(count);
  std::vector<int64_t> nv(count);
  gg_batch_recipe(count, n_lo, n_hi, seed, fam.data(), nv.data());
  std::vector<Csr> parts(count);
  std::atomic<int> bad{0};
  std::atomic<int64_t> next{0};
  std::vector<std::thread> pool;
  const int T = num_threads();
  for (int t = 0; t < T; ++t)
    pool.emplace_back([&] {
      for (;;) {
        const int64_t g = next.fetch_add(1);
        if (g >= count) break;
        int rc;
        const int64_t n = nv[g];
        if (fam[g] == 0) {
          rc = gen_er(n, 4 * n, seed + g, &parts[g]);
        } else if (fam[g] == 1) {
          rc = gen_ba(n, 4, seed + g, &parts[g]);
        } else {
          const int64_t k = static_cast<int64_t>(std::ceil(std::sqrt(static_cast<double>(n))));
          rc = gen_grid(k, k, 1, &parts[g]);
        }
        if (rc) bad.store(1);
      }
    });
  for (auto& th : pool) th.join();
  if (bad.load()) return nullptr;
  gg_graph* out = new (std::nothrow) gg_graph();
  if (!out) return nullptr;
  graph_off[0] = 0;
  std::vector<int64_t> eoff(count + 1, 0);
  for (int64_t g = 0; g < count; ++g) {
    graph_off[g + 1] = graph_off[g] + parts[g].n;
    eoff[g + 1] = eoff[g] + static_cast<int64_t>(parts[g].col_idx.size());
  }
  Csr& c = out->csr;
  c.n = graph_off[count];
  c.row_ptr.assign(c.n + 1, 0);
  c.col_idx.resize(eoff[count]);
  parallel_dynamic(count, 8, [&](int64_t b, int64_t e) {
    for (int64_t g = b; g < e; ++g) {
      const Csr& p = parts[g];
      for (int64_t v = 0; v < p.n; ++v) c.row_ptr[graph_off[g] + v] = p.row_ptr[v] + eoff[g];
      for (size_t k = 0; k < p.col_idx.size(); ++k)
        c.col_idx[eoff[g] + k] = p.col_idx[k] + static_cast<int32_t>(graph_off[g]);
    }
  });
  c.row_ptr[c.n] = eoff[count];
  return out;
}

}  // extern "C"
