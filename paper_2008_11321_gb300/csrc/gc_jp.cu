// JP colouring, Algorithm 3 (Section 4.1), by predecessor polling.
//
// Algorithm 3 colours a vertex once all its predecessors (neighbours of
// higher priority) are coloured, with the smallest colour none of them uses
// (GetColor).  Here a vertex is handed to a lane (degree <= kSmallDeg) or to a
// whole warp (larger degree); the lane/warp reads the adjacency, keeps the
// colours of predecessors already coloured and waits on the rest by polling
// their colour words until they turn non-zero, then writes its own colour.
// Colour words are written exactly once, so a non-zero value read with a
// relaxed GPU-scope load is final, and no predecessor counters, atomics or
// queues are needed (the Join of Algorithm 3 becomes the poll).
//
// Progress.  Workers take vertices from lists in (nearly) decreasing priority
// order.  Let v* be the unfinished vertex of highest priority: all its
// predecessors are finished.  If v* has not been taken yet, every worker of
// its list that is stuck holds a vertex placed before v* but of lower
// priority, which the order only allows inside v*'s own bucket (vertices whose
// order keys tie).  Buckets hold far fewer vertices than a list has workers,
// so some worker is free and takes v*.  Every block serves both lists, so
// this holds with or without all blocks resident.  Every wait is still
// bounded (4 s by default); a wait that runs out sets the error word and the
// remaining waits end early, so the kernel always returns.
//
// JP-ADG (the fused path of gc_color_graph) runs in three stages:
//   1. order: one counting-sort pass by (batch, top bits of rho_R) gives the
//      order without a comparison sort; isolated vertices take colour 1 at once
//      and drop out.  The first buckets, up to the core target (16384 by
//      default, at most 32768) vertices, form the
//      "core"; they are sorted exactly inside their (tiny) buckets.
//   2. core: the predecessors of each core vertex all lie in the core; they
//      are extracted across the whole GPU into compact lists of core-local
//      ids, then ONE thread-block cluster (up to 16 SMs) colours the core in
//      order with a copy of the core's colours in every CTA's shared memory,
//      where a dependency step costs a shared-memory poll rather than an L2
//      round trip.  The core holds the long chains of the DAG G_rho (the
//      densest part of the graph, which ADG ranks last).
//   3. bulk: every other vertex by global polling (above), with all core
//      colours already final.
// gc_jp_color with an arbitrary priority array orders the vertices with an
// exact radix sort and runs stage 3 on all of them.
#include <cstring>
#include <vector>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kJpThreads = 256;
constexpr int kJpWarps = kJpThreads / kWarp;
constexpr unsigned kBigBit = 0x80000000u;
constexpr int kCoreThreads = 1024;  // largest core CTA
constexpr int kCoreWarps = kCoreThreads / kWarp;
constexpr int kCoreWarpsDefault = 12;

__device__ __forceinline__ bool precedes(unsigned long long kw, int w, unsigned long long kv, int v) {
  return kw > kv || (kw == kv && w > v);
}

// Priorities.  key(v) is the 64-bit order key (rho(w) > rho(v) iff
// precedes(key(w), w, key(v), v)).  For neighbour w of v the colouring loops
// take g = pgather(w, color) first, then pred_g(g, w, key(v), v) (is w a
// predecessor?) and color_g(g, color, w) (its colour, 0 = not yet); a vertex
// stores cword(key(v), c) for colour c, and a colour word x means colour
// x & cmask().

struct KeyFused {  // JP-ADG: (batch << 32) | rho_R(v), rho_R from one seed
  using W = int;  // the colour word
  const int* batch;
  unsigned long long seed;
  __device__ __forceinline__ int bat(int v) const { return __ldg(batch + v); }
  __device__ __forceinline__ unsigned tie(int v) const { return tie_hash(seed, static_cast<unsigned>(v)); }
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(bat(v))) << 32) | tie(v);
  }
  using PG = unsigned long long;
  __device__ __forceinline__ PG pgather(int w, const int*) const { return (*this)(w); }
  __device__ __forceinline__ bool pred_g(PG kw, int w, unsigned long long kv, int v) const {
    return precedes(kw, w, kv, v);
  }
  __device__ __forceinline__ int color_g(PG, const int* color, int w) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ int cmask() const { return ~0; }
  __device__ __forceinline__ int cword(unsigned long long, int c) const { return c; }
};

// JP-ADG with each vertex's batch kept in the top 8 bits of its colour word
// (batch << 24 | colour; ADG took at most 255 rounds, and c colours need at
// least c(c-1)/2 edges, so colours stay below 2^24): one load of a
// neighbour's word gives both its priority and its colour, and the randomly
// read state is one n-word array instead of two.
struct KeyState {
  using W = int;
  const int* state;  // the colour array during JP-ADG
  unsigned long long seed;
  // a coherent load: colour bits of the array change while JP runs (the
  // batch bits never do)
  __device__ __forceinline__ int bat(int v) const { return static_cast<int>(static_cast<unsigned>(state[v]) >> 24); }
  __device__ __forceinline__ unsigned tie(int v) const { return tie_hash(seed, static_cast<unsigned>(v)); }
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(bat(v))) << 32) | tie(v);
  }
  using PG = int;
  __device__ __forceinline__ PG pgather(int w, const int* color) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ bool pred_g(PG x, int w, unsigned long long kv, int v) const {
    const unsigned long long kw =
        (static_cast<unsigned long long>(static_cast<unsigned>(x) >> 24) << 32) | tie(w);
    return precedes(kw, w, kv, v);
  }
  __device__ __forceinline__ int color_g(PG x, const int*, int) const { return x & 0xffffff; }
  __device__ __forceinline__ int cmask() const { return 0xffffff; }
  __device__ __forceinline__ int cword(unsigned long long kv, int c) const {
    return static_cast<int>(static_cast<unsigned>(kv >> 32) << 24) | c;
  }
};

// KeyState in a 16-bit word: batch << cb | colour, with cb colour bits.  It
// applies when the batch fits 16 - cb bits and every colour fits cb bits:
// a colour is at most 1 + |pred(v)|, and pred(v) lies among the neighbours
// that ADG's degree at removal D[v] counts (those in the same or a later
// batch), so colour <= 1 + max D[v].  On R-MAT scale 24 (7 batches, max D
// 2,901) 3 + 13 bits suffice, and the randomly read state of the bulk shrinks
// from 67 MB to 33.5 MB, well inside L2.
struct KeyState16 {
  using W = unsigned short;
  const unsigned short* state;  // the 16-bit state array during JP-ADG
  unsigned long long seed;
  int cb;  // colour bits
  __device__ __forceinline__ int bat(int v) const { return static_cast<int>(static_cast<unsigned>(state[v]) >> cb); }
  __device__ __forceinline__ unsigned tie(int v) const { return tie_hash(seed, static_cast<unsigned>(v)); }
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(bat(v))) << 32) | tie(v);
  }
  using PG = int;
  __device__ __forceinline__ PG pgather(int w, const unsigned short* color) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ bool pred_g(PG x, int w, unsigned long long kv, int v) const {
    const unsigned long long kw = (static_cast<unsigned long long>(static_cast<unsigned>(x) >> cb) << 32) | tie(w);
    return precedes(kw, w, kv, v);
  }
  __device__ __forceinline__ int color_g(PG x, const unsigned short*, int) const { return x & cmask(); }
  __device__ __forceinline__ int cmask() const { return (1 << cb) - 1; }
  __device__ __forceinline__ int cword(unsigned long long kv, int c) const {
    return static_cast<int>(static_cast<unsigned>(kv >> 32) << cb) | c;
  }
};

struct KeyPacked {  // JP-ADG over many disjoint graphs: rho_R precomputed per vertex
  using W = int;
  const int* batch;
  const unsigned* tiev;
  __device__ __forceinline__ int bat(int v) const { return __ldg(batch + v); }
  __device__ __forceinline__ unsigned tie(int v) const { return __ldg(tiev + v); }
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(bat(v))) << 32) | tie(v);
  }
  using PG = unsigned long long;
  __device__ __forceinline__ PG pgather(int w, const int*) const { return (*this)(w); }
  __device__ __forceinline__ bool pred_g(PG kw, int w, unsigned long long kv, int v) const {
    return precedes(kw, w, kv, v);
  }
  __device__ __forceinline__ int color_g(PG, const int* color, int w) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ int cmask() const { return ~0; }
  __device__ __forceinline__ int cword(unsigned long long, int c) const { return c; }
};

// JP-ADG over many disjoint graphs with the batch kept in the top 8 bits of
// the colour word (batches up to 255): one load of a neighbour's word gives
// its batch and colour.  rho_R of a vertex comes from its graph's seed and
// its id inside the graph; a neighbour is in the same graph (no edge joins
// two graphs), so its rho_R -- needed only when the batches are equal -- is
// computed from the vertex's own graph, with no load of the neighbour's.
struct KeyStateG {
  using W = int;
  const int* state;  // the colour array during JP
  const int* gid;    // graph of each vertex
  const unsigned long long* seed;  // per graph
  const long long* off;            // first vertex of each graph
  __device__ __forceinline__ int bat(int v) const { return static_cast<int>(static_cast<unsigned>(state[v]) >> 24); }
  __device__ __forceinline__ unsigned tie_in(int g, int v) const {
    return tie_hash(__ldg(seed + g), static_cast<unsigned>(v - __ldg(off + g)));
  }
  __device__ __forceinline__ unsigned tie(int v) const { return tie_in(__ldg(gid + v), v); }
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(bat(v))) << 32) | tie(v);
  }
  using PG = int;
  __device__ __forceinline__ PG pgather(int w, const int* color) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ bool pred_g(PG x, int w, unsigned long long kv, int v) const {
    const unsigned bw = static_cast<unsigned>(x) >> 24, bv = static_cast<unsigned>(kv >> 32);
    if (bw != bv) return bw > bv;
    const unsigned tw = tie_in(__ldg(gid + v), w), tv = static_cast<unsigned>(kv);
    return tw > tv || (tw == tv && w > v);
  }
  __device__ __forceinline__ int color_g(PG x, const int*, int) const { return x & 0xffffff; }
  __device__ __forceinline__ int cmask() const { return 0xffffff; }
  __device__ __forceinline__ int cword(unsigned long long kv, int c) const {
    return static_cast<int>(static_cast<unsigned>(kv >> 32) << 24) | c;
  }
};

// JP-ADG-O: the priority (batch, D at removal, id), with the batch kept in
// the top 8 bits of the colour word as in KeyState; D is read only for a
// neighbour of the same batch.
struct KeyStateD {
  using W = int;
  const int* state;  // the colour array during JP-ADG-O
  const int* D;
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(__ldg(state + v)) >> 24) << 32) |
           static_cast<unsigned>(__ldg(D + v));
  }
  using PG = int;
  __device__ __forceinline__ PG pgather(int w, const int* color) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ bool pred_g(PG x, int w, unsigned long long kv, int v) const {
    const unsigned bw = static_cast<unsigned>(x) >> 24, bv = static_cast<unsigned>(kv >> 32);
    if (bw != bv) return bw > bv;
    const unsigned dw = static_cast<unsigned>(__ldg(D + w)), dv = static_cast<unsigned>(kv);
    return dw > dv || (dw == dv && w > v);
  }
  __device__ __forceinline__ int color_g(PG x, const int*, int) const { return x & 0xffffff; }
  __device__ __forceinline__ int cmask() const { return 0xffffff; }
  __device__ __forceinline__ int cword(unsigned long long kv, int c) const {
    return static_cast<int>(static_cast<unsigned>(kv >> 32) << 24) | c;
  }
};

struct KeyGiven {  // any priority array
  using W = int;
  const unsigned long long* prio;
  __device__ __forceinline__ unsigned long long operator()(int v) const { return __ldg(prio + v); }
  using PG = unsigned long long;
  __device__ __forceinline__ PG pgather(int w, const int*) const { return (*this)(w); }
  __device__ __forceinline__ bool pred_g(PG kw, int w, unsigned long long kv, int v) const {
    return precedes(kw, w, kv, v);
  }
  __device__ __forceinline__ int color_g(PG, const int* color, int w) const { return ld_relaxed(color + w); }
  __device__ __forceinline__ int cmask() const { return ~0; }
  __device__ __forceinline__ int cword(unsigned long long, int c) const { return c; }
};

__device__ __forceinline__ long long gtid() {
  return static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() {
  return static_cast<long long>(gridDim.x) * blockDim.x;
}

// Per-launch constants of the bulk kernel, read from the control block once
// per block into shared memory.
struct JpLimits {
  unsigned long long wait_ns;  // bound of a wait
  int stall;                   // injected fault: vertex that never publishes (-1: none)
};

// ---------------------------------------------------------------------------
// Waiting on a colour word (global memory), bounded.  The poll does not
// back off: a sleeping waiter notices its predecessor late, and every such
// delay on a dependency chain adds to the launch (R-MAT 24: 32 -> 256 ns
// exponential backoff made the bulk 3% slower than polling flat out).
// ---------------------------------------------------------------------------
template <class Wd>
__device__ __forceinline__ int wait_color(const Wd* p, int cmask, JpCtl* ctl, const JpLimits& lim,
                                          unsigned long long& spins) {
  int c = ld_relaxed(p) & cmask;
  if (c != 0) return c;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    c = ld_relaxed(p) & cmask;
    if (c != 0) return c;
    ++spins;
    if ((it & 15u) == 0) {
      if (ld_relaxed(&ctl->err) != 0) return 1;
      if (global_ns() - t0 > lim.wait_ns) {
        atomicExch(&ctl->err, kDevTimeout);
        return 1;
      }
    }
  }
}

// GetColor for a vertex of degree <= kSmallDeg, by one lane: at most 32
// predecessors, so the smallest free colour is <= 33 and a 64-bit mask of
// used colours suffices.  Neighbours are read eight at a time so that their
// loads overlap; predecessors not yet coloured are remembered in a 32-bit
// position mask and waited on after the scan.
template <class Key>
__device__ int color_lane(int v, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                          const Key& key, typename Key::W* color, JpCtl* ctl, const JpLimits& lim,
                          unsigned long long& spins) {
  constexpr int U = 8;
  const unsigned long long kv = key(v);
  const long long s = row_ptr[v], e = row_ptr[v + 1];
  unsigned long long used = 0;
  unsigned later = 0;
  for (long long k = s; k < e; k += U) {
    int w[U], c[U];
    typename Key::PG g[U];
    bool pred[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = k + u < e ? __ldg(col + k + u) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) g[u] = w[u] >= 0 ? key.pgather(w[u], color) : typename Key::PG{};
#pragma unroll
    for (int u = 0; u < U; ++u) pred[u] = w[u] >= 0 && key.pred_g(g[u], w[u], kv, v);
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = pred[u] ? key.color_g(g[u], color, w[u]) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!pred[u]) continue;
      if (c[u] == 0)
        later |= 1u << static_cast<int>(k + u - s);
      else if (c[u] <= 64)
        used |= 1ull << (c[u] - 1);
    }
  }
  while (later) {
    const int pos = __ffs(later) - 1;
    later &= later - 1;
    const int cu = wait_color(color + __ldg(col + s + pos), key.cmask(), ctl, lim, spins);
    if (cu <= 64) used |= 1ull << (cu - 1);
  }
  const int c = __ffsll(static_cast<long long>(~used));
  if (v != lim.stall) st_relaxed(color + v, key.cword(kv, c));
  return c;
}

// GetColor for a larger vertex, by a whole warp.  Colours of predecessors in
// the window (base, base + kColorWin] are marked in a shared bitmap; if the
// window is full the smallest free colour lies above it and the predecessors
// are scanned again for the next window.
template <class Key>
__device__ int color_warp(int v, unsigned* bm, const long long* __restrict__ row_ptr,
                          const int* __restrict__ col, const Key& key, typename Key::W* color, JpCtl* ctl,
                          const JpLimits& lim, unsigned long long& spins) {
  const int lane = threadIdx.x & 31;
  const unsigned long long kv = key(v);
  const long long s = row_ptr[v], e = row_ptr[v + 1];
  for (int base = 0;; base += kColorWin) {
    bm[lane] = 0u;  // kColorWin / 32 == 32 words, one per lane
    __syncwarp();
    long long k = s + lane;
    bool more = k < e;
    while (__any_sync(kFull, more)) {
      if (more) {
        int pend[kPendCap];
        int np = 0;
        long long resume = -1;
        constexpr int U = 4;
        for (; k < e && resume < 0; k += 32 * U) {
          int w[U], c[U];
          typename Key::PG g[U];
          bool pred[U];
#pragma unroll
          for (int u = 0; u < U; ++u) w[u] = k + 32 * u < e ? __ldg(col + k + 32 * u) : -1;
#pragma unroll
          for (int u = 0; u < U; ++u) g[u] = w[u] >= 0 ? key.pgather(w[u], color) : typename Key::PG{};
#pragma unroll
          for (int u = 0; u < U; ++u) pred[u] = w[u] >= 0 && key.pred_g(g[u], w[u], kv, v);
#pragma unroll
          for (int u = 0; u < U; ++u) c[u] = pred[u] ? key.color_g(g[u], color, w[u]) : -1;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (!pred[u]) continue;
            if (c[u] == 0) {
              if (np == kPendCap) {
                if (resume < 0) resume = k + 32 * u;  // re-examined after the waits
                continue;
              }
              pend[np++] = w[u];
            } else if (resume < 0 && c[u] > base && c[u] <= base + kColorWin) {
              atomicOr(&bm[(c[u] - base - 1) >> 5], 1u << ((c[u] - base - 1) & 31));
            }
          }
        }
        for (int j = 0; j < np; ++j) {
          const int c = wait_color(color + pend[j], key.cmask(), ctl, lim, spins);
          if (c > base && c <= base + kColorWin)
            atomicOr(&bm[(c - base - 1) >> 5], 1u << ((c - base - 1) & 31));
        }
        more = resume >= 0;
        if (more) k = resume;
      }
    }
    __syncwarp();
    const unsigned freeb = ~bm[lane];
    const unsigned fm = __ballot_sync(kFull, freeb != 0u);
    __syncwarp();
    if (fm) {
      const int f = __ffs(fm) - 1;
      const unsigned fb = __shfl_sync(kFull, freeb, f);
      const int c = base + f * 32 + __ffs(fb);
      if (lane == 0 && v != lim.stall) st_relaxed(color + v, key.cword(kv, c));
      return c;
    }
  }
}

// Stage 3 (and the whole of gc_jp_color): colours the warp-path list
// big[0, nbig) and the lane-path list small[0, nsmall), taking vertices with
// the two counters cursors[0] and cursors[1].  nbig < 0 means: counts from
// ctl, small list right after the big one.  4 blocks per SM (up to 64
// registers) let the lane path keep 8 neighbour loads in flight: on R-MAT 24
// the bulk took 3.13 ms this way against 3.33 ms at 5 blocks with 4 loads
// (12 or 16 loads: 3.22 ms).
template <class Key>
__global__ void __launch_bounds__(kJpThreads, 4)
jp_color_kernel(JpCtl* ctl, unsigned long long* cursors, const long long* __restrict__ row_ptr,
                const int* __restrict__ col, Key key, const int* __restrict__ big, long long nbig,
                const int* __restrict__ small, long long nsmall, typename Key::W* color) {
  __shared__ unsigned s_bm[kJpWarps][kColorWin / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nbig < 0) {
    nbig = static_cast<long long>(ctl->nbig);
    nsmall = static_cast<long long>(ctl->nsmall);
    small = big + nbig;
  }
  bool big_done = nbig == 0, small_done = nsmall == 0;
  __shared__ JpLimits lim;  // in shared memory: no registers held for it
  if (threadIdx.x == 0) lim = JpLimits{ctl->wait_ns, ctl->stall};
  __syncthreads();
  const bool prefer_big = (warp & 3) != 0;  // 3/4 of the warps start on the warp path
  int local_max = 0;
  unsigned long long spins = 0;
  while (!(big_done && small_done)) {
    const bool take_big = !big_done && (prefer_big || small_done);
    if (take_big) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&cursors[0], 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= static_cast<unsigned long long>(nbig)) {
        big_done = true;
        continue;
      }
      const int c = color_warp(big[i], s_bm[warp], row_ptr, col, key, color, ctl, lim, spins);
      local_max = c > local_max ? c : local_max;
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&cursors[1], 32ull);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= static_cast<unsigned long long>(nsmall)) {
        small_done = true;
        continue;
      }
      const unsigned long long i = i0 + lane;
      if (i < static_cast<unsigned long long>(nsmall)) {
        const int c = color_lane(small[i], row_ptr, col, key, color, ctl, lim, spins);
        local_max = c > local_max ? c : local_max;
      }
      __syncwarp();
    }
  }
  local_max = warp_max(local_max);
  spins = warp_sum(spins);
  if (lane == 0) {
    atomicMax(&ctl->max_color, local_max);
    if (spins) atomicAdd(&ctl->spins, spins);
  }
}

__global__ void jp_init_kernel(JpCtl* ctl, unsigned long long wait_ns, int stall) {
  JpCtl c{};
  c.key_and = ~0ull;
  c.bstar = -1;
  c.wait_ns = wait_ns;
  c.stall = stall;
  *ctl = c;
}

// ---------------------------------------------------------------------------
// Exact order for an arbitrary priority array (gc_jp_color).
// ---------------------------------------------------------------------------
template <class Key>
__global__ void __launch_bounds__(256)
jp_keys_kernel(Key key, const long long* __restrict__ row_ptr, long long n,
               unsigned long long* __restrict__ keys, int* __restrict__ vals, JpCtl* ctl) {
  unsigned long long kor = 0, kand = ~0ull;
  for (long long i = gtid(); i < n; i += gstride()) {
    const int v = static_cast<int>(n - 1 - i);
    const unsigned long long sk = ~key(v);
    const bool big = row_ptr[v + 1] - row_ptr[v] > kSmallDeg;
    keys[i] = sk;
    vals[i] = static_cast<int>(static_cast<unsigned>(v) | (big ? kBigBit : 0u));
    kor |= sk;
    kand &= sk;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kor |= __shfl_xor_sync(kFull, kor, o);
    kand &= __shfl_xor_sync(kFull, kand, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&ctl->key_or, kor);
    atomicAnd(&ctl->key_and, kand);
  }
}

__global__ void jp_flags_kernel(const int* __restrict__ order, long long n, long long* flags,
                                JpCtl* ctl) {
  for (long long i = gtid(); i < n; i += gstride()) {
    const long long f = (static_cast<unsigned>(order[i]) & kBigBit) ? 1 : 0;
    flags[i] = f;
    if (i == n - 1) ctl->nbig = static_cast<unsigned long long>(f);
  }
}

// Stable partition of the sorted order: warp-path vertices first.
__global__ void jp_split_kernel(const int* __restrict__ order, const long long* __restrict__ pos,
                                long long n, int* __restrict__ plist, JpCtl* ctl) {
  const long long nbig = pos[n - 1] + static_cast<long long>(ctl->nbig);
  for (long long i = gtid(); i < n; i += gstride()) {
    const unsigned o = static_cast<unsigned>(order[i]);
    const int v = static_cast<int>(o & ~kBigBit);
    if (o & kBigBit)
      plist[pos[i]] = v;
    else
      plist[nbig + (i - pos[i])] = v;
  }
}

// Ordered path: where each batch starts in the rest of the order (sorted by
// batch), as positions in the warp-path list (pos) and the lane-path list
// (i - pos); -1 for batches with no vertex there.
__global__ void jpo_first_kernel(const int* __restrict__ order, long long n, const int* __restrict__ batch,
                                 int* __restrict__ first) {
  for (long long i = gtid(); i < n; i += gstride()) {
    const int b = batch[static_cast<unsigned>(order[i]) & ~kBigBit];
    if (i == 0 || batch[static_cast<unsigned>(order[i - 1]) & ~kBigBit] != b) first[b] = static_cast<int>(i);
  }
}

__global__ void jpo_bounds_kernel(const int* __restrict__ first, const long long* __restrict__ pos, int rounds,
                                  long long* __restrict__ bounds) {
  for (long long b = gtid(); b <= rounds; b += gstride()) {
    const int f = first[b];
    bounds[2 * b] = f < 0 ? -1 : pos[f];
    bounds[2 * b + 1] = f < 0 ? -1 : f - pos[f];
  }
}

__global__ void jp_count_kernel(const long long* __restrict__ pos, long long n, JpCtl* ctl) {
  const unsigned long long nbig = static_cast<unsigned long long>(pos[n - 1]) + ctl->nbig;
  ctl->nbig = nbig;
  ctl->nsmall = static_cast<unsigned long long>(n) - nbig;
}

__global__ void make_priority_kernel(const int* __restrict__ batch, long long n, unsigned long long seed,
                                     unsigned long long* __restrict__ key) {
  for (long long v = gtid(); v < n; v += gstride())
    key[v] = (static_cast<unsigned long long>(static_cast<unsigned>(batch[v])) << 32) |
             tie_hash(seed, static_cast<unsigned>(v));
}

// ---------------------------------------------------------------------------
// JP-ADG order: counting sort by bucket = (R - batch) << hb | top hb bits of
// ~rho_R, so ascending buckets are descending (batch, rho_R).  Counts are
// kept per degree class (warp path / lane path).
// ---------------------------------------------------------------------------
struct BucketPlan {
  int rounds;       // R = number of ADG rounds (batches 1..R)
  int hb;           // hash bits per batch
  long long B;      // buckets per class = R << hb
};

__device__ __forceinline__ long long bucket_of(int batch, unsigned h, const BucketPlan& bp) {
  const long long hi = static_cast<long long>(bp.rounds - batch) << bp.hb;
  return bp.hb == 0 ? hi : hi | static_cast<long long>((~h) >> (32 - bp.hb));
}

template <class Key>
__global__ void __launch_bounds__(256)
jpf_hist_kernel(Key key, const long long* __restrict__ row_ptr, long long n, BucketPlan bp,
                unsigned long long* __restrict__ cnt, typename Key::W* __restrict__ color, JpCtl* ctl) {
  bool isolated = false;
  for (long long v = gtid(); v < n; v += gstride()) {
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    if (deg == 0) {
      color[v] = static_cast<typename Key::W>(key.cword(key(static_cast<int>(v)), 1));  // isolated: colour 1
      isolated = true;
      continue;
    }
    color[v] = static_cast<typename Key::W>(key.cword(key(static_cast<int>(v)), 0));
    const long long b = bucket_of(key.bat(static_cast<int>(v)), key.tie(static_cast<int>(v)), bp);
    const long long cls = deg > kSmallDeg ? 0 : 1;
    atomicAdd(&cnt[cls * (bp.B + 1) + b], 1ull);
  }
  if (__any_sync(kFull, isolated) && (threadIdx.x & 31) == 0) atomicMax(&ctl->max_color, 1);
}

__global__ void jpf_total_kernel(const unsigned long long* __restrict__ cnt, long long B,
                                 unsigned long long* __restrict__ tot) {
  for (long long b = gtid(); b <= B; b += gstride())
    tot[b] = b < B ? cnt[b] + cnt[(B + 1) + b] : 0ull;
}

// Core = buckets [0, bstar]: the largest prefix of whole buckets holding at
// most `target` vertices.  off_* are exclusive scans with the total at [B].
__global__ void jpf_pick_kernel(const unsigned long long* __restrict__ off_tot, long long B,
                                unsigned long long target, JpCtl* ctl) {
  for (long long b = gtid(); b < B; b += gstride()) {
    const bool fits = off_tot[b + 1] <= target;
    const bool next_fits = b + 1 < B && off_tot[b + 2] <= target;
    if (fits && !next_fits) ctl->bstar = b;
  }
}

__global__ void jpf_bases_kernel(const unsigned long long* __restrict__ off_tot,
                                 const unsigned long long* __restrict__ off_cls, long long B,
                                 JpCtl* ctl) {
  const long long bs = ctl->bstar;
  const unsigned long long* off0 = off_cls;
  const unsigned long long* off1 = off_cls + (B + 1);
  const unsigned long long kc = off_tot[bs + 1];
  ctl->ncore = kc;
  ctl->base0 = off0[bs + 1];
  ctl->base1 = off1[bs + 1];
  ctl->nbig = off0[B] - off0[bs + 1];
  ctl->nsmall = off1[B] - off1[bs + 1];
}

// Class-list offsets at the first bucket of every batch group g = R - batch
// (g = 0..R, where g = R is the total): bounds[2g] = warp path, [2g+1] =
// lane path.  Read before the scatter advances the offsets.
__global__ void jpf_batch_bounds_kernel(const unsigned long long* __restrict__ off_cls, BucketPlan bp,
                                        unsigned long long* __restrict__ bounds) {
  for (long long g = gtid(); g <= bp.rounds; g += gstride()) {
    const long long b = g << bp.hb;
    bounds[2 * g] = off_cls[b];
    bounds[2 * g + 1] = off_cls[(bp.B + 1) + b];
  }
}

// Places every non-isolated vertex: core buckets into order[0, ncore), the
// rest into the warp-path list order[ncore, ncore + nbig) and the lane-path
// list after it.  Cursors are the exclusive scans, advanced atomically.
template <class Key>
__global__ void __launch_bounds__(256)
jpf_scatter_kernel(Key key, const long long* __restrict__ row_ptr, long long n, BucketPlan bp,
                   unsigned long long* cur_tot, unsigned long long* cur_cls, const JpCtl* ctl,
                   int* __restrict__ order) {
  const long long bs = ctl->bstar;
  const unsigned long long ncore = ctl->ncore, nbig = ctl->nbig;
  const unsigned long long base0 = ctl->base0, base1 = ctl->base1;
  for (long long v = gtid(); v < n; v += gstride()) {
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    if (deg == 0) continue;
    const long long b = bucket_of(key.bat(static_cast<int>(v)), key.tie(static_cast<int>(v)), bp);
    unsigned long long pos;
    if (b <= bs) {
      pos = atomicAdd(&cur_tot[b], 1ull);
    } else if (deg > kSmallDeg) {
      pos = ncore + (atomicAdd(&cur_cls[b], 1ull) - base0);
    } else {
      pos = ncore + nbig + (atomicAdd(&cur_cls[(bp.B + 1) + b], 1ull) - base1);
    }
    order[pos] = static_cast<int>(v);
  }
}

// Exact order inside each core bucket: by (rho_R, id) descending (all
// vertices of a bucket share their batch); then lid[v] = position of v in the
// core.  Buckets hold ~32 vertices on average, but one batch can hold most of
// a small graph: buckets of at most kSortSmall vertices (and, rarely, above
// kSortBig) get a per-thread insertion sort here, the others a shared-memory
// bitonic sort by one block each (jpf_core_sort_big_kernel).
constexpr int kSortSmall = 64;
constexpr int kSortBig = 16384;  // 128 KB of 64-bit sort values per block

template <class Key>
__global__ void jpf_core_sort_kernel(const unsigned long long* __restrict__ cur_tot, const JpCtl* ctl,
                                     Key key, int* __restrict__ order, int* __restrict__ lid) {
  const long long bs = ctl->bstar;
  for (long long b = gtid(); b <= bs; b += gstride()) {
    // after the scatter, cur_tot[b] is the end of bucket b
    const long long s = b == 0 ? 0 : static_cast<long long>(cur_tot[b - 1]);
    const long long e = static_cast<long long>(cur_tot[b]);
    if (e - s > kSortSmall && e - s <= kSortBig) continue;
    for (long long i = s + 1; i < e; ++i) {
      const int x = order[i];
      const unsigned long long kx = key(x);
      long long j = i - 1;
      while (j >= s) {
        const int y = order[j];
        if (precedes(key(y), y, kx, x)) break;
        order[j + 1] = y;
        --j;
      }
      order[j + 1] = x;
    }
    for (long long i = s; i < e; ++i) lid[order[i]] = static_cast<int>(i);
  }
}

// Core buckets of kSortSmall < size <= kSortBig vertices, each sorted by one
// block: a block checks 1024 buckets at once (one per thread), then sorts the
// large ones among them in turn: sort values (rho_R << 32 | id), padded with
// zeros to a power of two, bitonic sort descending in shared memory (a zero
// pad equals only vertex 0 with rho_R 0, which then takes the same place).
template <class Key>
__global__ void __launch_bounds__(1024)
jpf_core_sort_big_kernel(const unsigned long long* __restrict__ cur_tot, const JpCtl* ctl, Key key,
                         int* __restrict__ order, int* __restrict__ lid) {
  extern __shared__ unsigned long long s_v[];
  __shared__ long long s_big[1024];  // large buckets among this block's 1024
  __shared__ int s_nbig;
  const long long bs = ctl->bstar;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base <= bs;
       base += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    const long long b = base + threadIdx.x;
    if (b <= bs) {
      const long long k = static_cast<long long>(cur_tot[b]) - (b == 0 ? 0 : static_cast<long long>(cur_tot[b - 1]));
      if (k > kSortSmall && k <= kSortBig) s_big[atomicAdd(&s_nbig, 1)] = b;
    }
    __syncthreads();
    const int nbig = s_nbig;
    for (int t = 0; t < nbig; ++t) {
      const long long bb = s_big[t];
      const long long s = bb == 0 ? 0 : static_cast<long long>(cur_tot[bb - 1]);
      const int k = static_cast<int>(static_cast<long long>(cur_tot[bb]) - s);
      int p2 = 1;
      while (p2 < k) p2 <<= 1;
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        unsigned long long u = 0;
        if (i < k) {
          const int x = order[s + i];
          u = (static_cast<unsigned long long>(key.tie(x)) << 32) | static_cast<unsigned>(x);
        }
        s_v[i] = u;
      }
      __syncthreads();
      for (int size = 2; size <= p2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          for (int i = threadIdx.x; i < (p2 >> 1); i += blockDim.x) {
            const int lo = 2 * i - (i & (stride - 1));
            const int hi = lo + stride;
            const bool desc = (lo & size) == 0;
            const unsigned long long a = s_v[lo], c = s_v[hi];
            if (desc ? a < c : a > c) {
              s_v[lo] = c;
              s_v[hi] = a;
            }
          }
          __syncthreads();
        }
      }
      for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const int x = static_cast<int>(static_cast<unsigned>(s_v[i] & 0xffffffffull));
        order[s + i] = x;
        lid[x] = static_cast<int>(s + i);
      }
      __syncthreads();
    }
  }
}

// Per core vertex: capacity of its predecessor list (degree at removal) and
// the number of UPDATE-style edge chunks of its adjacency.
__global__ void jpf_core_prep_kernel(const int* __restrict__ order, const int* __restrict__ D,
                                     const long long* __restrict__ row_ptr, JpCtl* ctl,
                                     long long* __restrict__ cap, long long* __restrict__ ntask) {
  const long long kc = static_cast<long long>(ctl->ncore);
  unsigned long long degsum = 0;
  for (long long i = gtid(); i <= kc; i += gstride()) {
    if (i == kc) {
      cap[i] = 0;
      ntask[i] = 0;
      continue;
    }
    const int v = order[i];
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    cap[i] = D ? D[v] : (deg < i ? deg : i);  // without D: a core vertex has at most i predecessors
    ntask[i] = (deg + kChunk - 1) / kChunk;
    degsum += static_cast<unsigned long long>(deg);
  }
  degsum = warp_sum(degsum);
  if ((threadIdx.x & 31) == 0 && degsum) atomicAdd(&ctl->core_deg, degsum);
}

__global__ void jpf_core_tasks_kernel(const int* __restrict__ order, const long long* __restrict__ row_ptr,
                                      const long long* __restrict__ toff, const JpCtl* ctl,
                                      int* __restrict__ task_i, long long* __restrict__ task_start,
                                      int* __restrict__ task_len) {
  // a warp per core vertex: a hub's row of 10^5 entries is thousands of tasks
  const long long kc = static_cast<long long>(ctl->ncore);
  const int lane = threadIdx.x & 31;
  for (long long i = gtid() >> 5; i < kc; i += gstride() >> 5) {
    const int v = order[i];
    const long long rs = row_ptr[v], re = row_ptr[v + 1];
    const long long t0 = toff[i];
    for (long long c = lane; rs + c * kChunk < re; c += 32) {
      const long long st = rs + c * kChunk;
      task_i[t0 + c] = static_cast<int>(i);
      task_start[t0 + c] = st;
      task_len[t0 + c] = static_cast<int>(re - st < kChunk ? re - st : kChunk);
    }
  }
}

// Predecessor lists of the core in core-local ids, edges spread over the
// lanes of each warp across 32 tasks at a time (as in ADG's UPDATE).
// Core membership bitmap (n bits): set for the core vertices.
__global__ void jpf_core_bits_kernel(const int* __restrict__ order, const JpCtl* ctl, unsigned* __restrict__ cbits) {
  const long long kc = static_cast<long long>(ctl->ncore);
  for (long long i = gtid(); i < kc; i += gstride()) {
    const int v = order[i];
    atomicOr(&cbits[v >> 5], 1u << (v & 31));
  }
}

// Predecessor lists of the core vertices.  Every predecessor of a core vertex
// is in the core, and the core is in exact priority order, so w precedes the
// core vertex i exactly when w is in the core and lid[w] < i: the sweep tests
// core membership on a bitmap (n bits, resident in L2) and reads lid[w] only
// for core neighbours, instead of gathering every neighbour's priority.
__global__ void __launch_bounds__(256)
jpf_core_preds_kernel(const int* __restrict__ col, const unsigned* __restrict__ cbits,
                      const int* __restrict__ lid, const long long* __restrict__ toff,
                      const long long* __restrict__ poff, const JpCtl* ctl,
                      const int* __restrict__ task_i, const long long* __restrict__ task_start,
                      const int* __restrict__ task_len, int* __restrict__ pcnt, int* __restrict__ preds) {
  const long long ntasks = toff[ctl->ncore];
  const int lane = threadIdx.x & 31;
  const long long gwarp = gtid() >> 5, nwarps = gstride() >> 5;
  for (long long tile = gwarp; tile * 32 < ntasks; tile += nwarps) {
    const long long t = tile * 32 + lane;
    long long st = 0;
    int len = 0, ci = 0;
    if (t < ntasks) {
      st = task_start[t];
      len = task_len[t];
      ci = task_i[t];
    }
    // 4 edges per lane and step: 36 registers (60 at 8), and 0.67 instead
    // of 0.83 ms on R-MAT 24
    sweep_tile<4>(
        st, len, ci, col, [&](int w, int) { return static_cast<int>((__ldg(cbits + (w >> 5)) >> (w & 31)) & 1u); },
        [&](int w, int i, int in_core) {
          const int lw = in_core ? __ldg(lid + w) : 0;
          const bool pred = in_core && lw < i;
          // one atomic per core vertex among the lanes of this step (edges of
          // one task sit in consecutive lanes)
          const unsigned act = __activemask();
          const unsigned pm = __ballot_sync(act, pred);
          if (pred) {
            const unsigned grp = __match_any_sync(pm, i);
            const int leader = __ffs(grp) - 1;
            int base = 0;
            if ((threadIdx.x & 31) == leader) base = atomicAdd(&pcnt[i], __popc(grp));
            base = __shfl_sync(grp, base, leader);
            preds[poff[i] + base + __popc(grp & lanemask_lt())] = lw;
          }
        });
  }
}

// Exact predecessor counts -> int64 array for the offset scan.
__global__ void jpf_counts_kernel(const int* __restrict__ pcnt, const JpCtl* ctl, long long* __restrict__ out) {
  const long long kc = static_cast<long long>(ctl->ncore);
  for (long long i = gtid(); i <= kc; i += gstride()) out[i] = i < kc ? pcnt[i] : 0;
}

// Compacts the predecessor lists (written at capacity-sized slots) into one
// dense 16-bit stream in core order: list i at [qoff[i], qoff[i+1]).
__global__ void jpf_compact_kernel(const int* __restrict__ preds, const long long* __restrict__ poff,
                                   const long long* __restrict__ qoff, const JpCtl* ctl,
                                   unsigned short* __restrict__ cpreds) {
  const long long kc = static_cast<long long>(ctl->ncore);
  const int lane = threadIdx.x & 31;
  for (long long i = gtid() >> 5; i < kc; i += gstride() >> 5) {
    const long long src = poff[i], dst = qoff[i], cnt = qoff[i + 1] - qoff[i];
    for (long long k = lane; k < cnt; k += 32) cpreds[dst + k] = static_cast<unsigned short>(preds[src + k]);
  }
}

// Colours the core with one thread-block cluster of C CTAs (C <= 16, one per
// SM) of W warps each.  Core vertex i belongs to CTA (i / W) mod C, warp
// i mod W, so runs of W consecutive vertices (where many dependency steps
// fall) share a CTA; every warp takes its vertices in increasing order.  W is
// small (12 by default): warps that wait poll, and on a crowded SM their polls
// take the issue slots of the warps on the critical path.  Each CTA holds a full
// copy of the core's colours (16-bit, so a core of at most 32768 vertices,
// using at most 32768 colours) in its shared memory: a warp that colours
// vertex i stores the colour into all C copies (lane r into CTA r, through
// distributed shared memory), and waits for a predecessor by polling its own
// CTA's copy.  A warp reads its vertex's predecessor list (the compact 16-bit
// stream, core order) from global memory in 16-byte groups (the 8 colours of
// a group are loaded together), marks the colours already known and sets the
// others aside (up to kDeferLane per lane, in shared memory) without waiting,
// so that the scan never stalls behind a predecessor that is still being
// coloured; then it sweeps the set-aside ones, marking those coloured
// meanwhile, until one is left in the warp.  The two smallest free colours
// c1 < c2 are known by then, so the colour is (c1 if the last one's colour
// differs from c1, else c2) and is stored the moment the last one lands.
// Predecessors
// precede their successors in the exact core order and every CTA of a
// cluster is resident, so the warp holding the earliest unfinished vertex
// always finds all of its predecessors coloured: the cluster makes progress
// until every vertex is done.
//
// Used colours are marked in per-lane bitmaps (word q of lane l at q*32 + l,
// so a warp's marks never collide in a bank and need no atomics) while the
// list is scanned, then OR-ed across lanes (a rotated read) into the warp's
// merged words BEFORE it waits on the set-aside predecessors: those mark the
// merged words directly as they arrive, so once the last one lands only one
// word per lane is read to find the smallest free colour -- the 32-way OR is
// off the dependency chain.  A pass covers a 512-colour window and only
// ceil((|pred|+1)/32) words of it can hold the answer.
constexpr int kBitWords = 16;       // 512-colour window per pass
constexpr int kDeferLane = 40;      // predecessors a lane sets aside per vertex
constexpr int kCoreClusterMax = 16;
// shared memory of one core warp: its bitmaps, merged words and set-aside
// predecessors
constexpr size_t kCoreWarpBytes = kBitWords * 32 * sizeof(unsigned) + kBitWords * sizeof(unsigned) +
                                  kDeferLane * 32 * sizeof(unsigned short);

size_t core_smem_bytes(int warps, long long kc) {
  return static_cast<size_t>(warps) * kCoreWarpBytes + static_cast<size_t>(kc) * sizeof(unsigned short);
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster arrives; shared-memory writes
// before it (local or remote) are visible to every thread after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of this CTA's shared variable `p` in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_map(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_u16(unsigned addr, unsigned short v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}

template <class W>
__global__ void __launch_bounds__(kCoreThreads, 1)
jpf_core_solve_kernel(const int* __restrict__ order, const long long* __restrict__ qoff,
                      const unsigned short* __restrict__ stream, JpCtl* ctl, W* color) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int nwc = blockDim.x >> 5;  // warps per CTA
  unsigned* s_bits = reinterpret_cast<unsigned*>(s_dyn);  // [warp][word][lane]
  unsigned* s_merged = s_bits + nwc * kBitWords * 32;      // [warp][word]
  unsigned short* s_def = reinterpret_cast<unsigned short*>(s_merged + nwc * kBitWords);  // [warp][slot][lane]
  unsigned short* s_col = s_def + nwc * kDeferLane * 32;
  const int kc = static_cast<int>(ctl->ncore);
  const int rank = static_cast<int>(cluster_rank()), nctas = static_cast<int>(cluster_ctas());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kc; i += blockDim.x) s_col[i] = 0;
  __syncwarp();
  cluster_sync();  // every copy is cleared before any colour lands in it

  volatile unsigned short* vcol = s_col;
  unsigned* bits = s_bits + warp * kBitWords * 32;
  unsigned* merged = s_merged + warp * kBitWords;
  unsigned short* def = s_def + warp * kDeferLane * 32 + lane;
  const unsigned col_r = lane < nctas ? cluster_map(s_col, lane) : 0u;  // copy in CTA `lane`
  const uint4* groups = reinterpret_cast<const uint4*>(stream);
  // the wait bound (counted from the kernel's start) and the injected stall,
  // kept in shared memory: the inner loops are sensitive to every register
  __shared__ unsigned long long s_wait_ns;
  __shared__ int s_stall;
  if (threadIdx.x == 0) {
    s_wait_ns = ctl->wait_ns;
    s_stall = ctl->stall;
  }
  __syncthreads();
  const unsigned long long t0 = global_ns();
  bool timed_out = false;
  auto expired = [&]() { return timed_out || ld_relaxed(&ctl->err) != 0 || global_ns() - t0 > s_wait_ns; };
  int local_max = 0;
  for (int i = nwc * rank + warp; i < kc; i += nwc * nctas) {
    // an injected fault: this vertex never publishes its colour
    const bool stalled = s_stall >= 0 && __ldg(order + i) == s_stall;
    const long long a = qoff[i], b = qoff[i + 1];
    const int np = static_cast<int>(b - a);
    const int nw = np / 32 + 1 < kBitWords ? np / 32 + 1 : kBitWords;
    int c = 1;
    for (int base = 0; !timed_out; base += 32 * nw) {
      for (int q = 0; q < nw; ++q) bits[q * 32 + lane] = 0u;
      int nd = 0;
      bool late = false;  // after the merge: marks go to the merged words
      auto put = [&](int cj) {
        const int x = cj - base - 1;
        if (x >= 0 && x < 32 * nw) {
          if (!late)
            bits[(x >> 5) * 32 + lane] |= 1u << (x & 31);
          else
            atomicOr(&merged[x >> 5], 1u << (x & 31));
        }
      };
      // marks the set-aside predecessors coloured by now and keeps the rest
      auto sweep = [&]() {
        int k = 0;
        for (int d = 0; d < nd; ++d) {
          const int j = def[32 * d];
          const int cj = vcol[j];
          if (cj != 0)
            put(cj);
          else
            def[32 * k++] = static_cast<unsigned short>(j);
        }
        nd = k;
      };
      // sweeps until at most `keep` predecessors are left (bounded); no
      // sleep between sweeps: with 8 warps per SM the polls cost the
      // critical path little, while a sleeping warp notices its last
      // predecessor late (a 32 ns sleep after 64 sweeps cost R-MAT 24's core
      // 2.63 against 2.11 ms)
      auto drain = [&](int keep) {
        for (unsigned it = 0; nd > keep; ++it) {
          sweep();
          if (nd <= keep) break;
          if ((it & 255u) == 255u && expired()) {
            timed_out = true;
            nd = 0;
          }
        }
      };
      // the 8 ids of a 16-byte group whose positions are in the list (bit e
      // of `valid`): their colours are read first, all 8 loads in flight,
      // then marked or set aside
      auto take8 = [&](const uint4& v, unsigned valid) {
        const unsigned wv[4] = {v.x, v.y, v.z, v.w};
        int id[8], cj[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          id[e] = static_cast<int>((wv[e >> 1] >> (16 * (e & 1))) & 0xffffu);
          cj[e] = ((valid >> e) & 1u) ? static_cast<int>(vcol[id[e]]) : -1;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          if (cj[e] > 0) {
            put(cj[e]);
          } else if (cj[e] == 0) {
            if (nd == kDeferLane) drain(kDeferLane - 1);
            if (nd < kDeferLane) def[32 * nd++] = static_cast<unsigned short>(id[e]);
          }
        }
      };
      auto mask8 = [&](long long p) -> unsigned {
        const long long lo = a - p > 0 ? a - p : 0, hi = b - p < 8 ? b - p : 8;
        return hi > lo ? ((1u << hi) - 1u) & ~((1u << lo) - 1u) : 0u;
      };
      // positions [a, b) of the stream, 8 per 16-byte group, two groups per
      // lane in flight
      for (long long g = a / 8 + lane; g * 8 < b; g += 64) {
        const bool has2 = (g + 32) * 8 < b;
        const uint4 v0 = __ldg(groups + g);
        const uint4 v1 = has2 ? __ldg(groups + g + 32) : make_uint4(0u, 0u, 0u, 0u);
        take8(v0, mask8(g * 8));
        if (has2) take8(v1, mask8((g + 32) * 8));
      }
      __syncwarp();
      // lane q < nw ORs word q over all lanes (rotated so no bank repeats)
      // into the merged words, while set-aside predecessors may still be
      // uncoloured
      if (lane < nw) {
        unsigned word = 0u;
        for (int l = 0; l < 32; ++l) word |= bits[lane * 32 + ((lane + l) & 31)];
        merged[lane] = word;
      }
      __syncwarp();
      late = true;
      // Wait until at most one predecessor is left in the whole warp (each
      // lane first down to one of its own).  That one is usually the
      // previous vertex of the dependency chain: its colour cj decides
      // between the two smallest colours c1 < c2 still free, c = (cj == c1 ?
      // c2 : c1), so both are found before it lands and, once it does, the
      // colour is stored at once.
      drain(1);
      __syncwarp();
      unsigned rem = __ballot_sync(kFull, nd > 0);
      for (unsigned it = 0; __popc(rem) > 1; ++it) {
        if (nd > 0) sweep();
        rem = __ballot_sync(kFull, nd > 0);
        if ((it & 255u) == 255u && __popc(rem) > 1 && __any_sync(kFull, expired())) {
          timed_out = true;
          nd = 0;
          break;
        }
      }
      // a wait that ran out on any lane ends this warp's colouring: agree on
      // it before any warp-wide step, so that every lane leaves together and
      // no collective below or in a later vertex runs with lanes missing
      if (__any_sync(kFull, timed_out)) {
        timed_out = true;
        break;
      }
      if (rem != 0u) {
        __syncwarp();  // the other lanes' late marks are in the merged words
        const unsigned fb0 = lane < nw ? ~merged[lane] : 0u;
        const unsigned fm0 = __ballot_sync(kFull, fb0 != 0u);
        int c1 = 0, c2 = 0;
        if (fm0) {
          const int f1 = __ffs(fm0) - 1;
          const unsigned b1 = __shfl_sync(kFull, fb0, f1);
          c1 = base + f1 * 32 + __ffs(b1);
          const unsigned b1r = b1 & (b1 - 1u);
          const unsigned fm1 = fm0 & ~(1u << f1);
          const int f2 = fm1 ? __ffs(fm1) - 1 : 0;
          const unsigned b2 = __shfl_sync(kFull, fb0, f2);
          if (b1r)
            c2 = base + f1 * 32 + __ffs(b1r);
          else if (fm1)
            c2 = base + f2 * 32 + __ffs(b2);
        }
        if (c2 != 0) {  // both inside this pass's window
          const int j = __shfl_sync(kFull, static_cast<int>(def[0]), __ffs(rem) - 1);
          unsigned got = 0u;
          int cj = 0;
          for (unsigned it = 0;; ++it) {
            cj = vcol[j];
            got = __ballot_sync(kFull, cj != 0);
            if (got) break;
            if ((it & 255u) == 255u && __any_sync(kFull, expired())) {
              timed_out = true;
              break;
            }
          }
          nd = 0;
          if (timed_out) break;
          cj = __shfl_sync(kFull, cj, __ffs(got) - 1);
          c = cj == c1 ? c2 : c1;
          break;
        }
      }
      drain(0);
      __syncwarp();
      if (__any_sync(kFull, timed_out)) {
        timed_out = true;
        break;
      }
      const unsigned freeb = lane < nw ? ~merged[lane] : 0u;
      const unsigned fm = __ballot_sync(kFull, freeb != 0u);
      __syncwarp();
      if (fm) {
        const int f = __ffs(fm) - 1;
        const unsigned fb = __shfl_sync(kFull, freeb, f);
        c = base + f * 32 + __ffs(fb);
        break;
      }
    }
    if (lane < nctas && !stalled) st_cluster_u16(col_r + 2u * static_cast<unsigned>(i), static_cast<unsigned short>(c));
    local_max = c > local_max ? c : local_max;
  }
  local_max = warp_max(local_max);
  if (lane == 0) atomicMax(&ctl->max_color, local_max);
  if (__any_sync(kFull, timed_out) && lane == 0) atomicExch(&ctl->err, kDevTimeout);
  __syncwarp();
  cluster_sync();  // all colours have landed in every copy; no remote store is outstanding
  for (int t = threadIdx.x;; t += blockDim.x) {  // this CTA's vertices, increasing
    const int i = nwc * (rank + nctas * (t / nwc)) + t % nwc;
    if (i >= kc) break;
    color[order[i]] = static_cast<W>(color[order[i]] | s_col[i]);  // the word holds 0 or the batch bits
  }
}

// Shape of the core cluster: warps per CTA (gc_options.core_warps, default
// kCoreWarpsDefault) and the largest cluster (16, 8, ..., 1 CTAs) the device
// can place with the core's largest shared-memory footprint;
// gc_options.core_cluster may ask for fewer CTAs.
cudaError_t core_cluster_size(gc_context* ctx, int* out) {
  if (ctx->core_cluster > 0) {
    *out = ctx->core_cluster;
    return cudaSuccess;
  }
  const int warps = ctx->opt.core_warps >= 1 && ctx->opt.core_warps <= kCoreWarps ? ctx->opt.core_warps
                                                                                  : kCoreWarpsDefault;
  ctx->core_warps = warps;
  const size_t smem_max = core_smem_bytes(warps, kCoreMax);
  cudaError_t e = cudaSuccess;
  for (const void* k : {reinterpret_cast<const void*>(jpf_core_solve_kernel<int>),
                        reinterpret_cast<const void*>(jpf_core_solve_kernel<unsigned short>)}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_max));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  int limit = kCoreClusterMax;
  if (ctx->opt.core_cluster >= 1 && ctx->opt.core_cluster < limit) limit = ctx->opt.core_cluster;
  int best = 1;
  for (int cs = 1; cs <= limit; cs *= 2) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem_max;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, jpf_core_solve_kernel<int>, &cfg) != cudaSuccess || ncl < 1) {
      cudaGetLastError();  // clear the query's error; keep the last size that fits
      break;
    }
    best = cs;
  }
  ctx->core_cluster = best;
  *out = best;
  return cudaSuccess;
}

template <class Key>
cudaError_t launch_bulk(gc_context* ctx, JpCtl* ctl, unsigned long long* cursors, const long long* row_ptr,
                        const int* col, const Key& key, const int* big, long long nbig, const int* small,
                        long long nsmall, typename Key::W* color, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jp_color_kernel<Key>, kJpThreads, 0);
  if (e != cudaSuccess) return e;
  if (ctx->opt.bulk_blocks_per_sm > 0 && ctx->opt.bulk_blocks_per_sm < per_sm) per_sm = ctx->opt.bulk_blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  jp_color_kernel<Key><<<ctx->num_sms * per_sm, kJpThreads, 0, s>>>(ctl, cursors, row_ptr, col, key, big, nbig,
                                                                   small, nsmall, color);
  ++g_launches;
  return cudaGetLastError();
}

gc_status finish_jp(gc_context* ctx, JpCtl* ctl, int* num_colors_out, cudaStream_t s) {
  JpCtl* pin = static_cast<JpCtl*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, ctl, sizeof(JpCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  JpCtl h;
  memcpy(&h, pin, sizeof(h));
  ctx->stats.jp_spins = static_cast<int64_t>(h.spins);
  ctx->stats.core_vertices = static_cast<int64_t>(h.ncore);
  ctx->stats.core_preds = h.core_preds;
  ctx->stats.core_degree_sum = static_cast<int64_t>(h.core_deg);
  if (h.err != kDevOk) return GC_ERR_TIMEOUT;
  ctx->stats.num_colors = h.max_color;
  if (num_colors_out) *num_colors_out = h.max_color;
  return GC_OK;
}

BucketPlan make_plan(long long n, int rounds) {
  BucketPlan bp;
  bp.rounds = rounds < 1 ? 1 : rounds;
  // about 32 vertices per bucket on average, at most 2^22 buckets per class
  // and 20 hash bits; with n < 2^31 the expected bucket then holds at most a
  // few hundred vertices, far fewer than a list has workers
  int hb = 0;
  while (hb < 20 && (static_cast<long long>(bp.rounds) << (hb + 1)) <= (1ll << 22) &&
         (static_cast<long long>(bp.rounds) << (hb + 1)) * 32 <= n)
    ++hb;
  bp.hb = hb;
  bp.B = static_cast<long long>(bp.rounds) << hb;
  return bp;
}

// The JP core stage on the first kc vertices of `order` (plain vertex ids in
// exact priority order, with ctl->ncore == kc and lid[order[i]] == i):
// predecessor lists of the core, compacted to 16-bit core-local ids, then the
// core cluster (jpf_core_solve_kernel).  A core vertex's list is sized by
// D[v] (its degree at removal, from ADG) or, without D, by min(deg(v), i).
struct CoreBufs {
  int* lid;
  unsigned* cbits;
  long long* cap;
  long long* toff;
  int* pcnt;
  int* task_i;
  long long* task_start;
  int* task_len;
  long long* temp;  // at least scan_temp_elems(kCoreMax + 1) elements
};

template <class W>
gc_status run_core(gc_context* ctx, const gc_csr* g, const int* order, const int* D, long long kc, JpCtl* ctl,
                   const CoreBufs& cb, W* color, cudaStream_t s) {
  const long long n = g->n;
  const long long* rp = row_ptr_of(g);
  const int blocks = ctx->num_sms * 8;
    jpf_core_prep_kernel<<<blocks, 256, 0, s>>>(order, D, rp, ctl, cb.cap, cb.toff);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(exclusive_scan_i64(cb.cap, cb.cap, kc + 1, cb.temp, s));
    GC_TRY_CUDA(exclusive_scan_i64(cb.toff, cb.toff, kc + 1, cb.temp, s));
    long long* pin_ll = reinterpret_cast<long long*>(ctx->pinned);
    GC_TRY_CUDA(cudaMemcpyAsync(pin_ll, cb.cap + kc, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    const long long npred_cap = pin_ll[0] > 0 ? pin_ll[0] : 1;
    // aux: predecessor ids at capacity-sized slots (int32), then the dense
    // 16-bit stream
    const size_t pbytes = (static_cast<size_t>(npred_cap) * sizeof(int) + 255) & ~size_t(255);
    // (the 256 spare bytes cover the last 16-byte group a core warp reads)
    GC_TRY(ctx->reserve_aux(pbytes + static_cast<size_t>(npred_cap) * sizeof(unsigned short) + 256));
    int* preds = static_cast<int*>(ctx->aux);
    unsigned short* cpreds = reinterpret_cast<unsigned short*>(static_cast<char*>(ctx->aux) + pbytes);
    GC_TRY_CUDA(cudaMemsetAsync(cb.pcnt, 0, sizeof(int) * (kc + 1), s));
    jpf_core_tasks_kernel<<<blocks, 256, 0, s>>>(order, rp, cb.toff, ctl, cb.task_i, cb.task_start, cb.task_len);
    ++g_launches;
    ctx->timer_begin(gc_context::kTCorePreds, s);
    GC_TRY_CUDA(cudaMemsetAsync(cb.cbits, 0, sizeof(unsigned) * static_cast<size_t>((n + 31) / 32), s));
    jpf_core_bits_kernel<<<blocks, 256, 0, s>>>(order, ctl, cb.cbits);
    ++g_launches;
    jpf_core_preds_kernel<<<resident_grid(jpf_core_preds_kernel, 256, ctx->num_sms), 256, 0, s>>>(
        g->col_idx, cb.cbits, cb.lid, cb.toff, cb.cap, ctl, cb.task_i, cb.task_start, cb.task_len, cb.pcnt, preds);
    ++g_launches;
    ctx->timer_end(s);
    long long* qoff = cb.toff;  // task offsets are dead now
    jpf_counts_kernel<<<blocks, 256, 0, s>>>(cb.pcnt, ctl, qoff);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(exclusive_scan_i64(qoff, qoff, kc + 1, cb.temp, s));
    GC_TRY_CUDA(cudaMemcpyAsync(&ctl->core_preds, qoff + kc, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    jpf_compact_kernel<<<blocks, 256, 0, s>>>(preds, cb.cap, qoff, ctl, cpreds);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    int ncta = 1;
    GC_TRY_CUDA(core_cluster_size(ctx, &ncta));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(32 * ctx->core_warps);
    cfg.dynamicSmemBytes = core_smem_bytes(ctx->core_warps, kc);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ctx->stats.core_ctas = ncta;
    ctx->timer_begin(gc_context::kTCoreSolve, s);
    GC_TRY_CUDA(cudaLaunchKernelEx(&cfg, jpf_core_solve_kernel<W>, static_cast<const int*>(order),
                                   static_cast<const long long*>(qoff), static_cast<const unsigned short*>(cpreds),
                                   ctl, color));
    ++g_launches;
    ctx->timer_end(s);
    GC_TRY_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// gc_jp_color: exact radix-sorted order, bulk stage on every vertex.
// ---------------------------------------------------------------------------
size_t jp_scratch_bytes(long long n, long long nnz) {
  const size_t hist = sort_hist_elems(n);
  const size_t tmp = scan_temp_elems(static_cast<long long>(hist));
  const size_t tmp2 = scan_temp_elems(n);
  const size_t tmp3 = scan_temp_elems(kCoreMax + 1);
  const size_t t = tmp > tmp2 ? tmp : tmp2;
  const size_t kc = static_cast<size_t>(kCoreMax) + 1;
  const size_t ntask = kc + static_cast<size_t>(nnz / kChunk) + 1;
  return 2 * (static_cast<size_t>(n) * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) + hist * 8 +
         ((t > tmp3 ? t : tmp3) + 1) * 8 +
         // core stage: corder, lid, cbits, cap, toff, pcnt, tasks
         (kc * 4 + 256) + (static_cast<size_t>(n) * 4 + 256) + (static_cast<size_t>((n + 31) / 32) * 4 + 256) +
         2 * (kc * 8 + 256) + (kc * 4 + 256) + ntask * 16 + 3 * 256 + 4096;
}

namespace {
// KeyState: colour words start as batch << 24 (colour 0) and lose the batch
// bits at the end.
__global__ void state_init_kernel(const int* __restrict__ batch, long long n, int* __restrict__ color) {
  for (long long v = gtid(); v < n; v += gstride())
    color[v] = static_cast<int>(static_cast<unsigned>(batch[v]) << 24);
}

__global__ void state_strip_kernel(long long n, int* __restrict__ color) {
  for (long long v = gtid(); v < n; v += gstride()) color[v] &= 0xffffff;
}

// Core of the generic path: the first kc entries of the sorted order (vertex
// ids with the warp-path flag) as plain ids, and their core positions.
__global__ void jp_core_from_sorted_kernel(const int* __restrict__ order, long long kc, int* __restrict__ corder,
                                           int* __restrict__ lid, JpCtl* ctl) {
  for (long long i = gtid(); i < kc; i += gstride()) {
    const int v = static_cast<int>(static_cast<unsigned>(order[i]) & ~kBigBit);
    corder[i] = v;
    lid[v] = static_cast<int>(i);
  }
  if (gtid() == 0) ctl->ncore = static_cast<unsigned long long>(kc);
}
}  // namespace

// Exact order of `key` (radix sort), the top of it by the core cluster, the
// rest by one bulk launch.  With `state` (KeyStateD), colour words start as
// batch << 24 (state_batch) and lose those bits at the end.
template <class Key>
gc_status jp_run_exact(gc_context* ctx, Arena a, const gc_csr* g, const Key& key, const int* state_batch,
                       const int* core_D, int* color, int* num_colors_out, cudaStream_t s, int rounds = 0) {
  const long long n = g->n;
  if (num_colors_out) *num_colors_out = 0;
  ctx->stats.num_colors = 0;
  ctx->stats.jp_spins = 0;
  if (n == 0) return GC_OK;
  JpCtl* ctl = a.take<JpCtl>(1);
  SortBufs sb;
  sb.keys[0] = a.take<unsigned long long>(n);
  sb.keys[1] = a.take<unsigned long long>(n);
  sb.vals[0] = a.take<int>(n);
  sb.vals[1] = a.take<int>(n);
  sb.hist = a.take<long long>(sort_hist_elems(n));
  const size_t tmp = scan_temp_elems(static_cast<long long>(sort_hist_elems(n)));
  const size_t tmp2 = scan_temp_elems(n);
  const size_t tmp3 = scan_temp_elems(kCoreMax + 1);
  const size_t tt = tmp > tmp2 ? tmp : tmp2;
  sb.temp = a.take<long long>((tt > tmp3 ? tt : tmp3) + 1);
  // the core stage: the top of the exact order, coloured by the core cluster
  const long long kc = ctx->core_target < 0 ? 0 : (ctx->core_target > kCoreMax ? kCoreMax : (ctx->core_target > n ? n : ctx->core_target));
  const long long ntask_cap = kCoreMax + g->nnz / kChunk + 1;
  int* corder = a.take<int>(kCoreMax + 1);
  CoreBufs cb{a.take<int>(n), a.take<unsigned>((n + 31) / 32), a.take<long long>(kCoreMax + 1),
              a.take<long long>(kCoreMax + 1), a.take<int>(kCoreMax + 1), a.take<int>(ntask_cap),
              a.take<long long>(ntask_cap), a.take<int>(ntask_cap), sb.temp};
  if (!ctl || !sb.keys[0] || !sb.keys[1] || !sb.vals[0] || !sb.vals[1] || !sb.hist || !sb.temp || !corder ||
      !cb.lid || !cb.cbits || !cb.cap || !cb.toff || !cb.pcnt || !cb.task_i || !cb.task_start || !cb.task_len)
    return GC_ERR_OOM;
  const long long* rp = row_ptr_of(g);
  const int blocks = ctx->num_sms * 8;
  jp_init_kernel<<<1, 1, 0, s>>>(ctl, ctx->wait_ns, ctx->stall_vertex);
  ++g_launches;
  if (state_batch) {
    state_init_kernel<<<blocks, 256, 0, s>>>(state_batch, n, color);
    ++g_launches;
  }
  jp_keys_kernel<<<blocks, 256, 0, s>>>(key, rp, n, sb.keys[0], sb.vals[0], ctl);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  unsigned long long* pin = static_cast<unsigned long long*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, &ctl->key_or, 2 * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  const unsigned long long diff = pin[0] ^ pin[1];
  unsigned mask = 0;
  for (int d = 0; d < 8; ++d)
    if ((diff >> (8 * d)) & 255ull) mask |= 1u << d;
  cudaError_t err;
  const int res = radix_sort_pairs(sb, n, mask, s, &err);
  GC_TRY_CUDA(err);
  const int* order = sb.vals[res];
  long long* pos = reinterpret_cast<long long*>(sb.keys[res ^ 1]);
  int* plist = sb.vals[res ^ 1];
  if (!state_batch) GC_TRY_CUDA(cudaMemsetAsync(color, 0, sizeof(int) * n, s));
  if (kc > 0) {  // the top kc vertices: exact order known, coloured by the core cluster
    jp_core_from_sorted_kernel<<<blocks, 256, 0, s>>>(order, kc, corder, cb.lid, ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY(run_core(ctx, g, corder, core_D, kc, ctl, cb, color, s));
  }
  // the rest: warp-path list first, then the lane-path list, each in order
  const long long nrest = n - kc;
  if (nrest > 0) {
    const int* rest = order + kc;
    jp_flags_kernel<<<blocks, 256, 0, s>>>(rest, nrest, pos, ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(exclusive_scan_i64(pos, pos, nrest, sb.temp, s));
    jp_split_kernel<<<blocks, 256, 0, s>>>(rest, pos, nrest, plist, ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    jp_count_kernel<<<1, 1, 0, s>>>(pos, nrest, ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    if (rounds > 0) {
      // ordered by batch first: one launch per batch from the top, so that a
      // vertex only waits on earlier vertices of its own batch
      int* first = a.take<int>(static_cast<size_t>(rounds) + 1);
      long long* bounds = a.take<long long>(2 * (static_cast<size_t>(rounds) + 1));
      unsigned long long* cur = a.take<unsigned long long>(2 * (static_cast<size_t>(rounds) + 1));
      if (!first || !bounds || !cur) return GC_ERR_OOM;
      GC_TRY_CUDA(cudaMemsetAsync(first, 0xff, sizeof(int) * (rounds + 1), s));
      GC_TRY_CUDA(cudaMemsetAsync(cur, 0, sizeof(unsigned long long) * 2 * (rounds + 1), s));
      jpo_first_kernel<<<blocks, 256, 0, s>>>(rest, nrest, state_batch, first);
      jpo_bounds_kernel<<<(rounds + 256) / 256, 256, 0, s>>>(first, pos, rounds, bounds);
      g_launches += 2;
      GC_TRY_CUDA(cudaGetLastError());
      std::vector<long long> hb(2 * (static_cast<size_t>(rounds) + 1));
      GC_TRY_CUDA(cudaMemcpyAsync(hb.data(), bounds, sizeof(long long) * hb.size(), cudaMemcpyDeviceToHost, s));
      GC_TRY_CUDA(cudaMemcpyAsync(ctx->pinned, ctl, sizeof(JpCtl), cudaMemcpyDeviceToHost, s));
      GC_TRY_CUDA(cudaStreamSynchronize(s));
      const long long nbig = static_cast<long long>(static_cast<JpCtl*>(ctx->pinned)->nbig);
      const long long nsmall = nrest - nbig;
      long long end_b = nbig, end_s = nsmall;  // ends of the next batch up's ranges
      // batches from the lowest up, so each knows where the one below starts
      std::vector<long long> lo_b(rounds + 1, -1), hi_b(rounds + 1), lo_s(rounds + 1), hi_s(rounds + 1);
      for (int bt = 1; bt <= rounds; ++bt) {
        if (hb[2 * bt] < 0) continue;
        lo_b[bt] = hb[2 * bt];
        lo_s[bt] = hb[2 * bt + 1];
        hi_b[bt] = end_b;
        hi_s[bt] = end_s;
        end_b = lo_b[bt];
        end_s = lo_s[bt];
      }
      ctx->stats.bulk_launches = 0;
      for (int bt = rounds; bt >= 1; --bt) {
        if (lo_b[bt] < 0) continue;
        ctx->timer_begin(gc_context::kTBulk, s);
        GC_TRY_CUDA(launch_bulk(ctx, ctl, cur + 2 * bt, rp, g->col_idx, key, plist + lo_b[bt], hi_b[bt] - lo_b[bt],
                                plist + nbig + lo_s[bt], hi_s[bt] - lo_s[bt], color, s));
        ctx->timer_end(s);
        ++ctx->stats.bulk_launches;
      }
    } else {
      ctx->timer_begin(gc_context::kTBulk, s);
      GC_TRY_CUDA(launch_bulk(ctx, ctl, &ctl->big_cursor, rp, g->col_idx, key, plist, -1, nullptr, 0, color, s));
      ctx->timer_end(s);
      ctx->stats.bulk_launches = 1;
    }
  }
  if (state_batch) {
    state_strip_kernel<<<blocks, 256, 0, s>>>(n, color);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }
  return finish_jp(ctx, ctl, num_colors_out, s);
}

gc_status jp_run_given(gc_context* ctx, Arena a, const gc_csr* g, const unsigned long long* prio,
                       int* color, int* num_colors_out, cudaStream_t s) {
  return jp_run_exact(ctx, a, g, KeyGiven{prio}, nullptr, nullptr, color, num_colors_out, s);
}

gc_status jp_run_ordered(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D, int rounds,
                         int* color, int* num_colors_out, cudaStream_t s) {
  if (rounds <= 255)  // the batch fits the colour word
    return jp_run_exact(ctx, a, g, KeyStateD{color, D}, batch, D, color, num_colors_out, s, rounds);
  unsigned long long* key = a.take<unsigned long long>(g->n > 0 ? g->n : 1);
  if (!key) return GC_ERR_OOM;
  GC_TRY_CUDA(adg_o_priority(batch, D, g->n, key, ctx->num_sms, s));
  return jp_run_exact(ctx, a, g, KeyGiven{key}, nullptr, D, color, num_colors_out, s);
}

// ---------------------------------------------------------------------------
// JP-ADG (gc_color_graph): bucket order, core cluster, bulk polling.
// ---------------------------------------------------------------------------
size_t jpadg_scratch_bytes(long long n, long long nnz, int rounds) {
  const BucketPlan bp = make_plan(n, rounds);
  const size_t state16 = static_cast<size_t>(n) * 2 + 256;
  const size_t nb = static_cast<size_t>(bp.B + 1);
  const size_t kc = static_cast<size_t>(kCoreMax) + 1;
  const size_t ntask = kc + static_cast<size_t>(nnz / kChunk) + 1;
  const size_t sc = scan_temp_elems(static_cast<long long>(nb)) +
                    scan_temp_elems(static_cast<long long>(kc)) + 2;
  const size_t rb = (4 * (static_cast<size_t>(bp.rounds) + 1) * 8 + 512);
  return state16 + rb + 256 + 3 * (nb * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) + 2 * (kc * 8 + 256) +
         (kc * 4 + 256) + ntask * 16 + 3 * 256 + sc * 8 + static_cast<size_t>((n + 31) / 32) * 4 + 256 + 4096;
}

namespace {
template <class Key>
gc_status jp_adg_impl(gc_context* ctx, Arena a, const gc_csr* g, const Key& key, const int* D,
                      int rounds, typename Key::W* color, int* num_colors_out, cudaStream_t s) {
  const long long n = g->n, nnz = g->nnz;
  if (num_colors_out) *num_colors_out = 0;
  ctx->stats.num_colors = 0;
  ctx->stats.jp_spins = 0;
  if (n == 0) return GC_OK;
  const BucketPlan bp = make_plan(n, rounds);
  const long long nb = bp.B + 1;
  JpCtl* ctl = a.take<JpCtl>(1);
  unsigned long long* cnt = a.take<unsigned long long>(2 * nb);  // [class 0 | class 1]
  unsigned long long* tot = a.take<unsigned long long>(nb);
  int* order = a.take<int>(n);
  int* lid = a.take<int>(n);
  unsigned* cbits = a.take<unsigned>((n + 31) / 32);
  long long* cap = a.take<long long>(kCoreMax + 1);
  long long* toff = a.take<long long>(kCoreMax + 1);
  int* pcnt = a.take<int>(kCoreMax + 1);
  const long long ntask_cap = kCoreMax + nnz / kChunk + 1;
  int* task_i = a.take<int>(ntask_cap);
  long long* task_start = a.take<long long>(ntask_cap);
  int* task_len = a.take<int>(ntask_cap);
  const size_t sc = scan_temp_elems(nb) + scan_temp_elems(kCoreMax + 1) + 2;
  long long* temp = a.take<long long>(sc);
  unsigned long long* bounds = a.take<unsigned long long>(2 * (bp.rounds + 1));
  unsigned long long* cursors = a.take<unsigned long long>(2 * bp.rounds);
  if (!ctl || !cnt || !tot || !order || !lid || !cbits || !cap || !toff || !pcnt || !task_i || !task_start ||
      !task_len || !temp || !bounds || !cursors)
    return GC_ERR_OOM;
  const long long* rp = row_ptr_of(g);
  const int blocks = ctx->num_sms * 8;
  long long* cnt_ll = reinterpret_cast<long long*>(cnt);
  long long* tot_ll = reinterpret_cast<long long*>(tot);

  // 1. order
  jp_init_kernel<<<1, 1, 0, s>>>(ctl, ctx->wait_ns, ctx->stall_vertex);
  ++g_launches;
  GC_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * nb, s));
  jpf_hist_kernel<<<blocks, 256, 0, s>>>(key, rp, n, bp, cnt, color, ctl);
  ++g_launches;
  jpf_total_kernel<<<blocks, 256, 0, s>>>(cnt, bp.B, tot);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(exclusive_scan_i64(tot_ll, tot_ll, nb, temp, s));
  GC_TRY_CUDA(exclusive_scan_i64(cnt_ll, cnt_ll, nb, temp, s));
  GC_TRY_CUDA(exclusive_scan_i64(cnt_ll + nb, cnt_ll + nb, nb, temp, s));
  const long long target = ctx->core_target < 0 ? 0 : (ctx->core_target > kCoreMax ? kCoreMax : ctx->core_target);
  jpf_pick_kernel<<<blocks, 256, 0, s>>>(tot, bp.B, static_cast<unsigned long long>(target), ctl);
  ++g_launches;
  jpf_bases_kernel<<<1, 1, 0, s>>>(tot, cnt, bp.B, ctl);
  ++g_launches;
  jpf_batch_bounds_kernel<<<(bp.rounds + 256) / 256, 256, 0, s>>>(cnt, bp, bounds);
  ++g_launches;
  GC_TRY_CUDA(cudaMemsetAsync(cursors, 0, sizeof(unsigned long long) * 2 * bp.rounds, s));
  jpf_scatter_kernel<<<blocks, 256, 0, s>>>(key, rp, n, bp, tot, cnt, ctl, order);
  ++g_launches;
  jpf_core_sort_kernel<<<blocks, 256, 0, s>>>(tot, ctl, key, order, lid);
  ++g_launches;
  {
    const int smem = kSortBig * static_cast<int>(sizeof(unsigned long long));
    GC_TRY_CUDA(cudaFuncSetAttribute(jpf_core_sort_big_kernel<Key>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem));
    jpf_core_sort_big_kernel<<<ctx->num_sms, 1024, smem, s>>>(tot, ctl, key, order, lid);
    ++g_launches;
  }
  GC_TRY_CUDA(cudaGetLastError());

  // 2. core
  JpCtl* pin = static_cast<JpCtl*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, ctl, sizeof(JpCtl), cudaMemcpyDeviceToHost, s));
  std::vector<unsigned long long> hb(2 * (bp.rounds + 1));
  GC_TRY_CUDA(cudaMemcpyAsync(hb.data(), bounds, sizeof(unsigned long long) * hb.size(),
                              cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  const long long kc = static_cast<long long>(pin->ncore);
  const unsigned long long nbig = pin->nbig, base0 = pin->base0, base1 = pin->base1;
  if (kc > 0) {
    const CoreBufs cb{lid, cbits, cap, toff, pcnt, task_i, task_start, task_len, temp};
    GC_TRY(run_core(ctx, g, order, D, kc, ctl, cb, color, s));
  }

  // 3. bulk, one batch at a time from the top: all predecessors in higher
  // batches are final when a batch starts, so its workers only ever wait on
  // vertices of their own batch
  const int* big_list = order + kc;
  const int* small_list = order + kc + nbig;
  for (int grp = 0; grp < bp.rounds; ++grp) {
    auto range = [&](int cls, unsigned long long base, unsigned long long& lo, unsigned long long& hi) {
      lo = hb[2 * grp + cls] > base ? hb[2 * grp + cls] - base : 0;
      hi = hb[2 * (grp + 1) + cls] > base ? hb[2 * (grp + 1) + cls] - base : 0;
    };
    unsigned long long b0, b1, s0, s1;
    range(0, base0, b0, b1);
    range(1, base1, s0, s1);
    if (b1 <= b0 && s1 <= s0) continue;
    ctx->timer_begin(gc_context::kTBulk, s);
    GC_TRY_CUDA(launch_bulk(ctx, ctl, cursors + 2 * grp, rp, g->col_idx, key, big_list + b0,
                            static_cast<long long>(b1 > b0 ? b1 - b0 : 0), small_list + s0,
                            static_cast<long long>(s1 > s0 ? s1 - s0 : 0), color, s));
    ctx->timer_end(s);
    ++ctx->stats.bulk_launches;
  }
  return finish_jp(ctx, ctl, num_colors_out, s);
}

}  // namespace

namespace {
// KeyState16: state words start as batch << cb (colour 0); at the end the
// colours are copied out to the caller's 32-bit array.
__global__ void state16_init_kernel(const int* __restrict__ batch, long long n, int cb,
                                    unsigned short* __restrict__ st) {
  for (long long v = gtid(); v < n; v += gstride())
    st[v] = static_cast<unsigned short>(static_cast<unsigned>(batch[v]) << cb);
}

__global__ void state16_strip_kernel(const unsigned short* __restrict__ st, long long n, int cmask,
                                     int* __restrict__ color) {
  for (long long v = gtid(); v < n; v += gstride()) color[v] = static_cast<int>(st[v]) & cmask;
}
}  // namespace

// Colour bits of the 16-bit JP-ADG state word for `rounds` batches whose
// colours are at most max_d + 1, or 0 if the word cannot hold both.
int state16_colour_bits(int rounds, int max_d) {
  if (rounds < 1 || max_d < 0) return 0;
  int bb = 0;
  while ((1 << bb) <= rounds) ++bb;  // bits of the largest batch id
  const int cb = 16 - bb;
  if (cb < 2 || static_cast<long long>(max_d) + 1 > (1ll << cb) - 1) return 0;
  return cb;
}

gc_status jp_run_fused(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D,
                       int rounds, unsigned long long seed, int* color, int* num_colors_out,
                       cudaStream_t s) {
  const long long n = g->n;
  ctx->stats.jp_state_bits = 32;
  if (rounds > 255 || n == 0)
    return jp_adg_impl(ctx, a, g, KeyFused{batch, seed}, D, rounds, color, num_colors_out, s);
  const int blocks = ctx->num_sms * 8;
  const int cb = ctx->opt.jp_state16 ? state16_colour_bits(rounds, ctx->adg_max_removal_degree) : 0;
  ctx->stats.jp_state_bits = cb > 0 ? 16 : 32;
  if (cb > 0) {
    unsigned short* st = a.take<unsigned short>(n);
    if (!st) return GC_ERR_OOM;
    state16_init_kernel<<<blocks, 256, 0, s>>>(batch, n, cb, st);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY(jp_adg_impl(ctx, a, g, KeyState16{st, seed, cb}, D, rounds, st, num_colors_out, s));
    state16_strip_kernel<<<blocks, 256, 0, s>>>(st, n, (1 << cb) - 1, color);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    return GC_OK;
  }
  state_init_kernel<<<blocks, 256, 0, s>>>(batch, n, color);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY(jp_adg_impl(ctx, a, g, KeyState{color, seed}, D, rounds, color, num_colors_out, s));
  state_strip_kernel<<<blocks, 256, 0, s>>>(n, color);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  return GC_OK;
}

gc_status jp_run_packed(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* gid,
                        const unsigned long long* seed, const long long* off, const unsigned* tiev, const int* D,
                        int rounds, int* color, int* num_colors_out, cudaStream_t s) {
  if (rounds > 255 || g->n == 0) {
    if (!tiev && g->n > 0) return GC_ERR_INVALID_ARG;
    return jp_adg_impl(ctx, a, g, KeyPacked{batch, tiev}, D, rounds, color, num_colors_out, s);
  }
  const int blocks = ctx->num_sms * 8;
  state_init_kernel<<<blocks, 256, 0, s>>>(batch, g->n, color);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY(jp_adg_impl(ctx, a, g, KeyStateG{color, gid, seed, off}, D, rounds, color, num_colors_out, s));
  state_strip_kernel<<<blocks, 256, 0, s>>>(g->n, color);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  return GC_OK;
}

namespace {
__global__ void make_priority_kind_kernel(const long long* __restrict__ row_ptr, long long n, int kind,
                                          unsigned long long seed, unsigned long long* __restrict__ key) {
  for (long long v = gtid(); v < n; v += gstride()) {
    const unsigned h = tie_hash(seed, static_cast<unsigned>(v));
    const unsigned long long d = static_cast<unsigned long long>(row_ptr[v + 1] - row_ptr[v]);
    unsigned long long k;
    if (kind == GC_PRIO_R) {
      k = h;
    } else if (kind == GC_PRIO_FF) {
      k = 0xffffffffull - static_cast<unsigned long long>(v);
    } else if (kind == GC_PRIO_LF) {
      k = (d << 32) | h;
    } else {  // GC_PRIO_LLF: ceil(log2 d), 0 for d <= 1
      const unsigned long long lg = d <= 1 ? 0ull : 64ull - static_cast<unsigned long long>(__clzll(d - 1));
      k = (lg << 32) | h;
    }
    key[v] = k;
  }
}
}  // namespace

cudaError_t make_priority_kind(const long long* row_ptr, long long n, int kind, unsigned long long seed,
                               unsigned long long* key, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  make_priority_kind_kernel<<<num_sms * 8, 256, 0, s>>>(row_ptr, n, kind, seed, key);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t make_priority(const int* batch, long long n, unsigned long long seed,
                          unsigned long long* key, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  make_priority_kernel<<<num_sms * 8, 256, 0, s>>>(batch, n, seed, key);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gc
