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
// bounded (kWaitLimitNs); a wait that runs out sets the error word and the
// remaining waits end early, so the kernel always returns.
//
// JP-ADG (the fused path of gc_color_graph) runs in three stages:
//   1. order: one counting-sort pass by (batch, top bits of rho_R) gives the
//      order without a comparison sort; isolated vertices take colour 1 at once
//      and drop out.  The first buckets, up to kCoreTarget vertices, form the
//      "core"; they are sorted exactly inside their (tiny) buckets.
//   2. core: the predecessors of each core vertex all lie in the core; they
//      are extracted across the whole GPU into compact lists of core-local
//      ids, then ONE thread block colours the core in order with the colours in
//      shared memory, where a dependency step costs a shared-memory poll
//      rather than an L2 round trip.  The core holds the long chains of the
//      DAG G_rho (the densest part of the graph, which ADG ranks last).
//   3. bulk: every other vertex by global polling (above), with all core
//      colours already final.
// gc_jp_color with an arbitrary priority array orders the vertices with an
// exact radix sort and runs stage 3 on all of them.
#include <cstring>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kJpThreads = 256;
constexpr int kJpWarps = kJpThreads / kWarp;
constexpr unsigned kBigBit = 0x80000000u;
constexpr int kCoreThreads = 1024;
constexpr int kCoreWarps = kCoreThreads / kWarp;

struct KeyFused {  // JP-ADG: (batch << 32) | rho_R(v)
  const int* batch;
  unsigned long long seed;
  __device__ __forceinline__ unsigned long long operator()(int v) const {
    return (static_cast<unsigned long long>(static_cast<unsigned>(__ldg(batch + v))) << 32) |
           tie_hash(seed, static_cast<unsigned>(v));
  }
};

struct KeyGiven {  // any priority array
  const unsigned long long* prio;
  __device__ __forceinline__ unsigned long long operator()(int v) const { return __ldg(prio + v); }
};

__device__ __forceinline__ bool precedes(unsigned long long kw, int w, unsigned long long kv, int v) {
  return kw > kv || (kw == kv && w > v);
}

__device__ __forceinline__ long long gtid() {
  return static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() {
  return static_cast<long long>(gridDim.x) * blockDim.x;
}

// ---------------------------------------------------------------------------
// Waiting on a colour word (global memory), bounded, with backoff.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wait_color(const int* p, JpCtl* ctl, unsigned long long& spins) {
  int c = ld_relaxed(p);
  if (c != 0) return c;
  const unsigned long long t0 = global_ns();
  unsigned sleep_ns = 32;
  for (unsigned it = 1;; ++it) {
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns <<= 1;
    c = ld_relaxed(p);
    if (c != 0) return c;
    ++spins;
    if ((it & 15u) == 0) {
      if (ld_relaxed(&ctl->err) != 0) return 1;
      if (global_ns() - t0 > kWaitLimitNs) {
        atomicExch(&ctl->err, kDevTimeout);
        return 1;
      }
    }
  }
}

// GetColor for a vertex of degree <= kSmallDeg, by one lane: at most 32
// predecessors, so the smallest free colour is <= 33 and a 64-bit mask of
// used colours suffices.
template <class Key>
__device__ int color_lane(int v, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                          const Key& key, int* color, JpCtl* ctl, unsigned long long& spins) {
  const unsigned long long kv = key(v);
  const long long s = row_ptr[v], e = row_ptr[v + 1];
  unsigned long long used = 0;
  for (long long k = s; k < e; ++k) {
    const int w = __ldg(col + k);
    if (precedes(key(w), w, kv, v)) {
      const int c = wait_color(color + w, ctl, spins);
      if (c <= 64) used |= 1ull << (c - 1);
    }
  }
  const int c = __ffsll(static_cast<long long>(~used));
  st_relaxed(color + v, c);
  return c;
}

// GetColor for a larger vertex, by a whole warp.  Colours of predecessors in
// the window (base, base + kColorWin] are marked in a shared bitmap; if the
// window is full the smallest free colour lies above it and the predecessors
// are scanned again for the next window.
template <class Key>
__device__ int color_warp(int v, unsigned* bm, const long long* __restrict__ row_ptr,
                          const int* __restrict__ col, const Key& key, int* color, JpCtl* ctl,
                          unsigned long long& spins) {
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
        for (; k < e; k += 32) {
          const int w = __ldg(col + k);
          if (precedes(key(w), w, kv, v)) {
            const int c = ld_relaxed(color + w);
            if (c == 0) {
              if (np == kPendCap) {
                resume = k;
                break;
              }
              pend[np++] = w;
            } else if (c > base && c <= base + kColorWin) {
              atomicOr(&bm[(c - base - 1) >> 5], 1u << ((c - base - 1) & 31));
            }
          }
        }
        for (int j = 0; j < np; ++j) {
          const int c = wait_color(color + pend[j], ctl, spins);
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
      if (lane == 0) st_relaxed(color + v, c);
      return c;
    }
  }
}

// Stage 3 (and the whole of gc_jp_color): warp-path list plist[0, nbig) and
// lane-path list plist[nbig, nbig + nsmall), both from ctl.
template <class Key>
__global__ void __launch_bounds__(kJpThreads)
jp_color_kernel(JpCtl* ctl, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                Key key, const int* __restrict__ plist, int* color) {
  __shared__ unsigned s_bm[kJpWarps][kColorWin / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nbig = static_cast<long long>(ctl->nbig);
  const long long nsmall = static_cast<long long>(ctl->nsmall);
  bool big_done = nbig == 0, small_done = nsmall == 0;
  const bool prefer_big = (warp & 1) == 0;
  int local_max = 0;
  unsigned long long spins = 0;
  while (!(big_done && small_done)) {
    const bool take_big = !big_done && (prefer_big || small_done);
    if (take_big) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&ctl->big_cursor, 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= static_cast<unsigned long long>(nbig)) {
        big_done = true;
        continue;
      }
      const int c = color_warp(plist[i], s_bm[warp], row_ptr, col, key, color, ctl, spins);
      local_max = c > local_max ? c : local_max;
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&ctl->small_cursor, 32ull);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= static_cast<unsigned long long>(nsmall)) {
        small_done = true;
        continue;
      }
      const unsigned long long i = i0 + lane;
      if (i < static_cast<unsigned long long>(nsmall)) {
        const int c = color_lane(plist[nbig + static_cast<long long>(i)], row_ptr, col, key, color,
                                 ctl, spins);
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

__global__ void jp_init_kernel(JpCtl* ctl) {
  JpCtl c{};
  c.key_and = ~0ull;
  c.bstar = -1;
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

__global__ void __launch_bounds__(256)
jpf_hist_kernel(const int* __restrict__ batch, unsigned long long seed,
                const long long* __restrict__ row_ptr, long long n, BucketPlan bp,
                unsigned long long* __restrict__ cnt, int* __restrict__ color, JpCtl* ctl) {
  bool isolated = false;
  for (long long v = gtid(); v < n; v += gstride()) {
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    if (deg == 0) {
      color[v] = 1;  // isolated: no predecessor, smallest colour
      isolated = true;
      continue;
    }
    color[v] = 0;
    const long long b = bucket_of(batch[v], tie_hash(seed, static_cast<unsigned>(v)), bp);
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

// Places every non-isolated vertex: core buckets into order[0, ncore), the
// rest into the warp-path list order[ncore, ncore + nbig) and the lane-path
// list after it.  Cursors are the exclusive scans, advanced atomically.
__global__ void __launch_bounds__(256)
jpf_scatter_kernel(const int* __restrict__ batch, unsigned long long seed,
                   const long long* __restrict__ row_ptr, long long n, BucketPlan bp,
                   unsigned long long* cur_tot, unsigned long long* cur_cls, const JpCtl* ctl,
                   int* __restrict__ order) {
  const long long bs = ctl->bstar;
  const unsigned long long ncore = ctl->ncore, nbig = ctl->nbig;
  const unsigned long long base0 = ctl->base0, base1 = ctl->base1;
  for (long long v = gtid(); v < n; v += gstride()) {
    const long long deg = row_ptr[v + 1] - row_ptr[v];
    if (deg == 0) continue;
    const long long b = bucket_of(batch[v], tie_hash(seed, static_cast<unsigned>(v)), bp);
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

// Exact order inside each core bucket (the buckets are tiny): insertion sort
// by (rho_R, id) descending; then lid[v] = position of v in the core.
__global__ void jpf_core_sort_kernel(const unsigned long long* __restrict__ cur_tot, const JpCtl* ctl,
                                     KeyFused key, int* __restrict__ order, int* __restrict__ lid) {
  const long long bs = ctl->bstar;
  for (long long b = gtid(); b <= bs; b += gstride()) {
    // after the scatter, cur_tot[b] is the end of bucket b
    const long long s = b == 0 ? 0 : static_cast<long long>(cur_tot[b - 1]);
    const long long e = static_cast<long long>(cur_tot[b]);
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

// Per core vertex: capacity of its predecessor list (degree at removal) and
// the number of UPDATE-style edge chunks of its adjacency.
__global__ void jpf_core_prep_kernel(const int* __restrict__ order, const int* __restrict__ D,
                                     const long long* __restrict__ row_ptr, const JpCtl* ctl,
                                     long long* __restrict__ cap, long long* __restrict__ ntask) {
  const long long kc = static_cast<long long>(ctl->ncore);
  for (long long i = gtid(); i <= kc; i += gstride()) {
    if (i == kc) {
      cap[i] = 0;
      ntask[i] = 0;
      continue;
    }
    const int v = order[i];
    cap[i] = D[v];
    ntask[i] = (row_ptr[v + 1] - row_ptr[v] + kChunk - 1) / kChunk;
  }
}

__global__ void jpf_core_tasks_kernel(const int* __restrict__ order, const long long* __restrict__ row_ptr,
                                      const long long* __restrict__ toff, const JpCtl* ctl,
                                      int* __restrict__ task_i, long long* __restrict__ task_start,
                                      int* __restrict__ task_len) {
  const long long kc = static_cast<long long>(ctl->ncore);
  for (long long i = gtid(); i < kc; i += gstride()) {
    const int v = order[i];
    const long long rs = row_ptr[v], re = row_ptr[v + 1];
    long long t = toff[i];
    for (long long st = rs; st < re; st += kChunk, ++t) {
      task_i[t] = static_cast<int>(i);
      task_start[t] = st;
      task_len[t] = static_cast<int>(re - st < kChunk ? re - st : kChunk);
    }
  }
}

// Predecessor lists of the core in core-local ids, edges spread over the
// lanes of each warp across 32 tasks at a time (as in ADG's UPDATE).
__global__ void __launch_bounds__(256)
jpf_core_preds_kernel(const int* __restrict__ col, KeyFused key, const int* __restrict__ order,
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
    sweep_tile(st, len, ci, col, [&](int w, int i) {
      const int v = order[i];
      if (precedes(key(w), w, key(v), v)) {
        const int slot = atomicAdd(&pcnt[i], 1);
        preds[poff[i] + slot] = lid[w];
      }
    });
  }
}

// Colours the core in one block: warps take core vertices in order; a warp
// polls its predecessors' colours in shared memory (16-bit: a core of at most
// 65535 vertices uses at most 65535 colours) and writes the smallest colour
// none of them uses.  Predecessors precede their successors in the exact core
// order, so the warp holding the earliest unfinished vertex never waits on a
// vertex no warp holds.
__global__ void __launch_bounds__(kCoreThreads, 1)
jpf_core_solve_kernel(const int* __restrict__ order, const long long* __restrict__ poff,
                      const int* __restrict__ pcnt, const int* __restrict__ preds, JpCtl* ctl,
                      int* color) {
  extern __shared__ unsigned short s_col[];
  __shared__ unsigned s_bm[kCoreWarps][kColorWin / 32];
  __shared__ int s_next;
  const int kc = static_cast<int>(ctl->ncore);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kc; i += blockDim.x) s_col[i] = 0;
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  volatile unsigned short* vcol = s_col;
  const unsigned long long t0 = global_ns();
  int local_max = 0;
  bool timed_out = false;
  for (;;) {
    int i = 0;
    if (lane == 0) i = atomicAdd(&s_next, 1);
    i = __shfl_sync(kFull, i, 0);
    if (i >= kc) break;
    const int* pl = preds + poff[i];
    const int np = pcnt[i];
    int c = 0;
    for (int base = 0;; base += kColorWin) {
      s_bm[warp][lane] = 0u;
      __syncwarp();
      for (int k = lane; k < np; k += 32) {
        const int j = __ldg(pl + k);
        int cj = vcol[j];
        if (cj == 0) {
          unsigned it = 0;
          while ((cj = vcol[j]) == 0) {
            if ((++it & 1023u) == 0 &&
                (timed_out || ld_relaxed(&ctl->err) != 0 || global_ns() - t0 > kWaitLimitNs)) {
              timed_out = true;
              cj = 1;
              break;
            }
          }
        }
        if (cj > base && cj <= base + kColorWin)
          atomicOr(&s_bm[warp][(cj - base - 1) >> 5], 1u << ((cj - base - 1) & 31));
      }
      __syncwarp();
      const unsigned freeb = ~s_bm[warp][lane];
      const unsigned fm = __ballot_sync(kFull, freeb != 0u);
      __syncwarp();
      if (fm) {
        const int f = __ffs(fm) - 1;
        const unsigned fb = __shfl_sync(kFull, freeb, f);
        c = base + f * 32 + __ffs(fb);
        break;
      }
    }
    if (lane == 0) vcol[i] = static_cast<unsigned short>(c);
    local_max = c > local_max ? c : local_max;
  }
  if (__any_sync(kFull, timed_out) && lane == 0) atomicExch(&ctl->err, kDevTimeout);
  __syncthreads();
  for (int i = threadIdx.x; i < kc; i += blockDim.x) color[order[i]] = s_col[i];
  local_max = warp_max(local_max);
  if (lane == 0) atomicMax(&ctl->max_color, local_max);
}

cudaError_t launch_bulk(gc_context* ctx, JpCtl* ctl, const long long* row_ptr, const int* col,
                        const KeyFused* kf, const KeyGiven* kg, const int* plist, int* color,
                        cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e;
  if (kf)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jp_color_kernel<KeyFused>, kJpThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jp_color_kernel<KeyGiven>, kJpThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (ctx->timing) cudaEventRecord(ctx->ev[3], s);
  if (kf)
    jp_color_kernel<KeyFused><<<ctx->num_sms * per_sm, kJpThreads, 0, s>>>(ctl, row_ptr, col, *kf, plist, color);
  else
    jp_color_kernel<KeyGiven><<<ctx->num_sms * per_sm, kJpThreads, 0, s>>>(ctl, row_ptr, col, *kg, plist, color);
  ++g_launches;
  e = cudaGetLastError();
  if (ctx->timing) cudaEventRecord(ctx->ev[4], s);
  return e;
}

gc_status finish_jp(gc_context* ctx, JpCtl* ctl, int* num_colors_out, cudaStream_t s) {
  JpCtl* pin = static_cast<JpCtl*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, ctl, sizeof(JpCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  JpCtl h;
  memcpy(&h, pin, sizeof(h));
  ctx->stats.jp_spins = static_cast<int64_t>(h.spins);
  ctx->stats.ms_jp_color = 0.f;
  if (ctx->timing) cudaEventElapsedTime(&ctx->stats.ms_jp_color, ctx->ev[3], ctx->ev[4]);
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

}  // namespace

// ---------------------------------------------------------------------------
// gc_jp_color: exact radix-sorted order, bulk stage on every vertex.
// ---------------------------------------------------------------------------
size_t jp_scratch_bytes(long long n) {
  const size_t hist = sort_hist_elems(n);
  const size_t tmp = scan_temp_elems(static_cast<long long>(hist));
  const size_t tmp2 = scan_temp_elems(n);
  return 2 * (static_cast<size_t>(n) * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) +
         hist * 8 + ((tmp > tmp2 ? tmp : tmp2) + 1) * 8 + 2048;
}

gc_status jp_run_given(gc_context* ctx, Arena a, const gc_csr* g, const unsigned long long* prio,
                       int* color, int* num_colors_out, cudaStream_t s) {
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
  sb.temp = a.take<long long>((tmp > tmp2 ? tmp : tmp2) + 1);
  if (!ctl || !sb.keys[0] || !sb.keys[1] || !sb.vals[0] || !sb.vals[1] || !sb.hist || !sb.temp)
    return GC_ERR_OOM;
  const long long* rp = row_ptr_of(g);
  const KeyGiven key{prio};
  const int blocks = ctx->num_sms * 8;
  jp_init_kernel<<<1, 1, 0, s>>>(ctl);
  ++g_launches;
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
  jp_flags_kernel<<<blocks, 256, 0, s>>>(order, n, pos, ctl);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(exclusive_scan_i64(pos, pos, n, sb.temp, s));
  jp_split_kernel<<<blocks, 256, 0, s>>>(order, pos, n, plist, ctl);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  jp_count_kernel<<<1, 1, 0, s>>>(pos, n, ctl);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(cudaMemsetAsync(color, 0, sizeof(int) * n, s));
  GC_TRY_CUDA(launch_bulk(ctx, ctl, rp, g->col_idx, nullptr, &key, plist, color, s));
  return finish_jp(ctx, ctl, num_colors_out, s);
}

// ---------------------------------------------------------------------------
// JP-ADG (gc_color_graph): bucket order, core block, bulk polling.
// ---------------------------------------------------------------------------
size_t jpadg_scratch_bytes(long long n, long long nnz, int rounds) {
  const BucketPlan bp = make_plan(n, rounds);
  const size_t nb = static_cast<size_t>(bp.B + 1);
  const size_t kc = static_cast<size_t>(kCoreTarget) + 1;
  const size_t ntask = kc + static_cast<size_t>(nnz / kChunk) + 1;
  const size_t sc = scan_temp_elems(static_cast<long long>(nb)) +
                    scan_temp_elems(static_cast<long long>(kc)) + 2;
  return 256 + 3 * (nb * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) + 2 * (kc * 8 + 256) +
         (kc * 4 + 256) + ntask * 16 + 3 * 256 + sc * 8 + 4096;
}

gc_status jp_run_fused(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D,
                       int rounds, unsigned long long seed, int* color, int* num_colors_out,
                       cudaStream_t s) {
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
  long long* cap = a.take<long long>(kCoreTarget + 1);
  long long* toff = a.take<long long>(kCoreTarget + 1);
  int* pcnt = a.take<int>(kCoreTarget + 1);
  const long long ntask_cap = kCoreTarget + nnz / kChunk + 1;
  int* task_i = a.take<int>(ntask_cap);
  long long* task_start = a.take<long long>(ntask_cap);
  int* task_len = a.take<int>(ntask_cap);
  const size_t sc = scan_temp_elems(nb) + scan_temp_elems(kCoreTarget + 1) + 2;
  long long* temp = a.take<long long>(sc);
  if (!ctl || !cnt || !tot || !order || !lid || !cap || !toff || !pcnt || !task_i || !task_start ||
      !task_len || !temp)
    return GC_ERR_OOM;
  const long long* rp = row_ptr_of(g);
  const KeyFused key{batch, seed};
  const int blocks = ctx->num_sms * 8;
  long long* cnt_ll = reinterpret_cast<long long*>(cnt);
  long long* tot_ll = reinterpret_cast<long long*>(tot);

  // 1. order
  jp_init_kernel<<<1, 1, 0, s>>>(ctl);
  ++g_launches;
  GC_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * nb, s));
  jpf_hist_kernel<<<blocks, 256, 0, s>>>(batch, seed, rp, n, bp, cnt, color, ctl);
  ++g_launches;
  jpf_total_kernel<<<blocks, 256, 0, s>>>(cnt, bp.B, tot);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(exclusive_scan_i64(tot_ll, tot_ll, nb, temp, s));
  GC_TRY_CUDA(exclusive_scan_i64(cnt_ll, cnt_ll, nb, temp, s));
  GC_TRY_CUDA(exclusive_scan_i64(cnt_ll + nb, cnt_ll + nb, nb, temp, s));
  jpf_pick_kernel<<<blocks, 256, 0, s>>>(tot, bp.B, kCoreTarget, ctl);
  ++g_launches;
  jpf_bases_kernel<<<1, 1, 0, s>>>(tot, cnt, bp.B, ctl);
  ++g_launches;
  jpf_scatter_kernel<<<blocks, 256, 0, s>>>(batch, seed, rp, n, bp, tot, cnt, ctl, order);
  ++g_launches;
  jpf_core_sort_kernel<<<blocks, 256, 0, s>>>(tot, ctl, key, order, lid);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());

  // 2. core
  JpCtl* pin = static_cast<JpCtl*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, ctl, sizeof(JpCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  const long long kc = static_cast<long long>(pin->ncore);
  if (kc > 0) {
    jpf_core_prep_kernel<<<blocks, 256, 0, s>>>(order, D, rp, ctl, cap, toff);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(exclusive_scan_i64(cap, cap, kc + 1, temp, s));
    GC_TRY_CUDA(exclusive_scan_i64(toff, toff, kc + 1, temp, s));
    long long* pin_ll = reinterpret_cast<long long*>(ctx->pinned);
    GC_TRY_CUDA(cudaMemcpyAsync(pin_ll, cap + kc, sizeof(long long), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    const long long npred_cap = pin_ll[0];
    GC_TRY(ctx->reserve_aux(static_cast<size_t>(npred_cap > 0 ? npred_cap : 1) * sizeof(int)));
    int* preds = static_cast<int*>(ctx->aux);
    GC_TRY_CUDA(cudaMemsetAsync(pcnt, 0, sizeof(int) * (kc + 1), s));
    jpf_core_tasks_kernel<<<blocks, 256, 0, s>>>(order, rp, toff, ctl, task_i, task_start, task_len);
    ++g_launches;
    jpf_core_preds_kernel<<<blocks, 256, 0, s>>>(g->col_idx, key, order, lid, toff, cap, ctl, task_i,
                                                 task_start, task_len, pcnt, preds);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    const size_t smem = static_cast<size_t>(kc) * sizeof(unsigned short);
    GC_TRY_CUDA(cudaFuncSetAttribute(jpf_core_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
    jpf_core_solve_kernel<<<1, kCoreThreads, smem, s>>>(order, cap, pcnt, preds, ctl, color);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }

  // 3. bulk
  GC_TRY_CUDA(launch_bulk(ctx, ctl, rp, g->col_idx, &key, nullptr, order + kc, color, s));
  return finish_jp(ctx, ctl, num_colors_out, s);
}

cudaError_t make_priority(const int* batch, long long n, unsigned long long seed,
                          unsigned long long* key, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  make_priority_kernel<<<num_sms * 8, 256, 0, s>>>(batch, n, seed, key);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gc
