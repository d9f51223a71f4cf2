// DEC-ADG-ITR (Section 4.3) on the device: the ADG partitions
// R(l) = {v : batch[v] = l} are coloured from l = rho-bar down to 1, as in
// Algorithm 4, each by the ITR form of SIM-COL (Algorithm 5): every vertex
// still in U draws the smallest colour not in B_v, and of two adjacent
// vertices of U that drew the same colour the one with the lower key
// (rho_R(v), v) gives it back.  Every step reads only what the previous one
// left, so the result does not depend on the schedule.
//
// Per partition:
//   extract  one pass over the whole adjacency of each v in R(l): colours of
//            neighbours in higher partitions (final by now) go into B_v,
//            neighbours inside R(l) are copied to v's internal list (the
//            edges of G(l) = G[R(l)]), and v draws its first colour.  A
//            vertex without internal neighbours keeps it at once; the others
//            form U.
//   check    Part 2 on the internal lists: v keeps its draw unless an
//            internal neighbour with a higher key drew the same colour; the
//            others form the next U.
//   pick     Part 3, then Part 1 of the next iteration: v adds the colours of
//            its fixed internal neighbours to B_v and draws the smallest
//            colour not in it.
// The full adjacency is read once per vertex; the later iterations (hundreds
// on the dense top partition of a power-law graph) touch only G(l).
//
// State word of a vertex (the caller's colour array during the call):
//   bits 24..31  its batch, when rho-bar <= 255 (one load of a neighbour's
//                word then tells its partition and its colour); else 0, and
//                the batch array is read instead
//   bit  23      tentative: drawn in the current iteration, not yet kept
//   bits 0..22   colour (0: none yet).  Each kept colour is the smallest one
//                missing among the neighbours fixed before it, so a vertex of
//                colour c has neighbours of colours 1..c-1, and c colours
//                need c(c-1)/2 edges: c < 2^23 for any graph below 2^45 edges.
// B_v holds deg(v)+1 bits (the smallest colour not in B_v is at most
// |B_v| + 1 <= deg(v) + 1) at word (row_ptr[v] + v) / 32 + v, which leaves
// every vertex at least ceil((deg(v)+1)/32) words with no prefix sum.
// U is two lists in one buffer: warp-path vertices (more than 32 internal
// neighbours) from the front, lane-path vertices from the back.  The lists of
// iteration k use counters and cursors of slot k mod 3; the check of slot k
// clears slot k+2, which nothing reads any more, so no memset is needed
// between launches, and an empty slot makes a launch return at once.  The host
// launches iterations in growing chunks and reads |U| after each chunk.
#include <cstring>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kDecThreads = 256;
constexpr unsigned kTent = 1u << 23;
constexpr unsigned kColMask = kTent - 1u;
// Partitions x 2 lists counted in shared memory by the counting sort.
constexpr int kDecBinsSmem = 4096;
constexpr int kPlaceItems = 8;
// Iterations launched between two reads of |U|, at most.
constexpr int kDecChunkMax = 32;

struct PartRange {
  long long off_big, n_big;      // warp-path vertices (degree > kSmallDeg) of R(l) in `order`
  long long off_small, n_small;  // lane-path vertices
  unsigned long long cur_big, cur_small;  // cursors of the extraction
};

struct DecCtl {
  unsigned long long cnt[3][2];  // |U| of slot k % 3: [0] warp path, [1] lane path
  unsigned long long cur[3][4];  // cursors of slot k % 3: pick warp/lane, check warp/lane
  unsigned long long iters;      // pick launches that found U non-empty
  unsigned long long internal;   // sum of the internal list lengths
  int max_color;
  int err;                       // 1: a batch outside 1..rounds
  int nonempty;                  // partitions holding at least one vertex
  int pad;
};

struct DecArgs {
  const long long* row_ptr;
  const int* col;
  const int* batch;
  int* S;           // state words (the colour output)
  int* icol;        // internal lists, v's at icol[row_ptr[v] ..)
  int* ideg;        // internal list lengths
  unsigned* B;      // forbidden-colour bitmaps
  int* hint;        // first word of B_v that may have a free bit
  int* ubuf[2];     // U lists of even and odd slots
  long long ucap;   // capacity of each U buffer
  DecCtl* ctl;
  unsigned long long seed;
};

// U buffer of slot k (a select rather than an indexed parameter, which
// would put the argument block in local memory)
__device__ __forceinline__ int* ubuf_of(const DecArgs& A, int k) { return (k & 1) ? A.ubuf[1] : A.ubuf[0]; }

__device__ __forceinline__ long long bstart(const long long* row_ptr, int v) {
  return (row_ptr[v] + v) / 32 + v;
}

// (rho_R(u), u) > (rho_R(v), v)
__device__ __forceinline__ bool key_above(unsigned long long seed, int u, unsigned hv, int v) {
  const unsigned hu = tie_hash(seed, static_cast<unsigned>(u));
  return hu > hv || (hu == hv && u > v);
}

template <bool Packed>
__device__ __forceinline__ int state_word(int l, int c) {
  return Packed ? static_cast<int>((static_cast<unsigned>(l) << 24) | static_cast<unsigned>(c)) : c;
}

// ---- counting sort of the vertices by (batch, warp or lane path) ----------

__global__ void __launch_bounds__(kDecThreads)
dec_count_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ batch, long long n, int rounds,
                 bool packed, int* __restrict__ S, unsigned long long* __restrict__ bins, int* __restrict__ present,
                 DecCtl* ctl) {
  __shared__ unsigned sh[kDecBinsSmem];
  __shared__ int any_iso;
  const long long nb = 2ll * (rounds + 1);
  const bool use_sh = nb <= kDecBinsSmem;
  if (use_sh)
    for (long long i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0u;
  if (threadIdx.x == 0) any_iso = 0;
  __syncthreads();
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = batch[v];
    const long long d = row_ptr[v + 1] - row_ptr[v];
    if (b < 1 || b > rounds) {
      atomicExch(&ctl->err, 1);
      S[v] = 0;
      continue;
    }
    present[b] = 1;
    const int word = packed ? static_cast<int>(static_cast<unsigned>(b) << 24) : 0;
    if (d == 0) {  // isolated: B_v is empty and U has no neighbour, colour 1
      S[v] = word | 1;
      any_iso = 1;
      continue;
    }
    S[v] = word;
    const long long bin = 2ll * b + (d > kSmallDeg ? 0 : 1);
    if (use_sh)
      atomicAdd(&sh[bin], 1u);
    else
      atomicAdd(&bins[bin], 1ull);
  }
  __syncthreads();
  if (use_sh)
    for (long long i = threadIdx.x; i < nb; i += blockDim.x)
      if (sh[i]) atomicAdd(&bins[i], static_cast<unsigned long long>(sh[i]));
  if (threadIdx.x == 0 && any_iso) atomicMax(&ctl->max_color, 1);
}

// One block: exclusive scan of the bins in (batch, path) order into the
// partition ranges, and the count of non-empty partitions.
__global__ void __launch_bounds__(1024)
dec_scan_kernel(const unsigned long long* __restrict__ bins, const int* __restrict__ present, int rounds,
                PartRange* __restrict__ part, DecCtl* ctl) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nb = 2ll * (rounds + 1);
  if (threadIdx.x == 0) {
    carry = 0;
    part[0] = PartRange{};
  }
  int np = 0;
  for (int l = 1 + threadIdx.x; l <= rounds; l += blockDim.x) np += present[l];
  np = warp_sum(np);
  if (lane == 0 && np) atomicAdd(&ctl->nonempty, np);
  __syncthreads();
  for (long long base = 2; base < nb; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const unsigned long long x = i < nb ? bins[i] : 0ull;
    const unsigned long long incl = warp_inclusive_scan(x);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long ws = lane < static_cast<int>(blockDim.x >> 5) ? wsum[lane] : 0ull;
      wsum[lane] = warp_inclusive_scan(ws);
    }
    __syncthreads();
    const unsigned long long excl = carry + (warp ? wsum[warp - 1] : 0ull) + incl - x;
    if (i < nb) {
      PartRange& p = part[i >> 1];
      if ((i & 1) == 0) {
        p.off_big = static_cast<long long>(excl);
        p.n_big = static_cast<long long>(x);
        p.cur_big = 0;
      } else {
        p.off_small = static_cast<long long>(excl);
        p.n_small = static_cast<long long>(x);
        p.cur_small = 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
}

// Scatter: each block ranks its tile's vertices per bin in shared memory and
// reserves one range per bin with a single atomic.
__global__ void __launch_bounds__(kDecThreads)
dec_place_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ batch, long long n, int rounds,
                 const PartRange* __restrict__ part, unsigned long long* __restrict__ fill,
                 int* __restrict__ order) {
  __shared__ unsigned lcnt[kDecBinsSmem];
  __shared__ unsigned lbase[kDecBinsSmem];
  const long long nb = 2ll * (rounds + 1);
  const bool use_sh = nb <= kDecBinsSmem;
  constexpr long long kTile = static_cast<long long>(kDecThreads) * kPlaceItems;
  for (long long t0 = static_cast<long long>(blockIdx.x) * kTile; t0 < n;
       t0 += static_cast<long long>(gridDim.x) * kTile) {
    if (use_sh) {
      for (long long i = threadIdx.x; i < nb; i += blockDim.x) lcnt[i] = 0u;
      __syncthreads();
    }
    long long bin[kPlaceItems];
    unsigned rank[kPlaceItems];
#pragma unroll
    for (int j = 0; j < kPlaceItems; ++j) {
      const long long v = t0 + static_cast<long long>(j) * kDecThreads + threadIdx.x;
      bin[j] = -1;
      rank[j] = 0;
      if (v < n) {
        const int b = batch[v];
        const long long d = row_ptr[v + 1] - row_ptr[v];
        if (b >= 1 && b <= rounds && d > 0) {
          bin[j] = 2ll * b + (d > kSmallDeg ? 0 : 1);
          rank[j] = use_sh ? atomicAdd(&lcnt[bin[j]], 1u)
                           : static_cast<unsigned>(atomicAdd(&fill[bin[j]], 1ull));
        }
      }
    }
    if (use_sh) {
      __syncthreads();
      for (long long i = threadIdx.x; i < nb; i += blockDim.x)
        if (lcnt[i]) lbase[i] = static_cast<unsigned>(atomicAdd(&fill[i], static_cast<unsigned long long>(lcnt[i])));
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kPlaceItems; ++j) {
      if (bin[j] < 0) continue;
      const PartRange& p = part[bin[j] >> 1];
      const long long off = (bin[j] & 1) ? p.off_small : p.off_big;
      const long long pos = off + (use_sh ? lbase[bin[j]] : 0u) + rank[j];
      order[pos] = static_cast<int>(t0 + static_cast<long long>(j) * kDecThreads + threadIdx.x);
    }
    if (use_sh) __syncthreads();
  }
}

// ---- extraction and first draw --------------------------------------------

// One vertex per lane (degree <= kSmallDeg: B_v fits 64 bits).  All 32 lanes
// call it (v < 0: none) for the warp-aggregated append to U.
template <bool Packed>
__device__ int extract_lane(const DecArgs& A, int v, int l, unsigned long long* cnt, int* ub) {
  constexpr int U = 4;
  int c = 0;
  bool enter = false;
  int internal = 0;
  if (v >= 0) {
    const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
    unsigned long long used = 0;
    int id = 0;
    for (long long k = s; k < e; k += U) {
      int w[U], x[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) w[u] = k + u < e ? __ldg(A.col + k + u) : -1;
#pragma unroll
      for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
      if (!Packed) {
#pragma unroll
        for (int u = 0; u < U; ++u) b[u] = w[u] >= 0 ? __ldg(A.batch + w[u]) : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (w[u] < 0) continue;
        const int bw = Packed ? static_cast<int>(static_cast<unsigned>(x[u]) >> 24) : b[u];
        if (bw > l) {
          const unsigned cc = static_cast<unsigned>(x[u]) & kColMask;
          if (cc >= 1u && cc <= 64u) used |= 1ull << (cc - 1u);
        } else if (bw == l) {
          A.icol[s + id++] = w[u];
        }
      }
    }
    c = __ffsll(static_cast<long long>(~used));
    if (id == 0) {
      st_relaxed(A.S + v, state_word<Packed>(l, c));
    } else {
      st_relaxed(A.S + v, state_word<Packed>(l, c) | static_cast<int>(kTent));
      A.ideg[v] = id;
      A.hint[v] = 0;
      const long long bs = bstart(A.row_ptr, v);
      A.B[bs] = static_cast<unsigned>(used);
      if (e - s + 1 > 32) A.B[bs + 1] = static_cast<unsigned>(used >> 32);
      enter = true;
      internal = id;
    }
  }
  const unsigned m = __ballot_sync(kFull, enter);
  if (m) {
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    internal = warp_sum(internal);
    if (lane == 0) {
      base = atomicAdd(&cnt[1], static_cast<unsigned long long>(__popc(m)));
      atomicAdd(&A.ctl->internal, static_cast<unsigned long long>(internal));
    }
    base = __shfl_sync(kFull, base, 0);
    if (enter) ub[A.ucap - 1 - static_cast<long long>(base + __popc(m & lanemask_lt()))] = v;
  }
  return enter ? 0 : c;
}

// Smallest colour not in B_v by a warp, starting at word `from`: returns the
// colour and sets *word_out to its word.  B_v has a free bit among its first
// nw words (at most deg(v) of its deg(v)+1 colours are set).
__device__ __forceinline__ int warp_mex(const unsigned* Bv, long long from, long long nw, int* word_out) {
  const int lane = threadIdx.x & 31;
  for (long long base = from;; base += 32) {
    const long long i = base + lane;
    const unsigned word = i < nw ? __ldcg(Bv + i) : 0u;
    const unsigned fm = __ballot_sync(kFull, word != kFull);
    if (fm) {
      const int f = __ffs(fm) - 1;
      const unsigned fw = __shfl_sync(kFull, word, f);
      *word_out = static_cast<int>(base + f);
      return static_cast<int>(32 * (base + f)) + __ffs(~fw);
    }
  }
}

// One vertex of degree > kSmallDeg per warp.
template <bool Packed>
__device__ int extract_warp(const DecArgs& A, int v, int l, unsigned long long* cnt, int* ub) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
  const long long deg = e - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  for (long long i = lane; i < nw; i += 32) Bv[i] = 0u;
  __syncwarp();
  int id = 0;
  for (long long k0 = s; k0 < e; k0 += 32 * U) {
    int w[U], x[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long k = k0 + 32 * u + lane;
      w[u] = k < e ? __ldg(A.col + k) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
    if (!Packed) {
#pragma unroll
      for (int u = 0; u < U; ++u) b[u] = w[u] >= 0 ? __ldg(A.batch + w[u]) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int bw = w[u] < 0 ? 0 : (Packed ? static_cast<int>(static_cast<unsigned>(x[u]) >> 24) : b[u]);
      if (w[u] >= 0 && bw > l) {
        const long long cc = static_cast<long long>(static_cast<unsigned>(x[u]) & kColMask);
        if (cc >= 1 && cc <= deg + 1) atomicOr(Bv + ((cc - 1) >> 5), 1u << ((cc - 1) & 31));
      }
      const bool inner = w[u] >= 0 && bw == l;
      const unsigned m = __ballot_sync(kFull, inner);
      if (inner) A.icol[s + id + __popc(m & lanemask_lt())] = w[u];
      id += __popc(m);
    }
  }
  __syncwarp();
  int hw = 0;
  const int c = warp_mex(Bv, 0, nw, &hw);
  if (lane == 0) {
    if (id == 0) {
      st_relaxed(A.S + v, state_word<Packed>(l, c));
    } else {
      st_relaxed(A.S + v, state_word<Packed>(l, c) | static_cast<int>(kTent));
      A.ideg[v] = id;
      A.hint[v] = hw;
      atomicAdd(&A.ctl->internal, static_cast<unsigned long long>(id));
      if (id > kSmallDeg)
        ub[atomicAdd(&cnt[0], 1ull)] = v;
      else
        ub[A.ucap - 1 - static_cast<long long>(atomicAdd(&cnt[1], 1ull))] = v;
    }
  }
  return id == 0 ? c : 0;
}

template <bool Packed>
__global__ void __launch_bounds__(kDecThreads)
dec_extract_kernel(DecArgs A, PartRange* part, int l, const int* __restrict__ order, int slot) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PartRange* pr = part + l;
  const long long nbig = pr->n_big, nsmall = pr->n_small;
  const int* big = order + pr->off_big;
  const int* small = order + pr->off_small;
  unsigned long long* cnt = A.ctl->cnt[slot % 3];
  int* ub = ubuf_of(A, slot);
  bool big_done = nbig == 0, small_done = nsmall == 0;
  const bool prefer_big = (warp & 3) != 0;
  int local_max = 0;
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&pr->cur_big, 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= static_cast<unsigned long long>(nbig)) {
        big_done = true;
        continue;
      }
      const int c = extract_warp<Packed>(A, big[i], l, cnt, ub);
      local_max = c > local_max ? c : local_max;
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&pr->cur_small, 32ull);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= static_cast<unsigned long long>(nsmall)) {
        small_done = true;
        continue;
      }
      const unsigned long long i = i0 + lane;
      const int v = i < static_cast<unsigned long long>(nsmall) ? small[i] : -1;
      const int c = extract_lane<Packed>(A, v, l, cnt, ub);
      local_max = c > local_max ? c : local_max;
    }
  }
  local_max = warp_max(local_max);
  if (lane == 0 && local_max > 0) atomicMax(&A.ctl->max_color, local_max);
}

// ---- Part 2: conflicts inside U -------------------------------------------

__device__ bool check_lose_warp(const DecArgs& A, int v, unsigned t, unsigned hv) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v];
  const int id = A.ideg[v];
  for (int j0 = 0; j0 < id; j0 += 32 * U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + 32 * u + lane;
      w[u] = j < id ? __ldg(A.icol + s + j) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
    bool hit = false;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (w[u] >= 0 && (static_cast<unsigned>(x[u]) & kColMask) == t && key_above(A.seed, w[u], hv, v)) hit = true;
    if (__any_sync(kFull, hit)) return true;
  }
  return false;
}

__device__ bool check_lose_lane(const DecArgs& A, int v, unsigned t, unsigned hv) {
  constexpr int U = 4;
  const long long s = A.row_ptr[v];
  const int id = A.ideg[v];
  for (int j0 = 0; j0 < id; j0 += U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = j0 + u < id ? __ldg(A.icol + s + j0 + u) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (w[u] >= 0 && (static_cast<unsigned>(x[u]) & kColMask) == t && key_above(A.seed, w[u], hv, v))
        return true;
  }
  return false;
}

__global__ void __launch_bounds__(kDecThreads)
dec_check_kernel(DecArgs A, int slot) {
  DecCtl* ctl = A.ctl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x < 6) {  // slot + 2: no launch reads it any more
    const int z = (slot + 2) % 3;
    if (threadIdx.x < 2)
      ctl->cnt[z][threadIdx.x] = 0;
    else
      ctl->cur[z][threadIdx.x - 2] = 0;
  }
  const int sl = slot % 3;
  const unsigned long long nbig = ctl->cnt[sl][0], nsmall = ctl->cnt[sl][1];
  if (nbig + nsmall == 0) return;
  const int* ub = ubuf_of(A, slot);
  int* un = ubuf_of(A, slot + 1);
  unsigned long long* ncnt = ctl->cnt[(slot + 1) % 3];
  unsigned long long* cur = ctl->cur[sl];
  bool big_done = nbig == 0, small_done = nsmall == 0;
  const bool prefer_big = (warp & 3) != 0;
  int local_max = 0;
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&cur[2], 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nbig) {
        big_done = true;
        continue;
      }
      const int v = ub[i];
      const unsigned xv = static_cast<unsigned>(ld_relaxed(A.S + v));
      const unsigned t = xv & kColMask;
      const bool lose = check_lose_warp(A, v, t, tie_hash(A.seed, static_cast<unsigned>(v)));
      if (lane == 0) {
        if (lose)
          un[atomicAdd(&ncnt[0], 1ull)] = v;
        else
          st_relaxed(A.S + v, static_cast<int>(xv & ~kTent));
      }
      if (!lose) local_max = static_cast<int>(t) > local_max ? static_cast<int>(t) : local_max;
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&cur[3], 32ull);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= nsmall) {
        small_done = true;
        continue;
      }
      const unsigned long long i = i0 + lane;
      bool lose = false;
      int v = -1;
      if (i < nsmall) {
        v = ub[A.ucap - 1 - static_cast<long long>(i)];
        const unsigned xv = static_cast<unsigned>(ld_relaxed(A.S + v));
        const unsigned t = xv & kColMask;
        lose = check_lose_lane(A, v, t, tie_hash(A.seed, static_cast<unsigned>(v)));
        if (!lose) {
          st_relaxed(A.S + v, static_cast<int>(xv & ~kTent));
          local_max = static_cast<int>(t) > local_max ? static_cast<int>(t) : local_max;
        }
      }
      const unsigned m = __ballot_sync(kFull, lose);
      if (m) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ncnt[1], static_cast<unsigned long long>(__popc(m)));
        base = __shfl_sync(kFull, base, 0);
        if (lose) un[A.ucap - 1 - static_cast<long long>(base + __popc(m & lanemask_lt()))] = v;
      }
    }
  }
  local_max = warp_max(local_max);
  if (lane == 0 && local_max > 0) atomicMax(&ctl->max_color, local_max);
}

// ---- Part 3 and the next Part 1 --------------------------------------------

template <bool Packed>
__device__ void pick_warp(const DecArgs& A, int v, int l) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v];
  const long long deg = A.row_ptr[v + 1] - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  const int id = A.ideg[v];
  for (int j0 = 0; j0 < id; j0 += 32 * U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + 32 * u + lane;
      w[u] = j < id ? __ldg(A.icol + s + j) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (w[u] < 0 || (static_cast<unsigned>(x[u]) & kTent)) continue;
      const long long cc = static_cast<long long>(static_cast<unsigned>(x[u]) & kColMask);
      if (cc >= 1 && cc <= deg + 1) atomicOr(Bv + ((cc - 1) >> 5), 1u << ((cc - 1) & 31));
    }
  }
  __syncwarp();
  int hw = 0;
  const int c = warp_mex(Bv, A.hint[v], nw, &hw);
  if (lane == 0) {
    A.hint[v] = hw;
    st_relaxed(A.S + v, state_word<Packed>(l, c) | static_cast<int>(kTent));
  }
}

template <bool Packed>
__device__ void pick_lane(const DecArgs& A, int v, int l) {
  constexpr int U = 4;
  const long long s = A.row_ptr[v];
  const long long deg = A.row_ptr[v + 1] - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  const int id = A.ideg[v];
  for (int j0 = 0; j0 < id; j0 += U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = j0 + u < id ? __ldg(A.icol + s + j0 + u) : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (w[u] < 0 || (static_cast<unsigned>(x[u]) & kTent)) continue;
      const long long cc = static_cast<long long>(static_cast<unsigned>(x[u]) & kColMask);
      if (cc >= 1 && cc <= deg + 1) Bv[(cc - 1) >> 5] |= 1u << ((cc - 1) & 31);
    }
  }
  long long wi = A.hint[v];
  unsigned word = wi < nw ? Bv[wi] : 0u;
  while (word == kFull && wi + 1 < nw) word = Bv[++wi];
  const int c = static_cast<int>(32 * wi) + __ffs(~word);
  A.hint[v] = static_cast<int>(wi);
  st_relaxed(A.S + v, state_word<Packed>(l, c) | static_cast<int>(kTent));
}

template <bool Packed>
__global__ void __launch_bounds__(kDecThreads)
dec_pick_kernel(DecArgs A, int slot, int l) {
  DecCtl* ctl = A.ctl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sl = slot % 3;
  const unsigned long long nbig = ctl->cnt[sl][0], nsmall = ctl->cnt[sl][1];
  if (nbig + nsmall == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->iters, 1ull);
  const int* ub = ubuf_of(A, slot);
  unsigned long long* cur = ctl->cur[sl];
  bool big_done = nbig == 0, small_done = nsmall == 0;
  const bool prefer_big = (warp & 3) != 0;
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&cur[0], 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nbig) {
        big_done = true;
        continue;
      }
      pick_warp<Packed>(A, ub[i], l);
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&cur[1], 32ull);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= nsmall) {
        small_done = true;
        continue;
      }
      const unsigned long long i = i0 + lane;
      if (i < nsmall) pick_lane<Packed>(A, ub[A.ucap - 1 - static_cast<long long>(i)], l);
      __syncwarp();
    }
  }
}

__global__ void dec_strip_kernel(long long n, int* __restrict__ S) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x)
    S[v] = static_cast<int>(static_cast<unsigned>(S[v]) & kColMask);
}

size_t bitmap_words(long long n, long long nnz) { return static_cast<size_t>((nnz + n) / 32 + n + 2); }

template <bool Packed>
gc_status dec_loop(gc_context* ctx, const DecArgs& A, PartRange* part, const int* order, int rounds,
                   cudaStream_t s) {
  const int sms = ctx->num_sms;
  const int gx = resident_grid(dec_extract_kernel<Packed>, kDecThreads, sms);
  const int gk = resident_grid(dec_check_kernel, kDecThreads, sms);
  const int gp = resident_grid(dec_pick_kernel<Packed>, kDecThreads, sms);
  unsigned long long* pinned = static_cast<unsigned long long*>(ctx->pinned);
  int slot = 0;
  for (int l = rounds; l >= 1; --l) {
    ctx->timer_begin(gc_context::kTDecExtract, s);
    dec_extract_kernel<Packed><<<gx, kDecThreads, 0, s>>>(A, part, l, order, slot);
    ctx->timer_end(s);
    ctx->timer_begin(gc_context::kTDecIterate, s);
    dec_check_kernel<<<gk, kDecThreads, 0, s>>>(A, slot);
    ctx->timer_end(s);
    g_launches += 2;
    GC_TRY_CUDA(cudaGetLastError());
    ++slot;
    // every iteration keeps the highest-key vertex of U: at most |R(l)| <= n
    // of them; a partition that runs longer is an internal error
    long long launched = 0;
    for (int chunk = 2;; chunk = chunk < kDecChunkMax ? 2 * chunk : kDecChunkMax) {
      if (launched > A.ucap + 1) return GC_ERR_CUDA;
      launched += chunk;
      ctx->timer_begin(gc_context::kTDecIterate, s);
      for (int j = 0; j < chunk; ++j) {
        dec_pick_kernel<Packed><<<gp, kDecThreads, 0, s>>>(A, slot, l);
        dec_check_kernel<<<gk, kDecThreads, 0, s>>>(A, slot);
        g_launches += 2;
        ++slot;
      }
      ctx->timer_end(s);
      GC_TRY_CUDA(cudaGetLastError());
      GC_TRY_CUDA(cudaMemcpyAsync(pinned, A.ctl->cnt[slot % 3], 2 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s));
      GC_TRY_CUDA(cudaStreamSynchronize(s));
      if (pinned[0] + pinned[1] == 0) break;
    }
  }
  return GC_OK;
}

}  // namespace

size_t dec_scratch_bytes(long long n, long long nnz, int rounds) {
  const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
  const size_t nb = 2 * static_cast<size_t>(rounds > 0 ? rounds + 1 : 2);
  return 16 * 256 + sizeof(DecCtl) + sizeof(PartRange) * (static_cast<size_t>(rounds > 0 ? rounds : 0) + 1) +
         2 * 8 * nb + 4 * (nb / 2) + 4 * 5 * nn + 4 * static_cast<size_t>(nnz > 0 ? nnz : 1) + 4 * bitmap_words(n, nnz);
}

gc_status dec_itr_run(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, int rounds,
                      unsigned long long seed, int* color, int* num_colors_out, long long* iters_out,
                      cudaStream_t s) {
  const long long n = g->n, nnz = g->nnz;
  *num_colors_out = 0;
  *iters_out = 0;
  if (n == 0) return GC_OK;
  if (rounds < 1) return GC_ERR_INVALID_ARG;
  const bool packed = rounds <= 255;
  const long long nb = 2ll * (rounds + 1);
  DecCtl* ctl = a.take<DecCtl>(1);
  PartRange* part = a.take<PartRange>(static_cast<size_t>(rounds) + 1);
  unsigned long long* bins = a.take<unsigned long long>(nb);
  unsigned long long* fill = a.take<unsigned long long>(nb);
  int* present = a.take<int>(static_cast<size_t>(rounds) + 1);
  int* order = a.take<int>(n);
  int* ideg = a.take<int>(n);
  int* hint = a.take<int>(n);
  int* ub0 = a.take<int>(n);
  int* ub1 = a.take<int>(n);
  int* icol = a.take<int>(nnz > 0 ? nnz : 1);
  unsigned* B = a.take<unsigned>(bitmap_words(n, nnz));
  if (!ctl || !part || !bins || !fill || !present || !order || !ideg || !hint || !ub0 || !ub1 || !icol || !B)
    return GC_ERR_OOM;
  GC_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(DecCtl), s));
  GC_TRY_CUDA(cudaMemsetAsync(bins, 0, sizeof(unsigned long long) * nb, s));
  GC_TRY_CUDA(cudaMemsetAsync(fill, 0, sizeof(unsigned long long) * nb, s));
  GC_TRY_CUDA(cudaMemsetAsync(present, 0, sizeof(int) * (static_cast<size_t>(rounds) + 1), s));
  const long long* rp = row_ptr_of(g);
  {
    const int want = static_cast<int>((n + kDecThreads - 1) / kDecThreads);
    const int cap = resident_grid(dec_count_kernel, kDecThreads, ctx->num_sms);
    dec_count_kernel<<<want < cap ? want : cap, kDecThreads, 0, s>>>(rp, batch, n, rounds, packed, color, bins,
                                                                      present, ctl);
    dec_scan_kernel<<<1, 1024, 0, s>>>(bins, present, rounds, part, ctl);
    const long long tiles = (n + kDecThreads * kPlaceItems - 1) / (kDecThreads * kPlaceItems);
    const int pcap = resident_grid(dec_place_kernel, kDecThreads, ctx->num_sms);
    dec_place_kernel<<<static_cast<int>(tiles < pcap ? tiles : pcap), kDecThreads, 0, s>>>(rp, batch, n, rounds,
                                                                                            part, fill, order);
    g_launches += 3;
    GC_TRY_CUDA(cudaGetLastError());
  }
  DecArgs A{};
  A.row_ptr = rp;
  A.col = g->col_idx;
  A.batch = batch;
  A.S = color;
  A.icol = icol;
  A.ideg = ideg;
  A.B = B;
  A.hint = hint;
  A.ubuf[0] = ub0;
  A.ubuf[1] = ub1;
  A.ucap = n;
  A.ctl = ctl;
  A.seed = seed;
  if (packed)
    GC_TRY(dec_loop<true>(ctx, A, part, order, rounds, s));
  else
    GC_TRY(dec_loop<false>(ctx, A, part, order, rounds, s));
  if (packed) {
    const int grid = resident_grid(dec_strip_kernel, 256, ctx->num_sms);
    dec_strip_kernel<<<grid, 256, 0, s>>>(n, color);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }
  DecCtl h;
  GC_TRY_CUDA(cudaMemcpyAsync(ctx->pinned, ctl, sizeof(DecCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  memcpy(&h, ctx->pinned, sizeof(DecCtl));
  if (h.err) return GC_ERR_INVALID_ARG;
  *num_colors_out = h.max_color;
  *iters_out = static_cast<long long>(h.nonempty) + static_cast<long long>(h.iters);
  ctx->stats.dec_internal_edges = static_cast<int64_t>(h.internal);
  return GC_OK;
}

}  // namespace gc
