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
//            its fixed internal neighbours to B_v, drops them from its
//            internal list (in place), and draws the smallest colour not in
//            B_v.
//   tail     once U is small, the partition's remaining iterations run in one
//            launch of one thread-block cluster on shared-memory replicas
//            (see dec_tail_kernel).
// The full adjacency is read once per vertex (hubs in chunks over several
// warps), and a fixed neighbour once more; the later iterations (hundreds on
// the dense top partition of a power-law graph) touch only the edges of G(l)
// between vertices of U.
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

#include <vector>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kDecThreads = 256;
constexpr unsigned kTent = 1u << 23;
constexpr unsigned kColMask = kTent - 1u;
// Bins of the counting sort (3 per partition) counted in shared memory.
constexpr int kDecBinsSmem = 4095;
constexpr int kPlaceItems = 8;
// Iterations launched between two reads of |U|, at most.
constexpr int kDecChunkMax = 32;
// Hubs: vertices of degree above kHubChunk are extracted in chunks of
// kHubChunk edges by different warps, so one hub does not hold one warp for
// the whole launch (R-MAT 24's top partition holds a vertex of degree 406k).
constexpr long long kHubChunk = 4096;

// Vertices of R(l) in `order`: hubs, then warp-path vertices (degree in
// (kSmallDeg, kHubChunk]), then lane-path vertices.
struct PartRange {
  long long off_hub, n_hub;
  long long off_big, n_big;
  long long off_small, n_small;
  unsigned long long hub_tasks;  // chunks of all hubs
  unsigned long long cur_hub, cur_big, cur_small;  // cursors of the extraction
};

__device__ __forceinline__ int bin_of(long long d) { return d > kHubChunk ? 0 : (d > kSmallDeg ? 1 : 2); }

// Entries a warp takes per cursor step from a list of `count`, so that long
// lists cost few atomics on the one cursor word and short lists still spread
// over all warps: between 1 and 16.
__device__ __forceinline__ unsigned long long grab_size(unsigned long long count) {
  const unsigned long long warps = static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);
  const unsigned long long k = count / (8 * warps);
  return k < 1 ? 1 : (k > 16 ? 16 : k);
}

// Warp-wide append to a U list: each lane holds one vertex (or none, kind 0)
// for the warp-path list (kind 1, from the front) or the lane-path list
// (kind 2, from the back); one atomic per list and warp.
__device__ __forceinline__ void append_u(int v, int kind, unsigned long long* cnt, int* ub, long long ucap) {
  const unsigned mb = __ballot_sync(kFull, kind == 1), ms = __ballot_sync(kFull, kind == 2);
  if ((mb | ms) == 0u) return;
  const int lane = threadIdx.x & 31;
  unsigned long long bb = 0, bs = 0;
  if (lane == 0) {
    if (mb) bb = atomicAdd(&cnt[0], static_cast<unsigned long long>(__popc(mb)));
    if (ms) bs = atomicAdd(&cnt[1], static_cast<unsigned long long>(__popc(ms)));
  }
  bb = __shfl_sync(kFull, bb, 0);
  bs = __shfl_sync(kFull, bs, 0);
  if (kind == 1) ub[bb + __popc(mb & lanemask_lt())] = v;
  if (kind == 2) ub[ucap - 1 - static_cast<long long>(bs + __popc(ms & lanemask_lt()))] = v;
}

struct DecCtl {  // read back whole into the context's 256-byte pinned buffer
  unsigned long long cnt[3][4];  // U of slot k % 3: [0] warp-path, [1] lane-path vertices, [2] list entries,
                                 // [3] the longest list
  unsigned long long cur[3][4];  // cursors of slot k % 3: pick warp/lane, check warp/lane
  unsigned long long iters;      // iterations after each partition's first: pick launches that
                                 // found U non-empty, and the tail's
  unsigned long long internal;   // sum of the internal list lengths
  int max_color;
  int err;                       // 1: a batch outside 1..rounds; 2: the tail did not fit
  int nonempty;                  // partitions holding at least one vertex
  int pad;
};

static_assert(sizeof(DecCtl) <= 256, "DecCtl must fit the pinned read-back buffer");

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
  const long long* hubpre;  // inclusive prefix of the hubs' chunk counts, by position in `order`
  int* hdone;               // chunks finished, per hub (same positions)
  int* lid;                 // local id of a vertex of U in the tail kernel
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
  __shared__ unsigned char sh_present[kDecBinsSmem / 3 + 1];
  __shared__ int any_iso;
  const long long nb = 3ll * (rounds + 1);
  const bool use_sh = nb <= kDecBinsSmem;
  if (use_sh) {
    for (long long i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0u;
    for (long long i = threadIdx.x; i <= rounds; i += blockDim.x) sh_present[i] = 0;
  }
  if (threadIdx.x == 0) any_iso = 0;
  __syncthreads();
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int b = batch[v];
    const long long d = row_ptr[v + 1] - row_ptr[v];
    long long bin = -1;
    if (b < 1 || b > rounds) {
      atomicExch(&ctl->err, 1);
      S[v] = 0;
    } else {
      if (use_sh)
        sh_present[b] = 1;
      else
        present[b] = 1;
      const int word = packed ? static_cast<int>(static_cast<unsigned>(b) << 24) : 0;
      if (d == 0) {  // isolated: B_v is empty and U has no neighbour, colour 1
        S[v] = word | 1;
        any_iso = 1;
      } else {
        S[v] = word;
        bin = 3ll * b + bin_of(d);
      }
    }
    // lanes with the same bin add once (the bins are few, so many coincide)
    const unsigned peers = __match_any_sync(__activemask(), bin);
    if (bin >= 0 && static_cast<int>(threadIdx.x & 31) == __ffs(peers) - 1) {
      if (use_sh)
        atomicAdd(&sh[bin], static_cast<unsigned>(__popc(peers)));
      else
        atomicAdd(&bins[bin], static_cast<unsigned long long>(__popc(peers)));
    }
  }
  __syncthreads();
  if (use_sh) {
    for (long long i = threadIdx.x; i < nb; i += blockDim.x)
      if (sh[i]) atomicAdd(&bins[i], static_cast<unsigned long long>(sh[i]));
    for (long long i = threadIdx.x; i <= rounds; i += blockDim.x)
      if (sh_present[i]) present[i] = 1;
  }
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
  const long long nb = 3ll * (rounds + 1);
  if (threadIdx.x == 0) {
    carry = 0;
    part[0] = PartRange{};
  }
  int np = 0;
  for (int l = 1 + threadIdx.x; l <= rounds; l += blockDim.x) np += present[l];
  np = warp_sum(np);
  if (lane == 0 && np) atomicAdd(&ctl->nonempty, np);
  __syncthreads();
  for (long long base = 3; base < nb; base += blockDim.x) {
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
      PartRange& p = part[i / 3];
      if (i % 3 == 0) {
        p.off_hub = static_cast<long long>(excl);
        p.n_hub = static_cast<long long>(x);
        p.hub_tasks = 0;
        p.cur_hub = 0;
      } else if (i % 3 == 1) {
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
  const long long nb = 3ll * (rounds + 1);
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
          bin[j] = 3ll * b + bin_of(d);
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
      const PartRange& p = part[bin[j] / 3];
      const int kind = static_cast<int>(bin[j] % 3);
      const long long off = kind == 0 ? p.off_hub : (kind == 1 ? p.off_big : p.off_small);
      const long long pos = off + (use_sh ? lbase[bin[j]] : 0u) + rank[j];
      order[pos] = static_cast<int>(t0 + static_cast<long long>(j) * kDecThreads + threadIdx.x);
    }
    if (use_sh) __syncthreads();
  }
}

// One block per partition (grid-stride over partitions): the chunk counts of
// the partition's hubs as an inclusive prefix (hubpre, by position in
// `order`), and the internal count and the count of finished chunks at 0.
__global__ void __launch_bounds__(kDecThreads)
dec_hub_prep_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ order, int rounds,
                    PartRange* __restrict__ part, long long* __restrict__ hubpre, int* __restrict__ hdone,
                    int* __restrict__ ideg, unsigned* __restrict__ B) {
  constexpr int kWarps = kDecThreads / 32;
  __shared__ unsigned long long wsum[kWarps];
  __shared__ unsigned long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = 1 + blockIdx.x; l <= rounds; l += gridDim.x) {
    PartRange& p = part[l];
    const long long nh = p.n_hub, off = p.off_hub;
    if (nh == 0) continue;  // the same for the whole block
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nh; base += kDecThreads) {
      const long long i = base + threadIdx.x;
      unsigned long long x = 0;
      if (i < nh) {
        const int v = order[off + i];
        x = static_cast<unsigned long long>((row_ptr[v + 1] - row_ptr[v] + kHubChunk - 1) / kHubChunk);
        hdone[off + i] = 0;
        ideg[v] = 0;
      }
      const unsigned long long incl = warp_inclusive_scan(x);
      if (lane == 31) wsum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const unsigned long long ws = warp_inclusive_scan(lane < kWarps ? wsum[lane] : 0ull);
        __syncwarp();
        if (lane < kWarps) wsum[lane] = ws;
      }
      __syncthreads();
      if (i < nh) hubpre[off + i] = static_cast<long long>(carry + (warp ? wsum[warp - 1] : 0ull) + incl);
      __syncthreads();
      if (threadIdx.x == 0) carry += wsum[kWarps - 1];
      __syncthreads();
    }
    if (threadIdx.x == 0) p.hub_tasks = carry;
    __syncthreads();
  }
}

// The hubs' bitmaps cleared before their chunks mark them: one warp per hub,
// the whole GPU over every partition.
__global__ void __launch_bounds__(kDecThreads)
dec_hub_zero_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ order, int rounds,
                    const PartRange* __restrict__ part, unsigned* __restrict__ B) {
  const int lane = threadIdx.x & 31;
  const long long gw = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (int l = 1; l <= rounds; ++l) {
    const long long nh = part[l].n_hub, off = part[l].off_hub;
    for (long long i = gw; i < nh; i += nwarps) {
      const int v = order[off + i];
      const long long nw = (row_ptr[v + 1] - row_ptr[v] + 32) / 32;
      unsigned* Bv = B + bstart(row_ptr, v);
      for (long long j = lane; j < nw; j += 32) Bv[j] = 0u;
    }
  }
}

// ---- extraction and first draw --------------------------------------------

// One vertex per lane (degree <= kSmallDeg: B_v fits 64 bits).  All 32 lanes
// call it (v < 0: none) for the warp-aggregated append to U.
template <bool Packed>
__device__ int extract_lane(const DecArgs& A, int v, int l, unsigned long long* cnt, int* ub,
                            unsigned long long* inner_sum, int* inner_max) {
  constexpr int U = 4;
  int c = 0;
  bool enter = false;
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
      *inner_sum += static_cast<unsigned long long>(id);
      *inner_max = *inner_max > id ? *inner_max : id;
    }
  }
  append_u(v, enter ? 2 : 0, cnt, ub, A.ucap);
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

// The warp paths mark colours in a 32-word window of B_v held in shared
// memory (words [w0, w0 + 32): colours 32*w0 + 1 .. 32*w0 + 1024), so that
// the many marks of one vertex do not meet as atomics on a few global words;
// marks above the window go to B_v in global memory, and words below w0 are
// full already.
__device__ __forceinline__ void mark_colour(unsigned* win, unsigned* Bv, long long w0, long long cc) {
  const long long wi = (cc - 1) >> 5;
  const unsigned bit = 1u << ((cc - 1) & 31);
  if (wi >= w0 + 32)
    atomicOr(Bv + wi, bit);
  else if (wi >= w0)
    atomicOr(win + (wi - w0), bit);
}

// After the marks: writes the window back to B_v (words below nw) and returns
// the smallest colour not in B_v, searching the window first.
__device__ __forceinline__ int window_mex(const unsigned* win, unsigned* Bv, long long w0, long long nw,
                                          bool store, int* word_out) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const unsigned word = win[lane];  // kFull beyond nw
  if (store && w0 + lane < nw) Bv[w0 + lane] = word;
  const unsigned fm = __ballot_sync(kFull, word != kFull);
  if (fm) {
    const int f = __ffs(fm) - 1;
    const unsigned fw = __shfl_sync(kFull, word, f);
    *word_out = static_cast<int>(w0 + f);
    return static_cast<int>(32 * (w0 + f)) + __ffs(~fw);
  }
  return warp_mex(Bv, w0 + 32, nw, word_out);
}

// One vertex of degree > kSmallDeg per warp; win is the warp's window.
// *kind: 0 the vertex kept its colour, 1 it joins the warp-path list of U, 2
// the lane-path list.
template <bool Packed>
__device__ int extract_warp(const DecArgs& A, int v, int l, unsigned* win, int* kind,
                            unsigned long long* inner_sum, int* inner_max) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
  const long long deg = e - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  win[lane] = lane < nw ? 0u : kFull;
  for (long long i = 32 + lane; i < nw; i += 32) Bv[i] = 0u;
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
        if (cc >= 1 && cc <= deg + 1) mark_colour(win, Bv, 0, cc);
      }
      const bool inner = w[u] >= 0 && bw == l;
      const unsigned m = __ballot_sync(kFull, inner);
      if (inner) A.icol[s + id + __popc(m & lanemask_lt())] = w[u];
      id += __popc(m);
    }
  }
  int hw = 0;
  const int c = window_mex(win, Bv, 0, nw, id > 0, &hw);
  if (lane == 0) {
    if (id == 0) {
      st_relaxed(A.S + v, state_word<Packed>(l, c));
    } else {
      st_relaxed(A.S + v, state_word<Packed>(l, c) | static_cast<int>(kTent));
      A.ideg[v] = id;
      A.hint[v] = hw;
    }
  }
  *kind = id == 0 ? 0 : (id > kSmallDeg ? 1 : 2);
  if (lane == 0) *inner_sum += static_cast<unsigned long long>(id);  // summed over the warp later
  *inner_max = *inner_max > id ? *inner_max : id;
  return id == 0 ? c : 0;
}

// Chunk c (of nchunks) of hub v by a warp: the colours of higher partitions
// are ORed into B_v (through the warp's window for the first 1,024), the
// internal neighbours appended to v's list at slots reserved on ideg[v].  The
// warp that finishes the hub's last chunk (counted on *done) draws v's first
// colour; nothing waits.
template <bool Packed>
__device__ int extract_hub_chunk(const DecArgs& A, int v, long long c, long long nchunks, int l, unsigned* win,
                                 int* done, unsigned long long* cnt, int* ub) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
  const long long deg = e - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  const long long k_lo = s + c * kHubChunk;
  const long long k_hi = k_lo + kHubChunk < e ? k_lo + kHubChunk : e;
  win[lane] = 0u;
  __syncwarp();
  for (long long k0 = k_lo; k0 < k_hi; k0 += 32 * U) {
    int w[U], x[U], b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long k = k0 + 32 * u + lane;
      w[u] = k < k_hi ? __ldg(A.col + k) : -1;
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
        if (cc >= 1 && cc <= deg + 1) mark_colour(win, Bv, 0, cc);
      }
      const bool inner = w[u] >= 0 && bw == l;
      const unsigned m = __ballot_sync(kFull, inner);
      if (m) {
        int base = 0;
        if (lane == 0) base = atomicAdd(A.ideg + v, __popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (inner) A.icol[s + base + __popc(m & lanemask_lt())] = w[u];
      }
    }
  }
  __syncwarp();
  if (lane < nw && win[lane]) atomicOr(Bv + lane, win[lane]);
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atomicAdd(done, 1) == static_cast<int>(nchunks - 1);
  last = __shfl_sync(kFull, last, 0);
  if (!last) return 0;
  __threadfence();  // every chunk's marks and appends precede its count
  int hw = 0;
  const int col = warp_mex(Bv, 0, nw, &hw);
  const int id = __ldcg(A.ideg + v);
  if (lane == 0) {
    if (id == 0) {
      st_relaxed(A.S + v, state_word<Packed>(l, col));
    } else {
      st_relaxed(A.S + v, state_word<Packed>(l, col) | static_cast<int>(kTent));
      A.hint[v] = hw;
      atomicAdd(&A.ctl->internal, static_cast<unsigned long long>(id));
      atomicAdd(&cnt[2], static_cast<unsigned long long>(id));
      atomicMax(&cnt[3], static_cast<unsigned long long>(id));
      if (id > kSmallDeg)
        ub[atomicAdd(&cnt[0], 1ull)] = v;
      else
        ub[A.ucap - 1 - static_cast<long long>(atomicAdd(&cnt[1], 1ull))] = v;
    }
  }
  return id == 0 ? col : 0;
}

template <bool Packed>
__global__ void __launch_bounds__(kDecThreads)
dec_extract_kernel(DecArgs A, PartRange* part, int l, const int* __restrict__ order, int slot) {
  __shared__ unsigned s_win[kDecThreads / 32][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PartRange* pr = part + l;
  unsigned long long* cnt = A.ctl->cnt[slot % 3];
  int* ub = ubuf_of(A, slot);
  int local_max = 0;
  unsigned long long inner_sum = 0;  // this lane's share of the internal list lengths
  int inner_max = 0;                 // and the longest list it saw
  // hub chunks first, by every warp
  const unsigned long long ntask = pr->hub_tasks;
  if (ntask) {
    const long long nh = pr->n_hub;
    const long long* pre = A.hubpre + pr->off_hub;
    const int* hubs = order + pr->off_hub;
    for (;;) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(&pr->cur_hub, 1ull);
      t = __shfl_sync(kFull, t, 0);
      if (t >= ntask) break;
      long long lo = 0, hi = nh - 1;  // the hub whose prefix first exceeds t
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (static_cast<unsigned long long>(pre[mid]) > t)
          hi = mid;
        else
          lo = mid + 1;
      }
      const long long first = lo ? pre[lo - 1] : 0;
      const int c = extract_hub_chunk<Packed>(A, hubs[lo], static_cast<long long>(t) - first, pre[lo] - first, l,
                                              s_win[warp], A.hdone + pr->off_hub + lo, cnt, ub);
      local_max = c > local_max ? c : local_max;
    }
  }
  const unsigned long long nbig = pr->n_big, nsmall = pr->n_small;
  const int* big = order + pr->off_big;
  const int* small = order + pr->off_small;
  const unsigned long long kb = grab_size(nbig), ks = grab_size((nsmall + 31) / 32);
  bool big_done = nbig == 0, small_done = nsmall == 0;
  const bool prefer_big = (warp & 3) != 0;
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&pr->cur_big, kb);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nbig) {
        big_done = true;
        continue;
      }
      const unsigned long long iend = i + kb < nbig ? i + kb : nbig;
      int myv = -1, mykind = 0;  // lane j keeps the j-th vertex's outcome
      for (int j = 0; i + j < iend; ++j) {
        const int v = big[i + j];
        int kind = 0;
        const int c = extract_warp<Packed>(A, v, l, s_win[warp], &kind, &inner_sum, &inner_max);
        if (lane == j) {
          myv = v;
          mykind = kind;
        }
        local_max = c > local_max ? c : local_max;
      }
      append_u(myv, mykind, cnt, ub, A.ucap);
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&pr->cur_small, 32 * ks);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= nsmall) {
        small_done = true;
        continue;
      }
      for (unsigned long long g = 0; g < ks && i0 + 32 * g < nsmall; ++g) {
        const unsigned long long i = i0 + 32 * g + lane;
        const int v = i < nsmall ? small[i] : -1;
        const int c = extract_lane<Packed>(A, v, l, cnt, ub, &inner_sum, &inner_max);
        local_max = c > local_max ? c : local_max;
      }
    }
  }
  local_max = warp_max(local_max);
  inner_sum = warp_sum(inner_sum);
  inner_max = warp_max(inner_max);
  if (lane == 0) {
    if (local_max > 0) atomicMax(&A.ctl->max_color, local_max);
    if (inner_sum) {
      atomicAdd(&A.ctl->internal, inner_sum);
      atomicAdd(&cnt[2], inner_sum);  // U's list entries
      atomicMax(&cnt[3], static_cast<unsigned long long>(inner_max));
    }
  }
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
  if (blockIdx.x == 0 && threadIdx.x < 8) {  // slot + 2: no launch reads it any more
    const int z = (slot + 2) % 3;
    if (threadIdx.x < 4)
      ctl->cnt[z][threadIdx.x] = 0;
    else
      ctl->cur[z][threadIdx.x - 4] = 0;
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
  const unsigned long long kb = grab_size(nbig), ks = grab_size((nsmall + 31) / 32);
  int local_max = 0;
  unsigned long long edges = 0;  // list entries of this lane's losers (the next U)
  int longest = 0;               // and their longest list
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&cur[2], kb);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nbig) {
        big_done = true;
        continue;
      }
      const unsigned long long iend = i + kb < nbig ? i + kb : nbig;
      int myv = -1, mylose = 0;  // lane j keeps the j-th vertex's outcome
      for (int j = 0; i + j < iend; ++j) {
        const int v = ub[i + j];
        const unsigned xv = static_cast<unsigned>(ld_relaxed(A.S + v));
        const unsigned t = xv & kColMask;
        const bool lose = check_lose_warp(A, v, t, tie_hash(A.seed, static_cast<unsigned>(v)));
        if (lane == 0 && !lose) st_relaxed(A.S + v, static_cast<int>(xv & ~kTent));
        if (!lose) local_max = static_cast<int>(t) > local_max ? static_cast<int>(t) : local_max;
        if (lane == j) {
          myv = v;
          mylose = lose;
        }
      }
      if (mylose) {
        const int id = A.ideg[myv];
        edges += static_cast<unsigned long long>(id);
        longest = longest > id ? longest : id;
      }
      append_u(myv, mylose ? 1 : 0, ncnt, un, A.ucap);
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&cur[3], 32 * ks);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= nsmall) {
        small_done = true;
        continue;
      }
      for (unsigned long long g = 0; g < ks && i0 + 32 * g < nsmall; ++g) {
        const unsigned long long i = i0 + 32 * g + lane;
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
          } else {
            const int id = A.ideg[v];
            edges += static_cast<unsigned long long>(id);
            longest = longest > id ? longest : id;
          }
        }
        append_u(v, lose ? 2 : 0, ncnt, un, A.ucap);
      }
    }
  }
  edges = warp_sum(edges);
  longest = warp_max(longest);
  if (lane == 0 && edges) {
    atomicAdd(&ncnt[2], edges);
    atomicMax(&ncnt[3], static_cast<unsigned long long>(longest));
  }
  local_max = warp_max(local_max);
  if (lane == 0 && local_max > 0) atomicMax(&ctl->max_color, local_max);
}

// ---- Part 3 and the next Part 1 --------------------------------------------

template <bool Packed>
__device__ void pick_warp(const DecArgs& A, int v, int l, unsigned* win) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const long long s = A.row_ptr[v];
  const long long deg = A.row_ptr[v + 1] - s;
  const long long nw = (deg + 32) / 32;
  unsigned* Bv = A.B + bstart(A.row_ptr, v);
  const int id = A.ideg[v];
  const long long w0 = A.hint[v];  // words below the last colour's are full
  win[lane] = w0 + lane < nw ? __ldcg(Bv + w0 + lane) : kFull;
  __syncwarp();
  int kept = 0;  // the list is compacted in place to the neighbours still in U
  for (int j0 = 0; j0 < id; j0 += 32 * U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + 32 * u + lane;
      w[u] = j < id ? A.icol[s + j] : -1;  // plain loads: this kernel rewrites the list
    }
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool tent = w[u] >= 0 && (static_cast<unsigned>(x[u]) & kTent);
      if (w[u] >= 0 && !tent) {  // fixed: its colour joins B_v, and it leaves the list
        const long long cc = static_cast<long long>(static_cast<unsigned>(x[u]) & kColMask);
        if (cc >= 1 && cc <= deg + 1) mark_colour(win, Bv, w0, cc);
      }
      // every lane loaded the whole window before this first ballot, and the
      // writes land below the window's end: no entry is overwritten unread
      const unsigned m = __ballot_sync(kFull, tent);
      if (tent) A.icol[s + kept + __popc(m & lanemask_lt())] = w[u];
      kept += __popc(m);
    }
  }
  int hw = 0;
  const int c = window_mex(win, Bv, w0, nw, true, &hw);
  if (lane == 0) {
    A.ideg[v] = kept;
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
  int kept = 0;
  for (int j0 = 0; j0 < id; j0 += U) {
    int w[U], x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = j0 + u < id ? A.icol[s + j0 + u] : -1;
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = w[u] >= 0 ? ld_relaxed(A.S + w[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (w[u] < 0) continue;
      if (static_cast<unsigned>(x[u]) & kTent) {
        A.icol[s + kept++] = w[u];
        continue;
      }
      const long long cc = static_cast<long long>(static_cast<unsigned>(x[u]) & kColMask);
      if (cc >= 1 && cc <= deg + 1) Bv[(cc - 1) >> 5] |= 1u << ((cc - 1) & 31);
    }
  }
  A.ideg[v] = kept;
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
  __shared__ unsigned s_win[kDecThreads / 32][32];
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
  const unsigned long long kb = grab_size(nbig), ks = grab_size((nsmall + 31) / 32);
  while (!(big_done && small_done)) {
    if (!big_done && (prefer_big || small_done)) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(&cur[0], kb);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nbig) {
        big_done = true;
        continue;
      }
      const unsigned long long iend = i + kb < nbig ? i + kb : nbig;
      for (; i < iend; ++i) pick_warp<Packed>(A, ub[i], l, s_win[warp]);
    } else {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(&cur[1], 32 * ks);
      i0 = __shfl_sync(kFull, i0, 0);
      if (i0 >= nsmall) {
        small_done = true;
        continue;
      }
      const unsigned long long iend = i0 + 32 * ks < nsmall ? i0 + 32 * ks : nsmall;
      for (unsigned long long i = i0 + lane; i < iend; i += 32)
        pick_lane<Packed>(A, ub[A.ucap - 1 - static_cast<long long>(i)], l);
      __syncwarp();
    }
  }
}

// ---- the tail of a partition in one thread-block cluster -------------------
//
// Once U is small (at most kTailMax vertices whose internal lists fit the
// cluster's shared memory), the rest of the partition's SIM-COL iterations
// run in one launch of one cluster.  Every CTA keeps a replica of U's state
// words (colour | tentative, by local id) and its own share of the internal
// lists (16-bit local ids) in shared memory; the pick and the check are two
// phases separated by cluster barriers, and a vertex whose word changes
// writes it into every CTA's replica through distributed shared memory.  An
// iteration then costs two barriers and shared-memory scans instead of two
// launches and L2 round trips; the top partitions of power-law graphs are
// near-cliques that fix about one vertex per iteration for hundreds of
// iterations.

constexpr int kTailMax = 4096;  // |U| at most (16-bit local ids)
constexpr int kTailThreads = 1024;
constexpr int kTailClusterMax = 16;
constexpr int kTailSmem = 200 * 1024;
// replica, hashes and split prefix (4 B each per local id) and flag words
constexpr int kTailFixed = 12 * kTailMax + 4 + 64;
// per owned vertex: global id, window word index, window word, list length,
// bitmap words (20 B), so a vertex with d list entries takes 2 (d + 10) bytes
constexpr int kTailVertexWeight = 10;

__device__ __forceinline__ unsigned tail_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned tail_ctas() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// All threads of all CTAs arrive; shared-memory writes before it, local or
// remote, are visible to every thread after it.
__device__ __forceinline__ void tail_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of this CTA's shared variable `p` in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned tail_map(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"(static_cast<unsigned>(__cvta_generic_to_shared(p))), "r"(rank));
  return r;
}
__device__ __forceinline__ void tail_st(unsigned addr, unsigned v) {
  asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Largest per-CTA shared memory for the owned vertices of a split of U (u
// vertices, `entries` list entries, the longest list `longest`) over c CTAs,
// in bytes: each CTA's weight is below W / c plus the heaviest vertex.
__host__ __device__ __forceinline__ long long tail_need(long long u, long long entries, long long longest, int c) {
  const long long w = entries + kTailVertexWeight * u;
  return 2 * (w / c + 1 + longest + kTailVertexWeight) + 16;
}

template <bool Packed>
__global__ void __launch_bounds__(kTailThreads, 1)
dec_tail_kernel(DecArgs A, int slot, int l) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  unsigned* st = reinterpret_cast<unsigned*>(s_dyn);  // replica [kTailMax]
  unsigned* hk = st + kTailMax;                       // rho_R by local id [kTailMax]
  int* pre = reinterpret_cast<int*>(hk + kTailMax);   // split prefix [kTailMax + 1]
  unsigned* sc = reinterpret_cast<unsigned*>(pre + kTailMax + 1);  // [16]
  int* o_gv = reinterpret_cast<int*>(sc + 16);        // per owned vertex ...
  const int rank = static_cast<int>(tail_rank()), C = static_cast<int>(tail_ctas());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  DecCtl* ctl = A.ctl;
  const int sl = slot % 3;
  const long long nbig = static_cast<long long>(ctl->cnt[sl][0]);
  const int u = static_cast<int>(ctl->cnt[sl][0] + ctl->cnt[sl][1]);
  const int* ub = ubuf_of(A, slot);
  int* lid = A.lid;
  auto uid = [&](int i) -> int { return i < nbig ? ub[i] : ub[A.ucap - 1 - (i - nbig)]; };

  // 1. replica, hashes, local ids; weights ideg + kTailVertexWeight
  for (int i = threadIdx.x; i < u; i += blockDim.x) {
    const int v = uid(i);
    st[i] = static_cast<unsigned>(ld_relaxed(A.S + v)) & (kTent | kColMask);
    hk[i] = tie_hash(A.seed, static_cast<unsigned>(v));
    lid[v] = i;
    pre[i + 1] = A.ideg[v] + kTailVertexWeight;
  }
  if (threadIdx.x < 16) sc[threadIdx.x] = 0u;
  if (threadIdx.x == 0) pre[0] = 0;
  __syncthreads();
  // inclusive scan of pre[1..u] by warp 0 (u <= 4096: 128 steps of 32)
  if (warp == 0) {
    int carry = 0;
    for (int b = 1; b <= u; b += 32) {
      const int i = b + lane;
      const int x = i <= u ? pre[i] : 0;
      const int incl = warp_inclusive_scan(x);
      if (i <= u) pre[i] = carry + incl;
      carry += __shfl_sync(kFull, incl, 31);
    }
  }
  __syncthreads();
  // 2. CTA r owns the local ids i with pre[i] * C / W == r (contiguous);
  // every CTA checks every CTA's share, so all agree on a misfit
  const long long W = pre[u];
  auto first_of = [&](int r) -> int {  // first i with pre[i] * C >= r * W
    int lo = 0, hi = u;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (static_cast<long long>(pre[mid]) * C >= static_cast<long long>(r) * W)
        hi = mid;
      else
        lo = mid + 1;
    }
    return lo;
  };
  const long long avail = kTailSmem - kTailFixed;
  if (threadIdx.x < static_cast<unsigned>(C)) {
    const int r = threadIdx.x;
    const int a0 = first_of(r), a1 = r + 1 < C ? first_of(r + 1) : u;
    if (2ll * (pre[a1] - pre[a0]) + 16 > avail) atomicOr(&sc[3], 1u);
  }
  __syncthreads();
  if (sc[3]) {
    if (rank == 0 && threadIdx.x == 0) atomicExch(&ctl->err, 2);
    return;  // no cluster barrier or remote access has happened yet
  }
  const int lo = first_of(rank), hi = rank + 1 < C ? first_of(rank + 1) : u;
  const int o = hi - lo;
  int* o_hint = o_gv + o;
  unsigned* o_word = reinterpret_cast<unsigned*>(o_hint + o);
  int* o_cnt = reinterpret_cast<int*>(o_word + o);
  int* o_nwords = o_cnt + o;
  unsigned short* lists = reinterpret_cast<unsigned short*>(o_nwords + o);
  // list of owned vertex a at lists[pre[lo + a] - pre[lo] - kTailVertexWeight * a ..]
  auto list_off = [&](int a) -> int { return pre[lo + a] - pre[lo] - kTailVertexWeight * a; };

  // 3. owned lists in 16-bit local ids; neighbours fixed since the last pick
  // go into B_v and leave the list
  for (int a = warp; a < o; a += nwarps) {
    const int v = uid(lo + a);
    const long long s = A.row_ptr[v];
    const long long deg = A.row_ptr[v + 1] - s;
    const long long nw = (deg + 32) / 32;
    unsigned* Bv = A.B + bstart(A.row_ptr, v);
    const int id = A.ideg[v];
    unsigned short* L = lists + list_off(a);
    int kept = 0;
    for (int j0 = 0; j0 < id; j0 += 32) {
      const int j = j0 + lane;
      const int w = j < id ? A.icol[s + j] : -1;
      const unsigned x = w >= 0 ? static_cast<unsigned>(ld_relaxed(A.S + w)) : 0u;
      const bool tent = w >= 0 && (x & kTent);
      if (w >= 0 && !tent) {
        const long long cc = static_cast<long long>(x & kColMask);
        if (cc >= 1 && cc <= deg + 1) atomicOr(Bv + ((cc - 1) >> 5), 1u << ((cc - 1) & 31));
      }
      const unsigned m = __ballot_sync(kFull, tent);
      if (tent) L[kept + __popc(m & lanemask_lt())] = static_cast<unsigned short>(lid[w]);
      kept += __popc(m);
    }
    __syncwarp();
    if (lane == 0) {
      const int h = A.hint[v];
      o_gv[a] = v;
      o_hint[a] = h;
      o_word[a] = __ldcg(Bv + h);
      o_cnt[a] = kept;
      o_nwords[a] = static_cast<int>(nw);
    }
  }
  tail_sync();  // every replica complete before any remote write

  // 4. iterations
  int it = 0, local_max = 0;
  for (;;) {
    // pick: fixed neighbours into B_v (the window word, or B_v above it),
    // out of the list; draw the smallest free colour
    for (int a = warp; a < o; a += nwarps) {
      const int i = lo + a;
      if (!(st[i] & kTent)) continue;
      unsigned short* L = lists + list_off(a);
      const int cnt = o_cnt[a];
      const int h0 = o_hint[a];
      const int nw = o_nwords[a];
      unsigned* Bv = A.B + bstart(A.row_ptr, o_gv[a]);
      int kept = 0;
      for (int j0 = 0; j0 < cnt; j0 += 32) {
        const int k = j0 + lane;
        const int j = k < cnt ? L[k] : -1;
        const unsigned x = j >= 0 ? st[j] : 0u;
        const bool tent = j >= 0 && (x & kTent);
        if (j >= 0 && !tent) {
          const int wi = static_cast<int>(((x & kColMask) - 1u) >> 5);
          const unsigned bit = 1u << (((x & kColMask) - 1u) & 31);
          if (wi == h0)
            atomicOr(&o_word[a], bit);
          else if (wi > h0 && wi < nw)
            atomicOr(Bv + wi, bit);
        }
        const unsigned m = __ballot_sync(kFull, tent);
        if (tent) L[kept + __popc(m & lanemask_lt())] = static_cast<unsigned short>(j);
        kept += __popc(m);
      }
      __syncwarp();
      int t = 0;
      if (lane == 0) {
        o_cnt[a] = kept;
        int h = h0;
        unsigned word = o_word[a];
        while (word == kFull && h + 1 < nw) {
          Bv[h] = word;
          word = __ldcg(Bv + ++h);
        }
        o_word[a] = word;
        o_hint[a] = h;
        t = 32 * h + __ffs(~word);
      }
      t = __shfl_sync(kFull, t, 0);
      if (lane < C) tail_st(tail_map(&st[i], lane), kTent | static_cast<unsigned>(t));
    }
    tail_sync();
    // check: keep the draw unless a higher-key neighbour in U drew it too
    for (int a = warp; a < o; a += nwarps) {
      const int i = lo + a;
      const unsigned xi = st[i];
      if (!(xi & kTent)) continue;
      const unsigned t = xi & kColMask, hv = hk[i];
      const unsigned short* L = lists + list_off(a);
      const int cnt = o_cnt[a];
      bool hit = false;
      for (int k = lane; k < cnt && !hit; k += 32) {
        const int j = L[k];
        if ((st[j] & kColMask) == t && (hk[j] > hv || (hk[j] == hv && uid(j) > o_gv[a]))) hit = true;
      }
      const bool lose = __any_sync(kFull, hit);
      if (!lose) {
        if (lane < C) tail_st(tail_map(&st[i], lane), t);
        if (lane == 0) st_relaxed(A.S + o_gv[a], state_word<Packed>(l, static_cast<int>(t)));
        local_max = static_cast<int>(t) > local_max ? static_cast<int>(t) : local_max;
      }
    }
    tail_sync();
    // every replica now holds the same flags: each CTA sees alone whether U
    // is empty (the next pick rewrites only words that stay tentative)
    int left = 0;
    for (int i = threadIdx.x; i < u; i += blockDim.x) left |= static_cast<int>(st[i] & kTent);
    left = __syncthreads_or(left);
    ++it;
    if (!left) break;
    if (it > u) {  // cannot happen: every iteration keeps the highest key of U
      if (rank == 0 && threadIdx.x == 0) atomicExch(&ctl->err, 2);
      break;
    }
  }
  tail_sync();  // no CTA leaves while another may still read its shared memory

  local_max = warp_max(local_max);
  if (lane == 0 && local_max > 0) atomicMax(&ctl->max_color, local_max);
  if (rank == 0 && threadIdx.x == 0) {
    atomicAdd(&ctl->iters, static_cast<unsigned long long>(it));
    for (int z = 1; z <= 2; ++z) {  // slots slot+1, slot+2: empty, cursors at 0
      const int q = (slot + z) % 3;
      for (int f = 0; f < 4; ++f) ctl->cnt[q][f] = 0;
      for (int f = 0; f < 4; ++f) ctl->cur[q][f] = 0;
    }
  }
}

__global__ void dec_strip_kernel(long long n, int* __restrict__ S) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x)
    S[v] = static_cast<int>(static_cast<unsigned>(S[v]) & kColMask);
}

size_t bitmap_words(long long n, long long nnz) { return static_cast<size_t>((nnz + n) / 32 + n + 2); }

// CTAs of the tail cluster: the largest of 16, 8, 4, 2 that the device can
// place with the tail's shared memory (0: none).
int tail_cluster_size(gc_context* ctx) {
  if (ctx->tail_cluster != 0) return ctx->tail_cluster > 0 ? ctx->tail_cluster : 0;
  ctx->tail_cluster = -1;
  for (auto k : {dec_tail_kernel<true>, dec_tail_kernel<false>}) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  for (int cs = kTailClusterMax; cs >= 2; cs /= 2) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = kTailSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, dec_tail_kernel<true>, &cfg) == cudaSuccess && ncl >= 1) {
      ctx->tail_cluster = cs;
      return cs;
    }
    cudaGetLastError();
  }
  return 0;
}

// levels: the non-empty partitions, highest first.
template <bool Packed>
gc_status dec_loop(gc_context* ctx, const DecArgs& A, PartRange* part, const int* order,
                   const std::vector<int>& levels, cudaStream_t s) {
  const int sms = ctx->num_sms;
  const int tail_c = ctx->dec_tail ? tail_cluster_size(ctx) : 0;
  const int gx = resident_grid(dec_extract_kernel<Packed>, kDecThreads, sms);
  const int gk = resident_grid(dec_check_kernel, kDecThreads, sms);
  const int gp = resident_grid(dec_pick_kernel<Packed>, kDecThreads, sms);
  unsigned long long* pinned = static_cast<unsigned long long*>(ctx->pinned);
  int slot = 0;
  for (const int l : levels) {
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
    int gp_now = gp, gk_now = gk;  // U only shrinks: grids sized by the last |U| read
    for (int chunk = 2;; chunk = chunk < kDecChunkMax ? 2 * chunk : kDecChunkMax) {
      if (launched > A.ucap + 1) return GC_ERR_CUDA;
      launched += chunk;
      ctx->timer_begin(gc_context::kTDecIterate, s);
      for (int j = 0; j < chunk; ++j) {
        dec_pick_kernel<Packed><<<gp_now, kDecThreads, 0, s>>>(A, slot, l);
        dec_check_kernel<<<gk_now, kDecThreads, 0, s>>>(A, slot);
        g_launches += 2;
        ++slot;
      }
      ctx->timer_end(s);
      GC_TRY_CUDA(cudaGetLastError());
      GC_TRY_CUDA(cudaMemcpyAsync(pinned, A.ctl->cnt[slot % 3], 4 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, s));
      GC_TRY_CUDA(cudaStreamSynchronize(s));
      const unsigned long long u = pinned[0] + pinned[1];
      if (u == 0) break;
      if (tail_c > 0 && u <= static_cast<unsigned long long>(kTailMax) &&
          kTailFixed + tail_need(static_cast<long long>(u), static_cast<long long>(pinned[2]),
                                 static_cast<long long>(pinned[3]), tail_c) <= kTailSmem) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = tail_c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(tail_c);
        cfg.blockDim = dim3(kTailThreads);
        cfg.dynamicSmemBytes = kTailSmem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ctx->timer_begin(gc_context::kTDecIterate, s);
        GC_TRY_CUDA(cudaLaunchKernelEx(&cfg, dec_tail_kernel<Packed>, A, slot, l));
        ctx->timer_end(s);
        ++g_launches;
        ++ctx->stats.dec_tail_partitions;
        ++slot;  // the tail leaves slots slot+1 and slot+2 empty
        break;
      }
      // one warp per warp-path vertex, one per 32 lane-path vertices
      const unsigned long long warps = pinned[0] + (pinned[1] + 31) / 32;
      const unsigned long long want = (warps + kDecThreads / 32 - 1) / (kDecThreads / 32);
      gp_now = want < static_cast<unsigned long long>(gp) ? static_cast<int>(want) : gp;
      gk_now = want < static_cast<unsigned long long>(gk) ? static_cast<int>(want) : gk;
    }
  }
  return GC_OK;
}

}  // namespace

size_t dec_scratch_bytes(long long n, long long nnz, int rounds) {
  const size_t nn = static_cast<size_t>(n > 0 ? n : 1);
  const size_t nr = static_cast<size_t>(rounds > 0 ? rounds : 0) + 1;
  return 17 * 256 + sizeof(DecCtl) + sizeof(PartRange) * nr + 2 * 8 * 3 * nr + 4 * nr + 4 * 7 * nn + 8 * nn +
         4 * static_cast<size_t>(nnz > 0 ? nnz : 1) + 4 * bitmap_words(n, nnz);
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
  const long long nb = 3ll * (rounds + 1);
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
  long long* hubpre = a.take<long long>(n);
  int* hdone = a.take<int>(n);
  int* lid = a.take<int>(n);
  if (!lid) return GC_ERR_OOM;
  if (!ctl || !part || !bins || !fill || !present || !order || !ideg || !hint || !ub0 || !ub1 || !icol || !B ||
      !hubpre || !hdone)
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
    const int hblocks = rounds < 4 * ctx->num_sms ? rounds : 4 * ctx->num_sms;
    dec_hub_prep_kernel<<<hblocks, kDecThreads, 0, s>>>(rp, order, rounds, part, hubpre, hdone, ideg, B);
    dec_hub_zero_kernel<<<resident_grid(dec_hub_zero_kernel, kDecThreads, ctx->num_sms), kDecThreads, 0, s>>>(
        rp, order, rounds, part, B);
    g_launches += 5;
    GC_TRY_CUDA(cudaGetLastError());
  }
  // the partitions that hold vertices: a caller's batch array may leave many
  // of 1..num_rounds empty, and each would still cost launches and a read-back
  std::vector<int> levels;
  {
    std::vector<int> hp(static_cast<size_t>(rounds) + 1);
    GC_TRY_CUDA(cudaMemcpyAsync(hp.data(), present, sizeof(int) * hp.size(), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    for (int l = rounds; l >= 1; --l)
      if (hp[l]) levels.push_back(l);
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
  A.hubpre = hubpre;
  A.hdone = hdone;
  A.lid = lid;
  A.ctl = ctl;
  A.seed = seed;
  if (packed)
    GC_TRY(dec_loop<true>(ctx, A, part, order, levels, s));
  else
    GC_TRY(dec_loop<false>(ctx, A, part, order, levels, s));
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
  if (h.err == 1) return GC_ERR_INVALID_ARG;
  if (h.err) return GC_ERR_CUDA;  // the tail found U larger than its shared memory: cannot happen
  *num_colors_out = h.max_color;
  *iters_out = static_cast<long long>(h.nonempty) + static_cast<long long>(h.iters);
  ctx->stats.dec_internal_edges = static_cast<int64_t>(h.internal);
  return GC_OK;
}

}  // namespace gc
