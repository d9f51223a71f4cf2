// JP colouring, Algorithm 3 (Section 4.1), by predecessor polling.
//
// Algorithm 3 colours a vertex once all its predecessors (neighbours of
// higher priority) are coloured, with the smallest colour none of them uses
// (GetColor).  Here every vertex is handed to a lane (degree <= kSmallDeg) or
// to a whole warp (larger degree); the lane/warp reads the vertex's
// adjacency, keeps the colours of predecessors already coloured and waits on
// the rest by polling their colour words until they turn non-zero, then
// writes its own colour.  Colour words are written exactly once, so a
// non-zero value read with a relaxed GPU-scope load is final, and no
// predecessor counters, atomics or queues are needed (the Join of Algorithm 3
// becomes the poll).
//
// Progress: vertices are handed out in exactly decreasing (priority, id)
// order, from two lists (warp path, lane path) that each keep that order, and
// every block serves both lists.  The unfinished vertex of highest priority
// has only finished predecessors; if it has not been handed out yet, every
// vertex handed out before it on its list has a higher priority and is
// therefore finished, so its list's workers are free to take it.  Hence no
// wait cycle exists, with or without all blocks resident.  Every wait is still
// bounded (kWaitLimitNs); a wait that runs out sets the error word, and the
// remaining waits end early so the kernel always returns.
//
// The order is built by a stable radix sort of (~priority) with vertex ids
// pre-placed in decreasing order (so equal priorities fall back to the
// larger id first); the degree class rides in bit 31 of the sorted value
// and a stable partition splits the order into the two lists.
#include <cstring>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kJpThreads = 256;
constexpr int kJpWarps = kJpThreads / kWarp;
constexpr unsigned kBigBit = 0x80000000u;

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

__global__ void jp_init_kernel(JpCtl* ctl) {
  JpCtl c{};
  c.key_and = ~0ull;
  *ctl = c;
}

template <class Key>
__global__ void __launch_bounds__(kJpThreads)
jp_keys_kernel(Key key, const long long* __restrict__ row_ptr, long long n,
               unsigned long long* __restrict__ keys, int* __restrict__ vals, JpCtl* ctl) {
  unsigned long long kor = 0, kand = ~0ull;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
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

// flags[i] = 1 for warp-path vertices; the last flag is kept aside because
// the scan below runs in place.
__global__ void jp_flags_kernel(const int* __restrict__ order, long long n, long long* flags,
                                JpCtl* ctl) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long f = (static_cast<unsigned>(order[i]) & kBigBit) ? 1 : 0;
    flags[i] = f;
    if (i == n - 1) ctl->nbig = static_cast<unsigned long long>(f);
  }
}

// Stable partition: warp-path vertices first, then lane-path vertices.
__global__ void jp_split_kernel(const int* __restrict__ order, const long long* __restrict__ pos,
                                long long n, int* __restrict__ plist, JpCtl* ctl) {
  const long long nbig = pos[n - 1] + static_cast<long long>(ctl->nbig);
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned o = static_cast<unsigned>(order[i]);
    const int v = static_cast<int>(o & ~kBigBit);
    if (o & kBigBit)
      plist[pos[i]] = v;
    else
      plist[nbig + (i - pos[i])] = v;
  }
}

__global__ void jp_count_kernel(const long long* __restrict__ pos, long long n, JpCtl* ctl) {
  ctl->nbig = static_cast<unsigned long long>(pos[n - 1]) + ctl->nbig;
}

// Wait until *p != 0 (bounded); returns the value, or 1 once an error is set.
__device__ __forceinline__ int wait_color(const int* p, JpCtl* ctl, unsigned long long& spins) {
  int c = ld_relaxed(p);
  if (c != 0) return c;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    c = ld_relaxed(p);
    if (c != 0) return c;
    ++spins;
    if ((it & 63u) == 0) {
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

template <class Key>
__global__ void __launch_bounds__(kJpThreads)
jp_color_kernel(JpCtl* ctl, const long long* __restrict__ row_ptr, const int* __restrict__ col,
                Key key, const int* __restrict__ plist, long long n, int* color) {
  __shared__ unsigned s_bm[kJpWarps][kColorWin / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nbig = static_cast<long long>(ctl->nbig);
  const long long nsmall = n - nbig;
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

__global__ void make_priority_kernel(const int* __restrict__ batch, long long n, unsigned long long seed,
                                     unsigned long long* __restrict__ key) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x)
    key[v] = (static_cast<unsigned long long>(static_cast<unsigned>(batch[v])) << 32) |
             tie_hash(seed, static_cast<unsigned>(v));
}

template <class Key>
gc_status jp_run_impl(gc_context* ctx, Arena a, const gc_csr* g, Key key, int* color,
                      int* num_colors_out, cudaStream_t s) {
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

  const int blocks = ctx->num_sms * 8;
  jp_init_kernel<<<1, 1, 0, s>>>(ctl);
  ++g_launches;
  jp_keys_kernel<<<blocks, 256, 0, s>>>(key, row_ptr_of(g), n, sb.keys[0], sb.vals[0], ctl);
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

  int per_sm = 0;
  GC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jp_color_kernel<Key>, kJpThreads, 0));
  if (per_sm < 1) per_sm = 1;
  if (ctx->timing) GC_TRY_CUDA(cudaEventRecord(ctx->ev[3], s));
  jp_color_kernel<Key><<<ctx->num_sms * per_sm, kJpThreads, 0, s>>>(ctl, row_ptr_of(g), g->col_idx, key,
                                                                   plist, n, color);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  if (ctx->timing) GC_TRY_CUDA(cudaEventRecord(ctx->ev[4], s));

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

}  // namespace

size_t jp_scratch_bytes(long long n) {
  const size_t hist = sort_hist_elems(n);
  const size_t tmp = scan_temp_elems(static_cast<long long>(hist));
  const size_t tmp2 = scan_temp_elems(n);
  return 2 * (static_cast<size_t>(n) * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) +
         hist * 8 + ((tmp > tmp2 ? tmp : tmp2) + 1) * 8 + 2048;
}

gc_status jp_run_fused(gc_context* ctx, Arena a, const gc_csr* g, const int* batch,
                       unsigned long long seed, int* color, int* num_colors_out, cudaStream_t s) {
  return jp_run_impl(ctx, a, g, KeyFused{batch, seed}, color, num_colors_out, s);
}

gc_status jp_run_given(gc_context* ctx, Arena a, const gc_csr* g, const unsigned long long* prio,
                       int* color, int* num_colors_out, cudaStream_t s) {
  return jp_run_impl(ctx, a, g, KeyGiven{prio}, color, num_colors_out, s);
}

cudaError_t make_priority(const int* batch, long long n, unsigned long long seed,
                          unsigned long long* key, int num_sms, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  make_priority_kernel<<<num_sms * 8, 256, 0, s>>>(batch, n, seed, key);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gc
