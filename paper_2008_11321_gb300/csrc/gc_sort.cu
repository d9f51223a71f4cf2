// Stable LSD radix sort of (uint64 key, int32 value) pairs, 8-bit digits.
//
// Per pass: a tile histogram kernel writes the 256 digit counts of every
// 4096-item tile in digit-major order, one exclusive scan turns them into
// output offsets, and a scatter kernel ranks each tile's items stably
// (warp __match_any_sync ranks, combined across the block's warps) and
// writes them to their final places.  Digits that are constant over all
// keys are skipped by the caller through `digit_mask`.
#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096

__global__ void __launch_bounds__(kSortThreads)
sort_hist_kernel(const unsigned long long* __restrict__ keys, long long n, int shift,
                 long long* __restrict__ hist, long long ntiles) {
  __shared__ int counts[256];
  counts[threadIdx.x] = 0;
  __syncthreads();
  const long long base = static_cast<long long>(blockIdx.x) * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    long long idx = base + i;
    if (idx < n) atomicAdd(&counts[(keys[idx] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[static_cast<long long>(threadIdx.x) * ntiles + blockIdx.x] = counts[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads)
sort_scatter_kernel(const unsigned long long* __restrict__ keys_in, const int* __restrict__ vals_in,
                    unsigned long long* __restrict__ keys_out, int* __restrict__ vals_out,
                    long long n, int shift, const long long* __restrict__ offsets,
                    long long ntiles) {
  __shared__ int wcnt[kSortWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
  __syncwarp();

  const long long seg = static_cast<long long>(blockIdx.x) * kSortTile + warp * (kSortItems * 32);
  unsigned long long key[kSortItems];
  int val[kSortItems];
  int rank[kSortItems];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    long long idx = seg + r * 32 + lane;
    bool ok = idx < n;
    key[r] = ok ? keys_in[idx] : 0ull;
    val[r] = ok ? vals_in[idx] : 0;
    unsigned d = ok ? static_cast<unsigned>((key[r] >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(kFull, d);
    int pre = ok ? wcnt[warp][d] : 0;
    __syncwarp();
    if (ok && (peers & lt) == 0) wcnt[warp][d] = pre + __popc(peers);
    __syncwarp();
    rank[r] = pre + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: exclusive prefix over the warps of this block
  {
    const int d = threadIdx.x;  // kSortThreads == 256 digits
    int run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      int c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    long long idx = seg + r * 32 + lane;
    if (idx < n) {
      unsigned d = static_cast<unsigned>((key[r] >> shift) & 255u);
      long long pos = offsets[static_cast<long long>(d) * ntiles + blockIdx.x] + wcnt[warp][d] + rank[r];
      keys_out[pos] = key[r];
      vals_out[pos] = val[r];
    }
  }
}

}  // namespace

size_t sort_hist_elems(long long n) {
  long long ntiles = (n + kSortTile - 1) / kSortTile;
  return static_cast<size_t>(256 * (ntiles > 0 ? ntiles : 1));
}

int radix_sort_pairs(SortBufs& b, long long n, unsigned digit_mask, cudaStream_t s,
                     cudaError_t* err) {
  *err = cudaSuccess;
  int cur = 0;
  if (n <= 1) return cur;
  const long long ntiles = (n + kSortTile - 1) / kSortTile;
  for (int digit = 0; digit < 8; ++digit) {
    if (!(digit_mask >> digit & 1u)) continue;
    const int shift = digit * 8;
    sort_hist_kernel<<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(b.keys[cur], n, shift,
                                                                          b.hist, ntiles);
    ++g_launches;
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return cur;
    *err = exclusive_scan_i64(b.hist, b.hist, 256 * ntiles, b.temp, s);
    if (*err != cudaSuccess) return cur;
    sort_scatter_kernel<<<static_cast<unsigned>(ntiles), kSortThreads, 0, s>>>(
        b.keys[cur], b.vals[cur], b.keys[cur ^ 1], b.vals[cur ^ 1], n, shift, b.hist, ntiles);
    ++g_launches;
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return cur;
    cur ^= 1;
  }
  return cur;
}

}  // namespace gc
