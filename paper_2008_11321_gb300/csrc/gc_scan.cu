// Device-wide exclusive prefix sum of int64 values (tiles of 4096 per block,
// block totals scanned recursively, then added back).  `in` may equal `out`.
#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr long long kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
scan_tile_kernel(const long long* in, long long* out, long long count, long long* block_sums) {
  __shared__ long long warp_tot[kScanThreads / kWarp];
  const long long base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  long long x[kScanItems];
  long long run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    long long idx = base + i;
    x[i] = idx < count ? in[idx] : 0;
    run += x[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = warp_inclusive_scan(run);
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long t = warp_tot[lane];
    long long ti = warp_inclusive_scan(t);
    warp_tot[lane] = ti - t;
    if (lane == 31 && block_sums) block_sums[blockIdx.x] = ti;
  }
  __syncthreads();
  long long prefix = warp_tot[warp] + incl - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    long long idx = base + i;
    if (idx < count) out[idx] = prefix;
    prefix += x[i];
  }
}

__global__ void scan_add_kernel(long long* __restrict__ out, long long count,
                                const long long* __restrict__ block_offsets) {
  const long long blk = blockIdx.x;
  const long long add = block_offsets[blk];
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    long long idx = blk * kScanTile + i;
    if (idx < count) out[idx] += add;
  }
}

}  // namespace

size_t scan_temp_elems(long long count) {
  long long nb = (count + kScanTile - 1) / kScanTile;
  if (nb <= 1) return 0;
  return static_cast<size_t>(nb) + scan_temp_elems(nb);
}

cudaError_t exclusive_scan_i64(const long long* in, long long* out, long long count,
                               long long* temp, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long nb = (count + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    scan_tile_kernel<<<1, kScanThreads, 0, s>>>(in, out, count, nullptr);
    ++g_launches;
    return cudaGetLastError();
  }
  long long* sums = temp;
  scan_tile_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, out, count, sums);
  ++g_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = exclusive_scan_i64(sums, sums, nb, temp + nb, s);
  if (e != cudaSuccess) return e;
  scan_add_kernel<<<static_cast<unsigned>(nb), 256, 0, s>>>(out, count, sums);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gc
