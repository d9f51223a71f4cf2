// ADG-O (Algorithm 6; Section 5, "Explicit Ordering in R"): ADG whose removed
// set R is numbered in increasing order of D, giving the total order
// rho(v) = (vertices removed in earlier iterations) + (v's place in the sorted
// R).  Algorithm 6's UPDATE also decrements the vertices that follow v in the
// same R, but their D is never read again, so the iterations remove exactly
// Algorithm 1's sets and D at removal is the degree adg_run reports.  Hence
// rho orders the vertices by (batch, D at removal, id) -- equal D by
// increasing id, a reading, as the paper leaves ties open -- and is obtained
// here by one stable radix sort of the keys batch * 2^32 + D over the ids in
// increasing order (constant digits skipped), in place of a counting sort of
// each R.  JP-ADG-O (JP with priority rho) needs no random tie-break: its key
// is the same batch * 2^32 + D with equal keys broken by the larger id, which
// gc_jp_color's exact order takes as given.
#include <cstring>

#include "gc_internal.cuh"

namespace gc {
namespace {

__device__ __forceinline__ long long o_tid() { return static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long o_stride() { return static_cast<long long>(gridDim.x) * blockDim.x; }

__global__ void __launch_bounds__(256)
adg_o_keys_kernel(const int* __restrict__ batch, const int* __restrict__ D, long long n,
                  unsigned long long* __restrict__ keys, int* __restrict__ vals, unsigned long long* orand) {
  unsigned long long kor = 0, kand = ~0ull;
  for (long long v = o_tid(); v < n; v += o_stride()) {
    const unsigned long long k = (static_cast<unsigned long long>(static_cast<unsigned>(batch[v])) << 32) |
                                 static_cast<unsigned>(D[v]);
    if (keys) {
      keys[v] = k;
      vals[v] = static_cast<int>(v);
    }
    kor |= k;
    kand &= k;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kor |= __shfl_xor_sync(kFull, kor, o);
    kand &= __shfl_xor_sync(kFull, kand, o);
  }
  if ((threadIdx.x & 31) == 0 && orand) {
    atomicOr(&orand[0], kor);
    atomicAnd(&orand[1], kand);
  }
}

// JP-ADG-O's priority key: batch * 2^32 + D
__global__ void __launch_bounds__(256)
adg_o_prio_kernel(const int* __restrict__ batch, const int* __restrict__ D, long long n,
                  unsigned long long* __restrict__ key) {
  for (long long v = o_tid(); v < n; v += o_stride())
    key[v] = (static_cast<unsigned long long>(static_cast<unsigned>(batch[v])) << 32) | static_cast<unsigned>(D[v]);
}

__global__ void __launch_bounds__(256)
adg_o_rho_kernel(const int* __restrict__ order, long long n, int* __restrict__ rho) {
  for (long long i = o_tid(); i < n; i += o_stride()) rho[order[i]] = static_cast<int>(i);
}

// rank(v): neighbours with a higher rho (Algorithm 6's UPDATEandPRIORITIZE
// count), one warp per vertex.
__global__ void __launch_bounds__(256)
adg_o_rank_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ col, const int* __restrict__ rho,
                  long long n, int* __restrict__ rank) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = o_stride() >> 5;
  for (long long v = o_tid() >> 5; v < n; v += nwarps) {
    const int rv = __ldg(rho + v);
    int c = 0;
    for (long long k = row_ptr[v] + lane; k < row_ptr[v + 1]; k += 32) c += __ldg(rho + __ldg(col + k)) > rv;
    c = warp_sum(c);
    if (lane == 0) rank[v] = c;
  }
}

}  // namespace

size_t adg_o_scratch_bytes(long long n) {
  const size_t hist = sort_hist_elems(n);
  const size_t t1 = scan_temp_elems(static_cast<long long>(hist));
  return 2 * (static_cast<size_t>(n) * 8 + 256) + 2 * (static_cast<size_t>(n) * 4 + 256) + hist * 8 + 256 +
         (t1 + 1) * 8 + 256 + 2 * 256;
}

gc_status adg_o_order(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D, int* rho,
                      int* rank, cudaStream_t s) {
  const long long n = g->n;
  if (n == 0) return GC_OK;
  SortBufs sb;
  sb.keys[0] = a.take<unsigned long long>(n);
  sb.keys[1] = a.take<unsigned long long>(n);
  sb.vals[0] = a.take<int>(n);
  sb.vals[1] = a.take<int>(n);
  sb.hist = a.take<long long>(sort_hist_elems(n));
  sb.temp = a.take<long long>(scan_temp_elems(static_cast<long long>(sort_hist_elems(n))) + 1);
  unsigned long long* orand = a.take<unsigned long long>(2);
  if (!sb.keys[0] || !sb.keys[1] || !sb.vals[0] || !sb.vals[1] || !sb.hist || !sb.temp || !orand) return GC_ERR_OOM;
  const unsigned long long init[2] = {0ull, ~0ull};
  unsigned long long* pin = static_cast<unsigned long long*>(ctx->pinned);
  memcpy(pin, init, sizeof(init));
  GC_TRY_CUDA(cudaMemcpyAsync(orand, pin, sizeof(init), cudaMemcpyHostToDevice, s));
  const int blocks = resident_grid(adg_o_keys_kernel, 256, ctx->num_sms);
  adg_o_keys_kernel<<<blocks, 256, 0, s>>>(batch, D, n, sb.keys[0], sb.vals[0], orand);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(cudaMemcpyAsync(pin, orand, sizeof(init), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  const unsigned long long diff = pin[0] ^ pin[1];
  unsigned mask = 0;
  for (int d = 0; d < 8; ++d)
    if ((diff >> (8 * d)) & 255ull) mask |= 1u << d;
  cudaError_t err;
  const int res = radix_sort_pairs(sb, n, mask, s, &err);
  GC_TRY_CUDA(err);
  adg_o_rho_kernel<<<blocks, 256, 0, s>>>(sb.vals[res], n, rho);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  if (rank) {
    const int rblocks = resident_grid(adg_o_rank_kernel, 256, ctx->num_sms);
    adg_o_rank_kernel<<<rblocks, 256, 0, s>>>(row_ptr_of(g), g->col_idx, rho, n, rank);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }
  return GC_OK;
}

cudaError_t adg_o_priority(const int* batch, const int* D, long long n, unsigned long long* key, int num_sms,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = resident_grid(adg_o_prio_kernel, 256, num_sms);
  adg_o_prio_kernel<<<blocks, 256, 0, s>>>(batch, D, n, key);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace gc
