// Smallest-last order for JP-SL (Section 4.1 combines JP with the SL
// ordering): repeatedly remove a vertex of minimum degree in the remaining
// graph; the paper leaves ties open and the vertex of minimum (current degree,
// id) is taken.  The priority of JP-SL is the removal index: the vertex
// removed last is coloured first.
//
// The order is inherently sequential -- each removal may lower the degree of
// the next candidate -- so it runs in ONE thread block that removes one
// vertex per step.  Each vertex's key (degree << 32 | id, all ones once
// removed) lives in global memory; the minimum key of every chunk of
// kSlChunk vertices lives in shared memory.  A step takes the minimum over the
// chunk minima (a block reduction), marks the vertex removed, lowers its
// neighbours' keys (atomicMin into their chunk minima) and recomputes the
// minimum of its own chunk (another block reduction).  The loop runs exactly
// n steps and waits on nothing.  One block of 1024 threads removes a vertex
// every few microseconds: about 4 s for 2^20 vertices.
#include <climits>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kSlThreads = 1024;
constexpr long long kSlChunk = 2048;
constexpr long long kSlMaxChunks = 16384;  // 128 KB of shared chunk minima: n <= 2^25
constexpr unsigned long long kGone = ~0ull;

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(kFull, v, o);
    v = u < v ? u : v;
  }
  return v;
}

// keys and chunk minima
__global__ void sl_init_kernel(const long long* __restrict__ row_ptr, long long n, unsigned long long* __restrict__ key,
                               unsigned long long* __restrict__ cmin) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long k = (static_cast<unsigned long long>(row_ptr[v + 1] - row_ptr[v]) << 32) |
                                 static_cast<unsigned long long>(v);
    key[v] = k;
    atomicMin(&cmin[v / kSlChunk], k);
  }
}

// Block-wide minimum of one value per thread (all threads call it).
__device__ __forceinline__ unsigned long long block_min(unsigned long long v, unsigned long long* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_min_u64(v);
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  v = lane < (kSlThreads / 32) ? s_red[lane] : kGone;
  v = warp_min_u64(v);
  __syncthreads();  // s_red may be reused by the next call
  return v;
}

__global__ void __launch_bounds__(kSlThreads, 1)
sl_order_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ col, long long n,
                unsigned long long* key, const unsigned long long* __restrict__ cmin_init, int* __restrict__ order,
                int* err) {
  extern __shared__ unsigned long long s_cmin[];
  __shared__ unsigned long long s_red[32];
  const int tid = threadIdx.x;
  const long long nch = (n + kSlChunk - 1) / kSlChunk;
  for (long long c = tid; c < nch; c += kSlThreads) s_cmin[c] = cmin_init[c];
  __syncthreads();
  for (long long i = 0; i < n; ++i) {
    unsigned long long m = kGone;
    for (long long c = tid; c < nch; c += kSlThreads) m = s_cmin[c] < m ? s_cmin[c] : m;
    const unsigned long long best = block_min(m, s_red);
    if (best == kGone) {  // no vertex left before n removals: cannot happen
      if (tid == 0) atomicExch(err, 1);
      return;
    }
    const int v = static_cast<int>(best & 0xffffffffull);
    if (tid == 0) {
      order[i] = v;
      key[v] = kGone;
    }
    // the remaining neighbours lose one degree (each neighbour once: a simple
    // graph has no duplicate edges, so no two threads update one key)
    const long long rs = row_ptr[v], re = row_ptr[v + 1];
    for (long long k = rs + tid; k < re; k += kSlThreads) {
      const int w = col[k];
      const unsigned long long kw = key[w];
      if (kw != kGone) {
        const unsigned long long nk = kw - (1ull << 32);
        key[w] = nk;
        atomicMin(&s_cmin[w / kSlChunk], nk);
      }
    }
    __syncthreads();
    // v's chunk lost v: its minimum over the chunk's keys again
    const long long c = v / kSlChunk, base = c * kSlChunk;
    unsigned long long cm = kGone;
    for (long long j = base + tid; j < base + kSlChunk && j < n; j += kSlThreads) {
      const unsigned long long kj = key[j];
      cm = kj < cm ? kj : cm;
    }
    cm = block_min(cm, s_red);
    if (tid == 0) s_cmin[c] = cm;
    __syncthreads();
  }
}

__global__ void sl_priority_kernel(const int* __restrict__ order, long long n, unsigned long long* __restrict__ prio) {
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    prio[order[i]] = static_cast<unsigned long long>(i);
}

}  // namespace

size_t sl_scratch_bytes(long long n) {
  const long long nch = (n + kSlChunk - 1) / kSlChunk;
  return (static_cast<size_t>(n > 0 ? n : 1) * 8 + 256) + (static_cast<size_t>(n > 0 ? n : 1) * 4 + 256) +
         (static_cast<size_t>(nch > 0 ? nch : 1) * 8 + 256) + 256;
}

// JP-SL keys: prio[v] = the index at which v is removed in the smallest-last
// order (minimum (degree, id) first).  GC_ERR_OVERFLOW above 2^25 vertices.
gc_status sl_priority(gc_context* ctx, Arena a, const gc_csr* g, unsigned long long* prio, cudaStream_t s) {
  const long long n = g->n;
  if (n == 0) return GC_OK;
  const long long nch = (n + kSlChunk - 1) / kSlChunk;
  if (nch > kSlMaxChunks) return GC_ERR_OVERFLOW;
  unsigned long long* key = a.take<unsigned long long>(n);
  int* order = a.take<int>(n);
  unsigned long long* cmin = a.take<unsigned long long>(nch);
  int* err = a.take<int>(1);
  if (!key || !order || !cmin || !err) return GC_ERR_OOM;
  const long long* rp = row_ptr_of(g);
  GC_TRY_CUDA(cudaMemsetAsync(cmin, 0xff, sizeof(unsigned long long) * nch, s));
  GC_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  sl_init_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(rp, n, key, cmin);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  const int smem = static_cast<int>(nch * sizeof(unsigned long long));
  GC_TRY_CUDA(cudaFuncSetAttribute(sl_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(kSlMaxChunks * sizeof(unsigned long long))));
  sl_order_kernel<<<1, kSlThreads, smem, s>>>(rp, g->col_idx, n, key, cmin, order, err);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  sl_priority_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(order, n, prio);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  int* pin = static_cast<int*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  return *pin ? GC_ERR_CUDA : GC_OK;
}

}  // namespace gc
