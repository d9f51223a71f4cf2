// Autotuner: picks the context options (gc_options) that colour a given
// graph, or batch of graphs, fastest on this device.  The options change
// speed only, so every candidate must reproduce the colouring of the starting
// options exactly; the tuner checks that on the device after every trial.
//
// Search: coordinate descent.  Starting from the context's options, each
// dimension in turn (ADG's UPDATE direction and pull threshold -- the switch
// between the frontier-sparse push sweep and the dense pull sweep --, the
// number of hubs whose decrements UPDATE merges, the JP state word, the JP
// core's size, warps and cluster, the bulk kernel's blocks per SM, and for
// batches the persistent or segmented path) is set to
// each of its candidate values; a value is kept when its median time over
// `reps` runs (after one warm-up run) beats the best so far by more than 1%.
// The time of a run is taken with CUDA events on the caller's stream.
#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "gc_internal.cuh"

namespace gc {
namespace {

__global__ void count_diff_kernel(const int* __restrict__ a, const int* __restrict__ b, long long n,
                                  unsigned long long* __restrict__ diff) {
  unsigned long long d = 0;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    d += a[i] != b[i];
  d = warp_sum(d);
  if ((threadIdx.x & 31) == 0 && d) atomicAdd(diff, d);
}

struct Dim {
  std::function<void(gc_options&, int)> set;
  std::vector<int> values;
};

std::vector<Dim> dims_single(long long n) {
  std::vector<Dim> d;
  d.push_back({[](gc_options& o, int v) {
                 if (v < 0) {
                   o.update_mode = GC_UPDATE_PUSH;
                 } else {
                   o.update_mode = GC_UPDATE_AUTO;
                   o.pull_percent = v;
                 }
               },
               {-1, 25, 50, 100, 200}});
  d.push_back({[](gc_options& o, int v) { o.update_hubs = v; }, {0, 256, 512, 1024, 4096}});
  d.push_back({[](gc_options& o, int v) { o.jp_state16 = v; }, {0, 1}});
  std::vector<int> cores = {0, 4096, 8192, 16384, 24576, 32768};
  cores.erase(std::remove_if(cores.begin(), cores.end(), [n](int c) { return c > 0 && c / 2 >= n; }), cores.end());
  d.push_back({[](gc_options& o, int v) { o.core_target = v; }, cores});
  d.push_back({[](gc_options& o, int v) { o.core_warps = v; }, {4, 6, 8, 12}});
  d.push_back({[](gc_options& o, int v) { o.core_cluster = v; }, {4, 8, 16}});
  d.push_back({[](gc_options& o, int v) { o.bulk_blocks_per_sm = v; }, {0, 3, 4}});
  return d;
}

std::vector<Dim> dims_batch() {
  std::vector<Dim> d;
  d.push_back({[](gc_options& o, int v) { o.batch_mode = v; }, {GC_BATCH_PERSISTENT, GC_BATCH_SEGMENTED}});
  d.push_back({[](gc_options& o, int v) {
                 if (v < 0) {
                   o.update_mode = GC_UPDATE_PUSH;
                 } else {
                   o.update_mode = GC_UPDATE_AUTO;
                   o.pull_percent = v;
                 }
               },
               {-1, 25, 100}});
  d.push_back({[](gc_options& o, int v) { o.core_target = v; }, {0, 8192, 16384}});
  d.push_back({[](gc_options& o, int v) { o.bulk_blocks_per_sm = v; }, {0, 3}});
  return d;
}

}  // namespace

// Applies options to a context (they were range-checked by the caller) and
// forgets what was derived from the old ones.
void apply_options(gc_context* ctx, const gc_options& o) {
  ctx->opt = o;
  ctx->core_target = o.core_target;
  ctx->dec_tail = o.dec_tail != 0;
  ctx->wait_ns = static_cast<unsigned long long>(o.wait_limit_ms) * 1000000ull;
  ctx->core_cluster = 0;
  ctx->tail_cluster = 0;
}

// run(): one colouring into `out` (device, n ints) on stream s.
gc_status autotune(gc_context* ctx, long long n, const std::function<gc_status(int*)>& run, bool batch, int reps,
                   float budget_ms, gc_options* best_out, float* best_ms_out, float* start_ms_out, int* trials_out,
                   cudaStream_t s) {
  if (reps < 1) reps = 1;
  const size_t vb = (static_cast<size_t>(n > 0 ? n : 1) * 4 + 255) & ~size_t(255);
  void* buf = nullptr;
  if (ctx->fail_alloc || cudaMalloc(&buf, 2 * vb + 256) != cudaSuccess) {
    cudaGetLastError();
    return GC_ERR_OOM;
  }
  int* ref = static_cast<int*>(buf);
  int* out = reinterpret_cast<int*>(static_cast<char*>(buf) + vb);
  unsigned long long* diff = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 2 * vb);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gc_status st = GC_OK;
  const gc_options start = ctx->opt;
  gc_options best = start;
  float best_ms = 0.f, start_ms = 0.f, spent = 0.f;
  int trials = 0;
  auto time_it = [&](const gc_options& o, int* dst, float* ms) -> gc_status {
    apply_options(ctx, o);
    GC_TRY(run(dst));  // warm-up (also grows buffers)
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
      GC_TRY_CUDA(cudaEventRecord(e0, s));
      GC_TRY(run(dst));
      GC_TRY_CUDA(cudaEventRecord(e1, s));
      GC_TRY_CUDA(cudaEventSynchronize(e1));
      float x = 0.f;
      GC_TRY_CUDA(cudaEventElapsedTime(&x, e0, e1));
      t.push_back(x);
      spent += x;
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    ++trials;
    return GC_OK;
  };
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = GC_ERR_CUDA;
      break;
    }
    st = time_it(start, ref, &start_ms);
    if (st != GC_OK) break;
    best_ms = start_ms;
    const std::vector<Dim> dims = batch ? dims_batch() : dims_single(n);
    for (const Dim& d : dims) {
      for (int v : d.values) {
        if (budget_ms > 0.f && spent > budget_ms) break;
        gc_options o = best;
        d.set(o, v);
        if (memcmp(&o, &best, sizeof(o)) == 0) continue;
        float ms = 0.f;
        st = time_it(o, out, &ms);
        if (st != GC_OK) break;
        // the candidate must reproduce the starting options' colouring
        if (n > 0) {
          unsigned long long* pin = static_cast<unsigned long long*>(ctx->pinned);
          if ((st = gc_cuda_status(cudaMemsetAsync(diff, 0, sizeof(unsigned long long), s))) != GC_OK) break;
          count_diff_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(ref, out, n, diff);
          if ((st = gc_cuda_status(cudaGetLastError())) != GC_OK) break;
          if ((st = gc_cuda_status(cudaMemcpyAsync(pin, diff, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                                   s))) != GC_OK)
            break;
          if ((st = gc_cuda_status(cudaStreamSynchronize(s))) != GC_OK) break;
          if (*pin != 0) {  // options changed a result: a library defect, reported as such
            st = GC_ERR_CUDA;
            break;
          }
        }
        if (ms < best_ms * 0.99f) {
          best = o;
          best_ms = ms;
        }
      }
      if (st != GC_OK) break;
    }
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  apply_options(ctx, st == GC_OK ? best : start);
  if (st != GC_OK) return st;
  *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  if (start_ms_out) *start_ms_out = start_ms;
  if (trials_out) *trials_out = trials;
  return GC_OK;
}

}  // namespace gc
