// C ABI entry points (gcolor.h): context management, argument checks, CSR
// validation, and the orchestration of the ADG and JP kernels.
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include <functional>

#include <algorithm>

#include "gc_internal.cuh"

namespace gc {
thread_local int g_launches = 0;
thread_local char g_last_error[256] = "";

void note_cuda_error(cudaError_t e, const char* file, int line) {
  const char* base = strrchr(file, '/');
  snprintf(g_last_error, sizeof(g_last_error), "%s:%d: %s (%s)", base ? base + 1 : file, line, cudaGetErrorName(e),
           cudaGetErrorString(e));
}
}  // namespace gc

namespace {

constexpr uint32_t kEpsMax = 1u << 20;

// Per-call bookkeeping: resets the launch counter on entry and stores it in
// the context's statistics on exit.
struct CallScope {
  gc_context* ctx;
  explicit CallScope(gc_context* c) : ctx(c) {
    gc::g_launches = 0;
    ctx->tused = 0;
    ctx->stats.bulk_launches = 0;
    ctx->stats.core_vertices = 0;
    ctx->stats.core_preds = 0;
    ctx->stats.core_degree_sum = 0;
    ctx->stats.core_ctas = 0;
    ctx->stats.sim_iterations = 0;
    ctx->stats.dec_internal_edges = 0;
    ctx->stats.dec_tail_partitions = 0;
    ctx->stats.jp_state_bits = 0;
    ctx->stats.batch_path = 0;
  }
  ~CallScope() {
    if (!ctx) return;
    ctx->stats.launches = gc::g_launches;
    if (ctx->timing) {
      if (ctx->tused > 0) cudaEventSynchronize(ctx->tev[2 * ctx->tused - 1]);
      ctx->timers_collect();
    }
  }
};

// Make the context's device current for the scope, restore the caller's after.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

gc_status check_graph_args(const gc_csr* g) {
  if (!g) return GC_ERR_INVALID_ARG;
  if (g->n < 0 || g->nnz < 0 || g->n > static_cast<int64_t>(INT_MAX) - 1) return GC_ERR_INVALID_ARG;
  if (g->n > 0 && !row_ptr_of(g)) return GC_ERR_INVALID_ARG;
  if (g->nnz > 0 && !g->col_idx) return GC_ERR_INVALID_ARG;
  return GC_OK;
}

gc_status check_eps(uint32_t p, uint32_t q) {
  if (q == 0 || q > kEpsMax || p > kEpsMax) return GC_ERR_INVALID_ARG;
  return GC_OK;
}

// ---- CSR validation kernels ------------------------------------------------

__global__ void validate_rows_kernel(const long long* __restrict__ row_ptr, long long n, long long nnz,
                                     int* bad) {
  for (long long u = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; u <= n;
       u += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long r = row_ptr[u];
    if (u == 0 && r != 0) atomicExch(bad, 1);
    if (u == n && r != nnz) atomicExch(bad, 1);
    if (u < n) {
      const long long r1 = row_ptr[u + 1];
      if (r1 < r || r1 > nnz || r < 0) atomicExch(bad, 1);
    }
  }
}

__device__ bool row_contains(const int* col, long long s, long long e, int key) {
  while (s < e) {
    long long mid = s + ((e - s) >> 1);
    int x = col[mid];
    if (x == key) return true;
    if (x < key)
      s = mid + 1;
    else
      e = mid;
  }
  return false;
}

// One warp per row: ids in range, no self-loop, strictly increasing rows,
// and the reverse edge present.  Runs only after validate_rows_kernel passed.
__global__ void validate_edges_kernel(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                                      long long n, int* bad) {
  const int lane = threadIdx.x & 31;
  const long long gwarp = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = (static_cast<long long>(gridDim.x) * blockDim.x) >> 5;
  for (long long u = gwarp; u < n; u += nwarps) {
    const long long s = row_ptr[u], e = row_ptr[u + 1];
    for (long long k = s + lane; k < e; k += 32) {
      const int w = col[k];
      bool ok = w >= 0 && w < n && w != u;
      if (ok && k + 1 < e) ok = col[k + 1] > w;
      if (ok) ok = row_contains(col, row_ptr[w], row_ptr[w + 1], static_cast<int>(u));
      if (!ok) atomicExch(bad, 1);
    }
  }
}

gc_status timing_begin(gc_context* ctx, int idx, cudaStream_t s) {
  if (!ctx->timing) return GC_OK;
  GC_TRY_CUDA(cudaEventRecord(ctx->ev[idx], s));
  return GC_OK;
}

float timing_ms(gc_context* ctx, int a, int b) {
  float ms = 0.f;
  if (!ctx->timing) return 0.f;
  if (cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) != cudaSuccess) return 0.f;
  return ms;
}

// Upload by the SMs: 16-byte loads of mapped page-locked host memory (over
// the CPU-GPU link), four in flight per thread, stored to device memory.
__global__ void __launch_bounds__(256) host_copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                        long long n16) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

// Host -> device copy of `bytes`: by host_copy_kernel when asked for and the
// host buffer is page-locked and mapped with 16-byte alignment, else by the
// copy engine (cudaMemcpyAsync).
gc_status upload(gc_context* ctx, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return GC_OK;
  if (ctx->opt.host_upload == 1) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
        (reinterpret_cast<uintptr_t>(at.devicePointer) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
      const long long n16 = static_cast<long long>(bytes / 16);
      if (n16 > 0) {
        host_copy_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(static_cast<const uint4*>(at.devicePointer),
                                                          static_cast<uint4*>(dst), n16);
        ++gc::g_launches;
        GC_TRY_CUDA(cudaGetLastError());
      }
      const size_t done = static_cast<size_t>(n16) * 16;
      if (bytes > done)
        GC_TRY_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + done, static_cast<const char*>(src) + done,
                                    bytes - done, cudaMemcpyHostToDevice, s));
      return GC_OK;
    }
    cudaGetLastError();  // (an unregistered pointer is not an error to keep)
  }
  GC_TRY_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  return GC_OK;
}

// gc_color_graph_host copies col_idx in ranges (on the context's copy stream)
// from this many entries on.
constexpr int64_t kChunkedUploadMin = int64_t(1) << 22;

gc_status copy_stream_ready(gc_context* ctx) {
  if (!ctx->copy_stream &&
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->copy_stream = nullptr;
    return gc_cuda_status(cudaGetLastError());
  }
  for (auto& e : ctx->copy_ev)
    if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      e = nullptr;
      return gc_cuda_status(cudaGetLastError());
    }
  return GC_OK;
}

// Shared body of gc_color_graph and gc_color_graph_host.
// JP-ADG (median = false) or JP-ADG-M (median = true, p and q unused).
gc_status color_graph_device(gc_context* ctx, const gc_csr* g, uint32_t p, uint32_t q, uint64_t seed,
                             int32_t* color, int32_t* batch, int32_t* ncol, int32_t* nrounds,
                             cudaStream_t s, bool median = false, const gc::ColChunks* chunks = nullptr) {
  const long long n = g->n;
  const size_t vb = static_cast<size_t>(n > 0 ? n : 1) * 4 + 256;
  GC_TRY(ctx->reserve_vert(2 * vb));
  int* D = static_cast<int*>(ctx->vbuf);
  int* b = batch ? batch : reinterpret_cast<int*>(static_cast<char*>(ctx->vbuf) + vb);
  GC_TRY(ctx->reserve(median ? gc::adg_m_scratch_bytes(n, g->nnz) : gc::adg_scratch_bytes(n, g->nnz)));
  int rounds = 0, colors = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  if (median)
    GC_TRY(gc::adg_m_run(ctx, ctx->arena(), g, b, D, &rounds, s));
  else
    GC_TRY(gc::adg_run(ctx, ctx->arena(), g, p, q, b, D, &rounds, s, chunks));
  GC_TRY(timing_begin(ctx, 1, s));
  GC_TRY(ctx->reserve(gc::jpadg_scratch_bytes(n, g->nnz, rounds)));
  GC_TRY(gc::jp_run_fused(ctx, ctx->arena(), g, b, D, rounds, seed, color, &colors, s));
  GC_TRY(timing_begin(ctx, 2, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[2]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
    ctx->stats.ms_jp = timing_ms(ctx, 1, 2);
  }
  if (ncol) *ncol = colors;
  if (nrounds) *nrounds = rounds;
  return GC_OK;
}

}  // namespace

namespace {
// Grow a device buffer to at least `bytes` (contents are not kept).
gc_status grow(void** buf, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return GC_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  const size_t want = bytes + bytes / 8;
  if (cudaMalloc(buf, want) != cudaSuccess) {
    *buf = nullptr;
    cudaGetLastError();
    return GC_ERR_OOM;
  }
  *cap = want;
  return GC_OK;
}
}  // namespace

gc_status gc_context::reserve(size_t bytes) {
  return fail_alloc ? GC_ERR_OOM : grow(&scratch, &scratch_bytes, bytes);
}
gc_status gc_context::reserve_vert(size_t bytes) { return fail_alloc ? GC_ERR_OOM : grow(&vbuf, &vbuf_bytes, bytes); }
gc_status gc_context::reserve_aux(size_t bytes) { return fail_alloc ? GC_ERR_OOM : grow(&aux, &aux_bytes, bytes); }
gc_status gc_context::reserve_pack(size_t bytes) { return fail_alloc ? GC_ERR_OOM : grow(&pack, &pack_bytes, bytes); }

extern "C" {

const char* gc_last_error(void) { return gc::g_last_error; }

const char* gc_status_str(gc_status s) {
  switch (s) {
    case GC_OK: return "GC_OK";
    case GC_ERR_INVALID_ARG: return "GC_ERR_INVALID_ARG";
    case GC_ERR_INVALID_GRAPH: return "GC_ERR_INVALID_GRAPH";
    case GC_ERR_OOM: return "GC_ERR_OOM";
    case GC_ERR_CUDA: return "GC_ERR_CUDA";
    case GC_ERR_TIMEOUT: return "GC_ERR_TIMEOUT";
    case GC_ERR_OVERFLOW: return "GC_ERR_OVERFLOW";
  }
  return "GC_ERR_UNKNOWN";
}

gc_status gc_options_init(gc_options* opt) {
  if (!opt) return GC_ERR_INVALID_ARG;
  gc_options o{};
  o.struct_size = sizeof(gc_options);
  o.core_target = static_cast<int32_t>(gc::kCoreDefault);
  o.core_cluster = 16;
  o.core_warps = 12;
  o.dec_tail = 1;
  o.update_mode = GC_UPDATE_AUTO;
  o.pull_percent = 25;
  o.bulk_blocks_per_sm = 0;
  o.wait_limit_ms = static_cast<uint32_t>(gc::kWaitLimitNs / 1000000ull);
  o.jp_state16 = 0;
  o.batch_mode = GC_BATCH_AUTO;
  o.update_hubs = 512;
  o.host_upload = 1;
  o.round_graph = 1;
  *opt = o;
  return GC_OK;
}

}  // extern "C"

namespace {
// Options as the library uses them: defaults, overwritten by the prefix of
// the struct the caller knows, then range-checked.
gc_status read_options(const gc_options* opt, gc_options* out) {
  gc_options o;
  gc_options_init(&o);
  if (opt) {
    if (opt->struct_size < sizeof(uint32_t) || opt->struct_size > sizeof(gc_options)) return GC_ERR_INVALID_ARG;
    memcpy(reinterpret_cast<char*>(&o) + sizeof(uint32_t), reinterpret_cast<const char*>(opt) + sizeof(uint32_t),
           opt->struct_size - sizeof(uint32_t));
    o.struct_size = sizeof(gc_options);
  }
  if (o.core_target < 0 || o.core_target > gc::kCoreMax || o.core_cluster < 1 || o.core_cluster > 16 ||
      o.core_warps < 1 || o.core_warps > 32 || (o.dec_tail != 0 && o.dec_tail != 1) ||
      o.update_mode < GC_UPDATE_AUTO || o.update_mode > GC_UPDATE_PULL || o.pull_percent < 0 ||
      o.pull_percent > 100000 || o.bulk_blocks_per_sm < 0 || o.bulk_blocks_per_sm > 32 || o.wait_limit_ms < 1 ||
      o.wait_limit_ms > 600000 || (o.jp_state16 != 0 && o.jp_state16 != 1) || o.batch_mode < GC_BATCH_AUTO ||
      o.batch_mode > GC_BATCH_PERSISTENT || o.update_hubs < 0 || o.update_hubs > 4096 ||
      (o.host_upload != 0 && o.host_upload != 1) || (o.round_graph != 0 && o.round_graph != 1))
    return GC_ERR_INVALID_ARG;
  *out = o;
  return GC_OK;
}
}  // namespace

extern "C" {

gc_status gc_create(gc_context** out, int device, const gc_options* opt) {
  if (!out) return GC_ERR_INVALID_ARG;
  *out = nullptr;
  gc_options o;
  GC_TRY(read_options(opt, &o));
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return GC_ERR_CUDA;
  }
  if (device < 0 || device >= count) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return GC_ERR_CUDA;
  gc_context* ctx = new (std::nothrow) gc_context();
  if (!ctx) return GC_ERR_OOM;
  ctx->device = device;
  gc::apply_options(ctx, o);
  // failure injection for tests of the error paths (see gc_context)
  if (const char* env = getenv("GC_INJECT_STALL")) ctx->stall_vertex = atoi(env);
  if (const char* env = getenv("GC_INJECT_OOM")) ctx->fail_alloc = env[0] != '\0' && env[0] != '0';
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess) {
    delete ctx;
    return GC_ERR_CUDA;
  }
  if (cudaMallocHost(&ctx->pinned, 256) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return GC_ERR_OOM;
  }
  for (auto& ev : ctx->ev) {
    if (cudaEventCreate(&ev) != cudaSuccess) {
      gc_destroy(ctx);
      return GC_ERR_CUDA;
    }
  }
  for (auto& ev : ctx->tev) {
    if (cudaEventCreate(&ev) != cudaSuccess) {
      gc_destroy(ctx);
      return GC_ERR_CUDA;
    }
  }
  *out = ctx;
  return GC_OK;
}

void gc_destroy(gc_context* ctx) {
  if (!ctx) return;
  DeviceGuard guard(ctx->device);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->vbuf) cudaFree(ctx->vbuf);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->pack) cudaFree(ctx->pack);
  if (ctx->h_graph) cudaFree(ctx->h_graph);
  gc::loop_graph_free(&ctx->adg_graph);
  gc::loop_graph_free(&ctx->batch_graph);
  for (auto& e : ctx->copy_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (auto& ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : ctx->tev)
    if (ev) cudaEventDestroy(ev);
  delete ctx;
}

gc_status gc_get_options(const gc_context* ctx, gc_options* out) {
  if (!ctx || !out) return GC_ERR_INVALID_ARG;
  *out = ctx->opt;
  return GC_OK;
}

gc_status gc_set_options(gc_context* ctx, const gc_options* opt) {
  if (!ctx || !opt) return GC_ERR_INVALID_ARG;
  gc_options o;
  GC_TRY(read_options(opt, &o));
  gc::apply_options(ctx, o);
  return GC_OK;
}

gc_status gc_autotune(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q, uint64_t seed, int32_t reps,
                      float budget_ms, gc_options* best_out, float* best_ms_out, float* start_ms_out,
                      gc_stream stream) {
  if (!ctx || !best_out) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int timing = ctx->timing;
  ctx->timing = 0;
  const gc_status st = gc::autotune(
      ctx, g->n,
      [&](int* out) { return color_graph_device(ctx, g, eps_p, eps_q, seed, out, nullptr, nullptr, nullptr, s); },
      false, reps, budget_ms, best_out, best_ms_out, start_ms_out, nullptr, s);
  ctx->timing = timing;
  return st;
}

gc_status gc_autotune_batch(gc_context* ctx, const gc_batch_csr* b, const gc_job* jobs, int32_t reps,
                            float budget_ms, gc_options* best_out, float* best_ms_out, float* start_ms_out,
                            gc_stream stream) {
  if (!ctx || !b || !jobs || !best_out || b->num_graphs < 1 || b->num_graphs > INT_MAX || !b->graph_off)
    return GC_ERR_INVALID_ARG;
  if (b->n < 0 || b->nnz < 0 || b->n > static_cast<int64_t>(INT_MAX) - 1) return GC_ERR_INVALID_ARG;
  if (b->n > 0 && !b->row_ptr) return GC_ERR_INVALID_ARG;
  if (b->nnz > 0 && !b->col_idx) return GC_ERR_INVALID_ARG;
  for (int64_t g = 0; g < b->num_graphs; ++g) GC_TRY(check_eps(jobs[g].eps_p, jobs[g].eps_q));
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int timing = ctx->timing;
  ctx->timing = 0;
  const gc_status st = gc::autotune(
      ctx, b->n, [&](int* out) { return gc::batch_color(ctx, b, jobs, out, nullptr, nullptr, nullptr, s); }, true,
      reps, budget_ms, best_out, best_ms_out, start_ms_out, nullptr, s);
  ctx->timing = timing;
  return st;
}

gc_status gc_get_stats(const gc_context* ctx, gc_stats* out) {
  if (!ctx || !out) return GC_ERR_INVALID_ARG;
  *out = ctx->stats;
  return GC_OK;
}

gc_status gc_set_timing(gc_context* ctx, int enable) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return GC_OK;
}

gc_status gc_validate_csr(gc_context* ctx, const gc_csr* g, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g->n == 0) return g->nnz == 0 ? GC_OK : GC_ERR_INVALID_GRAPH;
  GC_TRY(ctx->reserve(256));
  int* bad = static_cast<int*>(ctx->scratch);
  int* pin = static_cast<int*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  validate_rows_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(row_ptr_of(g), g->n, g->nnz, bad);
  ++gc::g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(cudaMemcpyAsync(pin, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  if (*pin) return GC_ERR_INVALID_GRAPH;
  if (g->nnz == 0) return GC_OK;
  validate_edges_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(row_ptr_of(g), g->col_idx, g->n, bad);
  ++gc::g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  GC_TRY_CUDA(cudaMemcpyAsync(pin, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  return *pin ? GC_ERR_INVALID_GRAPH : GC_OK;
}

gc_status gc_adg_partition(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q,
                           int32_t* batch_out, int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx || !num_rounds_out) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  if (g->n > 0 && !batch_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GC_TRY(ctx->reserve(gc::adg_scratch_bytes(g->n, g->nnz)));
  GC_TRY(ctx->reserve_vert(static_cast<size_t>(g->n > 0 ? g->n : 1) * 4 + 256));
  int rounds = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  GC_TRY(gc::adg_run(ctx, ctx->arena(), g, eps_p, eps_q, batch_out, static_cast<int*>(ctx->vbuf),
                     &rounds, s));
  GC_TRY(timing_begin(ctx, 1, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[1]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
  }
  *num_rounds_out = rounds;
  return GC_OK;
}

gc_status gc_make_priority(gc_context* ctx, int64_t n, const int32_t* batch, uint64_t seed,
                           uint64_t* key_out, gc_stream stream) {
  if (!ctx || n < 0 || n > static_cast<int64_t>(INT_MAX) - 1) return GC_ERR_INVALID_ARG;
  if (n > 0 && (!batch || !key_out)) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  GC_TRY_CUDA(gc::make_priority(batch, n, seed, reinterpret_cast<unsigned long long*>(key_out),
                                ctx->num_sms, reinterpret_cast<cudaStream_t>(stream)));
  return GC_OK;
}

gc_status gc_make_priority_kind(gc_context* ctx, const gc_csr* g, int32_t kind, uint64_t seed, uint64_t* key_out,
                                gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  if (kind < GC_PRIO_R || kind > GC_PRIO_SL) return GC_ERR_INVALID_ARG;
  if (g->n > 0 && !key_out) return GC_ERR_INVALID_ARG;
  if (kind == GC_PRIO_SL && g->n > (1ll << 25)) return GC_ERR_OVERFLOW;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  if (kind == GC_PRIO_SL) {
    GC_TRY(ctx->reserve(gc::sl_scratch_bytes(g->n)));
    return gc::sl_priority(ctx, ctx->arena(), g, reinterpret_cast<unsigned long long*>(key_out),
                           reinterpret_cast<cudaStream_t>(stream));
  }
  GC_TRY_CUDA(gc::make_priority_kind(row_ptr_of(g), g->n, kind, seed, reinterpret_cast<unsigned long long*>(key_out),
                                     ctx->num_sms, reinterpret_cast<cudaStream_t>(stream)));
  return GC_OK;
}

gc_status gc_jp_color(gc_context* ctx, const gc_csr* g, const uint64_t* priority, int32_t* color_out,
                      int32_t* num_colors_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  if (g->n > 0 && (!priority || !color_out)) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GC_TRY(ctx->reserve(gc::jp_scratch_bytes(g->n, g->nnz)));
  int colors = 0;
  GC_TRY(timing_begin(ctx, 1, s));
  GC_TRY(gc::jp_run_given(ctx, ctx->arena(), g, reinterpret_cast<const unsigned long long*>(priority),
                          color_out, &colors, s));
  GC_TRY(timing_begin(ctx, 2, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[2]));
    ctx->stats.ms_jp = timing_ms(ctx, 1, 2);
  }
  if (num_colors_out) *num_colors_out = colors;
  return GC_OK;
}

gc_status gc_color_graph(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q,
                         uint64_t seed, int32_t* color_out, int32_t* batch_out,
                         int32_t* num_colors_out, int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  if (g->n > 0 && !color_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  return color_graph_device(ctx, g, eps_p, eps_q, seed, color_out, batch_out, num_colors_out,
                            num_rounds_out, reinterpret_cast<cudaStream_t>(stream));
}

gc_status gc_adg_m_partition(gc_context* ctx, const gc_csr* g, int32_t* batch_out, int32_t* num_rounds_out,
                             gc_stream stream) {
  if (!ctx || !num_rounds_out) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  if (g->n > 0 && !batch_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GC_TRY(ctx->reserve(gc::adg_m_scratch_bytes(g->n, g->nnz)));
  GC_TRY(ctx->reserve_vert(static_cast<size_t>(g->n > 0 ? g->n : 1) * 4 + 256));
  int rounds = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  GC_TRY(gc::adg_m_run(ctx, ctx->arena(), g, batch_out, static_cast<int*>(ctx->vbuf), &rounds, s));
  GC_TRY(timing_begin(ctx, 1, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[1]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
  }
  *num_rounds_out = rounds;
  return GC_OK;
}

gc_status gc_color_graph_m(gc_context* ctx, const gc_csr* g, uint64_t seed, int32_t* color_out, int32_t* batch_out,
                           int32_t* num_colors_out, int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  if (g->n > 0 && !color_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  return color_graph_device(ctx, g, 0, 1, seed, color_out, batch_out, num_colors_out, num_rounds_out,
                            reinterpret_cast<cudaStream_t>(stream), true);
}

gc_status gc_adg_o_order(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q, int32_t* batch_out,
                         int32_t* rho_out, int32_t* rank_out, int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  if (g->n > 0 && !rho_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = g->n;
  const size_t vb = static_cast<size_t>(n > 0 ? n : 1) * 4 + 256;
  GC_TRY(ctx->reserve_vert(2 * vb));
  int* D = static_cast<int*>(ctx->vbuf);
  int* b = batch_out ? batch_out : reinterpret_cast<int*>(static_cast<char*>(ctx->vbuf) + vb);
  GC_TRY(ctx->reserve(gc::adg_scratch_bytes(n, g->nnz)));
  int rounds = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  GC_TRY(gc::adg_run(ctx, ctx->arena(), g, eps_p, eps_q, b, D, &rounds, s));
  GC_TRY(ctx->reserve(gc::adg_o_scratch_bytes(n)));
  GC_TRY(gc::adg_o_order(ctx, ctx->arena(), g, b, D, rho_out, rank_out, s));
  GC_TRY(timing_begin(ctx, 1, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[1]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
  }
  if (num_rounds_out) *num_rounds_out = rounds;
  return GC_OK;
}

gc_status gc_color_graph_o(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q, int32_t* color_out,
                           int32_t* batch_out, int32_t* num_colors_out, int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  if (g->n > 0 && !color_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = g->n;
  const size_t vb = static_cast<size_t>(n > 0 ? n : 1) * 4 + 256;
  GC_TRY(ctx->reserve_vert(2 * vb));
  int* D = static_cast<int*>(ctx->vbuf);
  int* b = batch_out ? batch_out : reinterpret_cast<int*>(static_cast<char*>(ctx->vbuf) + vb);
  GC_TRY(ctx->reserve(gc::adg_scratch_bytes(n, g->nnz)));
  int rounds = 0, colors = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  GC_TRY(gc::adg_run(ctx, ctx->arena(), g, eps_p, eps_q, b, D, &rounds, s));
  GC_TRY(timing_begin(ctx, 1, s));
  // JP scratch (and a key array beyond 255 iterations) after ADG's, which is dead
  const size_t key_bytes = (static_cast<size_t>(n > 0 ? n : 1) * 8 + 255) & ~size_t(255);
  GC_TRY(ctx->reserve(key_bytes + gc::jp_scratch_bytes(n, g->nnz)));
  GC_TRY(gc::jp_run_ordered(ctx, ctx->arena(), g, b, D, rounds, color_out, &colors, s));
  GC_TRY(timing_begin(ctx, 2, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[2]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
    ctx->stats.ms_jp = timing_ms(ctx, 1, 2);
  }
  ctx->stats.adg_rounds = rounds;
  if (num_colors_out) *num_colors_out = colors;
  if (num_rounds_out) *num_rounds_out = rounds;
  return GC_OK;
}

gc_status gc_dec_itr_color(gc_context* ctx, const gc_csr* g, const int32_t* batch, int32_t num_rounds,
                           uint64_t seed, int32_t* color_out, int32_t* num_colors_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  if (g->n > 0 && (!batch || !color_out || num_rounds < 1)) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GC_TRY(ctx->reserve(gc::dec_scratch_bytes(g->n, g->nnz, num_rounds)));
  int colors = 0;
  long long iters = 0;
  GC_TRY(timing_begin(ctx, 1, s));
  GC_TRY(gc::dec_itr_run(ctx, ctx->arena(), g, batch, num_rounds, seed, color_out, &colors, &iters, s));
  GC_TRY(timing_begin(ctx, 2, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[2]));
    ctx->stats.ms_jp = timing_ms(ctx, 1, 2);
  }
  ctx->stats.num_colors = colors;
  ctx->stats.sim_iterations = iters;
  if (num_colors_out) *num_colors_out = colors;
  return GC_OK;
}

gc_status gc_color_graph_dec_itr(gc_context* ctx, const gc_csr* g, uint32_t eps_p, uint32_t eps_q, uint64_t seed,
                                 int32_t* color_out, int32_t* batch_out, int32_t* num_colors_out,
                                 int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx) return GC_ERR_INVALID_ARG;
  GC_TRY(check_graph_args(g));
  GC_TRY(check_eps(eps_p, eps_q));
  if (g->n > 0 && !color_out) return GC_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = g->n;
  const size_t vb = static_cast<size_t>(n > 0 ? n : 1) * 4 + 256;
  GC_TRY(ctx->reserve_vert(2 * vb));
  int* D = static_cast<int*>(ctx->vbuf);
  int* b = batch_out ? batch_out : reinterpret_cast<int*>(static_cast<char*>(ctx->vbuf) + vb);
  GC_TRY(ctx->reserve(gc::adg_scratch_bytes(n, g->nnz)));
  int rounds = 0, colors = 0;
  long long iters = 0;
  GC_TRY(timing_begin(ctx, 0, s));
  GC_TRY(gc::adg_run(ctx, ctx->arena(), g, eps_p, eps_q, b, D, &rounds, s));
  GC_TRY(timing_begin(ctx, 1, s));
  GC_TRY(ctx->reserve(gc::dec_scratch_bytes(n, g->nnz, rounds)));
  GC_TRY(gc::dec_itr_run(ctx, ctx->arena(), g, b, rounds, seed, color_out, &colors, &iters, s));
  GC_TRY(timing_begin(ctx, 2, s));
  if (ctx->timing) {
    GC_TRY_CUDA(cudaEventSynchronize(ctx->ev[2]));
    ctx->stats.ms_adg = timing_ms(ctx, 0, 1);
    ctx->stats.ms_jp = timing_ms(ctx, 1, 2);
  }
  ctx->stats.num_colors = colors;
  ctx->stats.sim_iterations = iters;
  if (num_colors_out) *num_colors_out = colors;
  if (num_rounds_out) *num_rounds_out = rounds;
  return GC_OK;
}

gc_status gc_color_graph_host(gc_context* ctx, int64_t n, int64_t nnz, const int64_t* row_ptr,
                              const int32_t* col_idx, uint32_t eps_p, uint32_t eps_q, uint64_t seed,
                              int32_t* color_out, int32_t* batch_out, int32_t* num_colors_out,
                              int32_t* num_rounds_out, gc_stream stream) {
  if (!ctx || n < 0 || nnz < 0 || n > static_cast<int64_t>(INT_MAX) - 1) return GC_ERR_INVALID_ARG;
  if (!row_ptr || (nnz > 0 && !col_idx) || (n > 0 && !color_out)) return GC_ERR_INVALID_ARG;
  GC_TRY(check_eps(eps_p, eps_q));
  DeviceGuard guard(ctx->device);
  CallScope scope(ctx);
  if (!guard.ok) return GC_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // context-owned device copies: row_ptr | col_idx | color | batch
  const size_t b_rp = (static_cast<size_t>(n + 1) * 8 + 255) & ~size_t(255);
  const size_t b_ci = (static_cast<size_t>(nnz) * 4 + 255) & ~size_t(255);
  const size_t b_v = (static_cast<size_t>(n) * 4 + 255) & ~size_t(255);
  const size_t need = b_rp + b_ci + 2 * b_v + 256;
  if (need > ctx->h_graph_bytes) {
    if (ctx->h_graph) cudaFree(ctx->h_graph);
    ctx->h_graph = nullptr;
    ctx->h_graph_bytes = 0;
    if (cudaMalloc(&ctx->h_graph, need) != cudaSuccess) {
      cudaGetLastError();
      return GC_ERR_OOM;
    }
    ctx->h_graph_bytes = need;
  }
  char* base = static_cast<char*>(ctx->h_graph);
  gc_csr g;
  g.n = n;
  g.nnz = nnz;
  g.row_ptr = reinterpret_cast<const int64_t*>(base);
  g.col_idx = reinterpret_cast<const int32_t*>(base + b_rp);
  int32_t* d_color = reinterpret_cast<int32_t*>(base + b_rp + b_ci);
  int32_t* d_batch = reinterpret_cast<int32_t*>(base + b_rp + b_ci + b_v);
  GC_TRY(upload(ctx, const_cast<int64_t*>(g.row_ptr), row_ptr, static_cast<size_t>(n + 1) * 8, s));
  // col_idx in vertex ranges of about equal size on the context's copy
  // stream (by the copy engine, or by the SM copy with host_upload), so that
  // ADG's first round starts on the ranges already copied; small graphs take
  // one copy on s
  gc::ColChunks chunks;
  if (nnz >= kChunkedUploadMin) {
    GC_TRY(copy_stream_ready(ctx));
    GC_TRY_CUDA(cudaEventRecord(ctx->copy_ev[gc::kUploadChunks], s));  // earlier work on s is done with the buffers
    GC_TRY_CUDA(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev[gc::kUploadChunks], 0));
    chunks.k = gc::kUploadChunks;
    chunks.lo[0] = 0;
    for (int c = 1; c < chunks.k; ++c) {
      // the first vertex whose row starts at or after c/k of the entries
      const int64_t target = nnz / chunks.k * c;
      chunks.lo[c] = std::lower_bound(row_ptr, row_ptr + n + 1, target) - row_ptr;
      if (chunks.lo[c] < chunks.lo[c - 1]) chunks.lo[c] = chunks.lo[c - 1];
      if (chunks.lo[c] > n) chunks.lo[c] = n;
    }
    chunks.lo[chunks.k] = n;
    // entry ranges: each range's first row start rounded up to 4 entries (16
    // bytes, so the SM copy keeps its alignment; a range then also carries
    // the first entries of the next one), kept within [0, nnz) and
    // increasing, so that the copies cover the entries exactly once
    // whatever row_ptr holds
    int64_t pos[gc::kUploadChunks + 1];
    pos[0] = 0;
    pos[chunks.k] = nnz;
    for (int c = 1; c < chunks.k; ++c)
      pos[c] = std::min<int64_t>((std::max<int64_t>(row_ptr[chunks.lo[c]], pos[c - 1]) + 3) & ~int64_t(3), nnz);
    for (int c = 0; c < chunks.k; ++c) {
      const int64_t a = pos[c], b = pos[c + 1];
      if (b > a)
        GC_TRY(upload(ctx, const_cast<int32_t*>(g.col_idx) + a, col_idx + a, static_cast<size_t>(b - a) * 4,
                      ctx->copy_stream));
      GC_TRY_CUDA(cudaEventRecord(ctx->copy_ev[c], ctx->copy_stream));
      chunks.ready[c] = ctx->copy_ev[c];
    }
  } else if (nnz > 0) {
    GC_TRY(upload(ctx, const_cast<int32_t*>(g.col_idx), col_idx, static_cast<size_t>(nnz) * 4, s));
  }
  GC_TRY(color_graph_device(ctx, &g, eps_p, eps_q, seed, d_color, d_batch, num_colors_out, num_rounds_out, s,
                            false, chunks.k > 0 ? &chunks : nullptr));
  if (n > 0) {
    GC_TRY_CUDA(cudaMemcpyAsync(color_out, d_color, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
    if (batch_out)
      GC_TRY_CUDA(cudaMemcpyAsync(batch_out, d_batch, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
  }
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  return GC_OK;
}

gc_status gc_color_batch(gc_context* ctx, const gc_batch_csr* b, const gc_job* jobs, int32_t* color_out,
                         int32_t* batch_out, int32_t* num_colors_out, int32_t* num_rounds_out,
                         gc_stream stream) {
  if (!ctx || !b || b->num_graphs < 1 || b->num_graphs > INT_MAX || !jobs || !b->graph_off)
    return GC_ERR_INVALID_ARG;
  if (b->n < 0 || b->nnz < 0 || b->n > static_cast<int64_t>(INT_MAX) - 1) return GC_ERR_INVALID_ARG;
  if (b->n > 0 && (!b->row_ptr || !color_out)) return GC_ERR_INVALID_ARG;
  if (b->nnz > 0 && !b->col_idx) return GC_ERR_INVALID_ARG;
  for (int64_t g = 0; g < b->num_graphs; ++g) GC_TRY(check_eps(jobs[g].eps_p, jobs[g].eps_q));
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return GC_ERR_CUDA;
  CallScope scope(ctx);
  return gc::batch_color(ctx, b, jobs, color_out, batch_out, num_colors_out, num_rounds_out,
                         reinterpret_cast<cudaStream_t>(stream));
}

gc_status gc_color_batch_list(gc_context* ctx, int64_t num_graphs, const gc_csr* graphs, const gc_job* jobs,
                              int32_t* const* color_out, gc_stream stream) {
  if (!ctx || num_graphs < 1 || num_graphs > INT_MAX || !graphs || !jobs || !color_out)
    return GC_ERR_INVALID_ARG;
  for (int64_t g = 0; g < num_graphs; ++g) {
    GC_TRY(check_graph_args(&graphs[g]));
    GC_TRY(check_eps(jobs[g].eps_p, jobs[g].eps_q));
    if (graphs[g].n > 0 && !color_out[g]) return GC_ERR_INVALID_ARG;
  }
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return GC_ERR_CUDA;
  CallScope scope(ctx);
  return gc::batch_color_list(ctx, num_graphs, graphs, jobs, color_out, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
