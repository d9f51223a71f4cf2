// Internal declarations of the GB300 colouring library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

#include "gcolor.h"

namespace gc {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Edges per task of the edge sweeps (ADG's UPDATE, JP's core extraction): a
// vertex of degree d becomes ceil(d / kChunk) tasks, so one hub cannot hold a
// warp for long and hub-heavy rounds still spread over every warp.
constexpr int kChunk = 256;
// Independent edges each lane keeps in flight in the edge sweeps.
constexpr int kSweepUnroll = 8;
// Vertices of degree <= kSmallDeg are coloured one per lane, larger ones one
// per warp (at most kSmallDeg predecessors -> the colour fits a 64-bit mask).
constexpr int kSmallDeg = 32;
// Colour window of the warp path: a 1024-bit shared-memory bitmap per warp.
constexpr int kColorWin = 1024;
// Pending (still uncoloured) predecessors a lane of the warp path remembers.
constexpr int kPendCap = 16;

// Device-side error codes (written to a control block, mapped to gc_status).
enum DevErr : int { kDevOk = 0, kDevTimeout = 1, kDevOverflow = 2 };

// How long any device-side wait may spin before it gives up (nanoseconds of
// %globaltimer).
constexpr unsigned long long kWaitLimitNs = 4000000000ull;

// Control block of one ADG run (device memory, in the context's scratch).
struct AdgCtl {
  unsigned long long sigma;      // sum of D over U in the current round
  unsigned long long sum_R;      // this round: sum of D over R
  unsigned long long cut;        // this round: decrements (edges R -> U\R)
  unsigned long long ntasks;     // this round: UPDATE tasks appended
  unsigned long long total_U;    // sum over rounds of |U|
  unsigned long long total_dec;  // sum over rounds of the cut
  unsigned long long rows_U;     // sum of the row lengths (CSR entries) over U
  unsigned long long rows_R;     // this round: sum of the row lengths over R
  unsigned long long pull_sigma; // pull round: sum of the recounted D over U'
  unsigned long long ntasks_pull;// pull round: tasks over U' appended
  int size_U;                    // |U| of the current round
  int size_Unext;                // this round: survivors appended
  int T;                         // threshold of the current round (clamped)
  int round;                     // l (1-based) of the current round
  unsigned p, q;                 // eps = p / q
  int mode;                      // GC_UPDATE_AUTO / _PUSH / _PULL
  int pull_percent;              // AUTO: pull when rows(U') <= pull_percent % of rows(R)
  int pull_rounds;               // rounds that pulled
  int max_removal_degree;        // largest D at removal so far: every colour of
                                 // JP-ADG is at most this + 1 (a vertex's
                                 // predecessors are among the neighbours D counts)
  int hub_min_degree;            // UPDATE merges decrements aimed at vertices of at
                                 // least this degree (INT_MAX: none)
  int hub_cap;                   // hubs the rank table holds
  int n_hubs;                    // hubs ranked by round 1's partition
  int graph_err;                 // graph-launched rounds: a round removed no vertex
};

static_assert(sizeof(AdgCtl) <= 256, "AdgCtl must fit the pinned read-back buffer");

// Direction of this round's UPDATE, decided on the device after the
// partition from the entries each direction must sweep: push sweeps the rows
// of R, pull the rows of U'.  Every kernel of the round evaluates it on the
// same control block, so they agree without a host round trip.
#ifdef __CUDACC__
__device__ __forceinline__ bool adg_pulls(const AdgCtl& c) {
  if (c.size_Unext == 0 || c.mode == GC_UPDATE_PUSH) return false;
  if (c.mode == GC_UPDATE_PULL) return true;
  const unsigned long long rows_up = c.rows_U - c.rows_R;
  return static_cast<unsigned __int128>(rows_up) * 100u <=
         static_cast<unsigned __int128>(c.rows_R) * static_cast<unsigned>(c.pull_percent);
}
#endif

// Control block of one JP run (must fit the context's 256-byte pinned buffer).
struct JpCtl {
  unsigned long long big_cursor;
  unsigned long long small_cursor;
  unsigned long long key_or;     // OR over the sort keys (constant digits)
  unsigned long long key_and;    // AND over the sort keys
  unsigned long long spins;      // polls that found an uncoloured predecessor
  unsigned long long nbig;       // vertices in the warp-path list
  unsigned long long nsmall;     // vertices in the lane-path list
  unsigned long long ncore;      // vertices coloured by the core cluster
  unsigned long long base0;      // warp-path offset of the first bulk bucket
  unsigned long long base1;      // lane-path offset of the first bulk bucket
  long long bstar;               // last core bucket (-1: no core)
  long long core_preds;          // predecessor entries of the core
  unsigned long long core_deg;   // degree sum of the core vertices
  unsigned long long wait_ns;    // bound of every wait on a colour (ns)
  int max_color;
  int err;
  int stall;                     // injected fault: this vertex never publishes its colour (-1: none)
};
static_assert(sizeof(JpCtl) <= 256, "JpCtl must fit the pinned read-back buffer");

// Largest core coloured by the shared-memory cluster (16-bit ids and colours;
// each CTA keeps 2 bytes per core vertex next to 144 KB of bitmaps and
// deferred predecessors, within the 227 KB a block may use) and its default
// target size.
constexpr long long kCoreMax = 32768;
constexpr long long kCoreDefault = 16384;

// Bump allocator over the context's scratch arena (256-byte aligned slices).
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Device-wide exclusive scan helpers (gc_scan.cu).  `temp` needs
// scan_temp_elems(count) elements.
size_t scan_temp_elems(long long count);
cudaError_t exclusive_scan_i64(const long long* in, long long* out, long long count,
                               long long* temp, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs, ascending by key (gc_sort.cu).
// Only the 8-bit digits set in `digit_mask` are sorted (bit i = digit i).
// Returns the buffer index (0 or 1) that holds the result.
struct SortBufs {
  unsigned long long* keys[2];
  int* vals[2];
  long long* hist;   // 256 * ntiles
  long long* temp;   // scan temp
};
size_t sort_hist_elems(long long n);
int radix_sort_pairs(SortBufs& b, long long n, unsigned digit_mask, cudaStream_t s,
                     cudaError_t* err);

// ADG rounds on the device (gc_adg.cu).  Scratch sized by adg_scratch_bytes.
size_t adg_scratch_bytes(long long n, long long nnz);
// The column indices of vertex ranges [lo[c], lo[c+1]) arriving on another
// stream, range c complete when ready[c] fires: round 1's UPDATE sweeps each
// range once its event has fired (round 1's partition needs row offsets only),
// so the copy of col_idx overlaps ADG's first round.
constexpr int kUploadChunks = 8;
// A context's round-loop graph (gc_graph.cu).
struct LoopGraph {
  std::vector<unsigned char> key;   // of the graph built
  std::vector<unsigned char> seen;  // of the previous call
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
struct ColChunks {
  int k = 0;
  long long lo[kUploadChunks + 1] = {};
  cudaEvent_t ready[kUploadChunks] = {};
};
// D (n ints) receives each vertex's degree at removal.
gc_status adg_run(gc_context* ctx, Arena a, const gc_csr* g, unsigned p, unsigned q, int* batch,
                  int* D, int* rounds_out, cudaStream_t s, const ColChunks* chunks = nullptr);

// ADG-M rounds (gc_adg.cu): median degree, R = the ceil(|U|/2) smallest
// (D, id) of U.  D receives each vertex's degree at removal.
size_t adg_m_scratch_bytes(long long n, long long nnz);
gc_status adg_m_run(gc_context* ctx, Arena a, const gc_csr* g, int* batch, int* D, int* rounds_out,
                    cudaStream_t s);

// JP colouring by predecessor polling (gc_jp.cu).
size_t jp_scratch_bytes(long long n, long long nnz);
size_t jpadg_scratch_bytes(long long n, long long nnz, int rounds);
// batch: ADG batches; D: degree at removal (from adg_run); rounds: ADG rounds.
gc_status jp_run_fused(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D,
                       int rounds, unsigned long long seed, int* color, int* num_colors_out,
                       cudaStream_t s);
gc_status jp_run_given(gc_context* ctx, Arena a, const gc_csr* g, const unsigned long long* prio,
                       int* color, int* num_colors_out, cudaStream_t s);
// JP-ADG-O: JP in the exact order (batch, D, id) descending, D = degree at
// removal from adg_run.  Scratch: jp_scratch_bytes(n, nnz) + 8n.
gc_status jp_run_ordered(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D, int rounds,
                         int* color, int* num_colors_out, cudaStream_t s);
// ADG-O (gc_adg_o.cu): rho (and, if rank is not null, the count of
// higher-rho neighbours) from ADG's batches and degrees at removal; and
// JP-ADG-O's key batch * 2^32 + D.
size_t adg_o_scratch_bytes(long long n);
gc_status adg_o_order(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* D, int* rho,
                      int* rank, cudaStream_t s);
cudaError_t adg_o_priority(const int* batch, const int* D, long long n, unsigned long long* key, int num_sms,
                           cudaStream_t s);

// DEC-ADG-ITR colouring of the partitions batch[] = 1..rounds (gc_dec.cu).
// iters_out: SIM-COL iterations summed over the partitions.
size_t dec_scratch_bytes(long long n, long long nnz, int rounds);
// Also sets stats.dec_internal_edges.
gc_status dec_itr_run(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, int rounds,
                      unsigned long long seed, int* color, int* num_colors_out, long long* iters_out,
                      cudaStream_t s);
// gc_color_batch body (gc_batch.cu).
size_t batch_adg_scratch_bytes(long long n, long long nnz, long long G);
gc_status batch_color(gc_context* ctx, const gc_batch_csr* b, const gc_job* jobs, int32_t* color_out,
                      int32_t* batch_out, int32_t* num_colors_out, int32_t* num_rounds_out, cudaStream_t s);

gc_status batch_color_list(gc_context* ctx, long long G, const gc_csr* graphs, const gc_job* jobs,
                           int32_t* const* color_out, cudaStream_t s);
// The batch in one persistent launch, a block per graph (gc_batch_persist.cu):
// batch_order sorts the graph ids by decreasing size and returns the largest
// graph's vertices and CSR entries; djobs is a device copy of the jobs.
size_t batch_persistent_scratch_bytes(long long n, long long G);
gc_status batch_order(gc_context* ctx, Arena& a, const gc_batch_csr* b, int** order_out, long long* max_n,
                      long long* max_nnz, cudaStream_t s);
gc_status batch_color_persistent(gc_context* ctx, Arena a, const gc_batch_csr* b, const gc_job* djobs,
                                 const int* order, int32_t* color_out, int32_t* batch_out, int32_t* num_colors_out,
                                 int32_t* num_rounds_out, cudaStream_t s);

// A round loop as a CUDA graph (gc_graph.cu): capture(stream, handle) makes
// the launches of one body iteration on `stream`; its last kernel sets the
// handle's condition.  cudaSuccess with *exec, cudaErrorNotReady on the
// first call with a key (the caller then runs its host loop), or the error
// that stopped the build.
cudaError_t loop_graph(LoopGraph** slot, const void* key, size_t key_bytes,
                       const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& capture,
                       cudaGraphExec_t* exec);
void loop_graph_free(LoopGraph** slot);

// JP-ADG on the disjoint union of many graphs.  Vertex v of graph gid[v]
// (first vertex off[gid[v]]) has the tie-break rho_R of its own graph's seed,
// seed[gid[v]], and its id inside the graph; runs of more than 255 rounds
// need tiev[v], that tie-break precomputed (else tiev may be null).
gc_status jp_run_packed(gc_context* ctx, Arena a, const gc_csr* g, const int* batch, const int* gid,
                        const unsigned long long* seed, const long long* off, const unsigned* tiev, const int* D,
                        int rounds, int* color, int* num_colors_out, cudaStream_t s);
// Options (gc_tune.cu): apply range-checked options to a context; the
// autotuner times run() (one colouring into its argument, n ints) under
// candidate options and leaves the fastest applied.
void apply_options(gc_context* ctx, const gc_options& o);
gc_status autotune(gc_context* ctx, long long n, const std::function<gc_status(int*)>& run, bool batch, int reps,
                   float budget_ms, gc_options* best_out, float* best_ms_out, float* start_ms_out, int* trials_out,
                   cudaStream_t s);
cudaError_t make_priority(const int* batch, long long n, unsigned long long seed,
                          unsigned long long* key, int num_sms, cudaStream_t s);
// JP-SL keys (gc_sl.cu): the smallest-last removal index of every vertex.
size_t sl_scratch_bytes(long long n);
gc_status sl_priority(gc_context* ctx, Arena a, const gc_csr* g, unsigned long long* prio, cudaStream_t s);
// JP-R / FF / LF / LLF keys (gc_make_priority_kind); kind already checked.
cudaError_t make_priority_kind(const long long* row_ptr, long long n, int kind, unsigned long long seed,
                               unsigned long long* key, int num_sms, cudaStream_t s);

}  // namespace gc

// The opaque context.
constexpr long long kCoreDefault_ = gc::kCoreDefault;
struct gc_context {
  int device = 0;
  int num_sms = 0;
  int coop = 0;
  int timing = 0;
  gc_options opt{};                       // the options of gc_create, defaults filled in
  long long core_target = kCoreDefault_;  // JP-ADG core size (vertices)
  unsigned long long wait_ns = gc::kWaitLimitNs;  // bound of every device-side wait
  // Failure injection, for tests of the error paths (read from the
  // environment at gc_create): a vertex whose colour is never published (so
  // that its successors' waits run out), and allocation failure.
  int stall_vertex = -1;
  bool fail_alloc = false;
  int core_cluster = 0;                   // CTAs of the core cluster (0: not chosen yet)
  bool dec_tail = true;                   // DEC-ADG-ITR: finish small U in one cluster launch
  int tail_cluster = 0;                   // CTAs of that cluster (0: not chosen yet, -1: none fits)
  int core_warps = 0;                     // warps per core CTA
  int adg_max_removal_degree = -1;        // of the last ADG run (-1: unknown)
  // scratch arena (device)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // small page-locked host buffer for scalar read-back
  void* pinned = nullptr;
  // per-vertex state that outlives one phase (D, an internal batch array)
  void* vbuf = nullptr;
  size_t vbuf_bytes = 0;
  // predecessor lists of the JP core
  void* aux = nullptr;
  size_t aux_bytes = 0;
  // packed union of gc_color_batch_list
  void* pack = nullptr;
  size_t pack_bytes = 0;
  // buffers owned for gc_color_graph_host, and its copy stream and events
  void* h_graph = nullptr;
  size_t h_graph_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  // the round-loop graphs of ADG (gc_adg.cu) and of the segmented batch
  // path (gc_batch.cu)
  gc::LoopGraph* adg_graph = nullptr;
  gc::LoopGraph* batch_graph = nullptr;
  cudaEvent_t copy_ev[gc::kUploadChunks + 1] = {};  // per range, then "the device buffers are free"
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // kernel-group timers: event pairs recorded around launches when timing is
  // on, summed per group after the call's final synchronisation
  static constexpr int kTimerPairs = 128;
  cudaEvent_t tev[2 * kTimerPairs] = {};
  int tgroup[kTimerPairs] = {};
  int tused = 0;
  gc_stats stats{};

  enum TimerGroup { kTUpdate = 0, kTCoreSolve = 1, kTBulk = 2, kTCorePreds = 3, kTDecExtract = 4, kTDecIterate = 5 };
  void timer_begin(int group, cudaStream_t s) {
    if (!timing || tused >= kTimerPairs || !tev[2 * tused]) return;
    tgroup[tused] = group;
    cudaEventRecord(tev[2 * tused], s);
  }
  void timer_end(cudaStream_t s) {
    if (!timing || tused >= kTimerPairs || !tev[2 * tused]) return;
    cudaEventRecord(tev[2 * tused + 1], s);
    ++tused;
  }
  // after the stream is synchronised
  void timers_collect() {
    float sum[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < tused; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, tev[2 * i], tev[2 * i + 1]) == cudaSuccess) sum[tgroup[i]] += ms;
    }
    stats.ms_adg_update = sum[kTUpdate];
    stats.ms_core_solve = sum[kTCoreSolve];
    stats.ms_jp_color = sum[kTBulk];
    stats.ms_core_preds = sum[kTCorePreds];
    stats.ms_dec_extract = sum[kTDecExtract];
    stats.ms_dec_iterate = sum[kTDecIterate];
    tused = 0;
  }
  gc_status reserve(size_t bytes);      // scratch arena
  gc_status reserve_vert(size_t bytes); // vbuf
  gc_status reserve_aux(size_t bytes);  // aux
  gc_status reserve_pack(size_t bytes); // pack
  gc::Arena arena() const {
    gc::Arena a;
    a.base = static_cast<char*>(scratch);
    a.cap = scratch_bytes;
    return a;
  }
};

// int64_t is `long` on LP64 Linux while the kernels use `long long`.
inline const long long* row_ptr_of(const gc_csr* g) {
  return reinterpret_cast<const long long*>(g->row_ptr);
}

namespace gc {
// Kernels launched by the current entry-point call on this host thread.
extern thread_local int g_launches;
}  // namespace gc

// Map a CUDA error to a status (and leave no sticky state behind).
inline gc_status gc_cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GC_OK;
  if (e == cudaErrorMemoryAllocation) return GC_ERR_OOM;
  return GC_ERR_CUDA;
}

namespace gc {
// Where the last failing CUDA call of this host thread was made (gc_last_error).
void note_cuda_error(cudaError_t e, const char* file, int line);
}  // namespace gc

#define GC_TRY_CUDA(expr)                              \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) {                           \
      gc::note_cuda_error(e_, __FILE__, __LINE__);     \
      return gc_cuda_status(e_);                       \
    }                                                  \
  } while (0)

#define GC_TRY(expr)                 \
  do {                               \
    gc_status s_ = (expr);           \
    if (s_ != GC_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------------------
// Device helpers shared by the kernels of this library.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace gc {

// Blocks of `threads` threads of `kernel` that fit on the whole GPU at once:
// grid-stride kernels launched with this many blocks have no second wave.
template <class K>
int resident_grid(K kernel, int threads, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return num_sms * per_sm;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed(const unsigned short* p) {
  unsigned short v;
  asm volatile("ld.relaxed.gpu.global.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return static_cast<int>(v);
}

__device__ __forceinline__ void st_relaxed(unsigned short* p, int v) {
  asm volatile("st.relaxed.gpu.global.u16 [%0], %1;" ::"l"(p), "h"(static_cast<unsigned short>(v)) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(kFull, v, o);
    v = u > v ? u : v;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// One block step's appends to two global lists: warp w appends wa entries to
// the list whose length is *ca and wb to the one whose length is *cb.  The
// block adds its totals with one atomic each (instead of one per warp on the
// same address) and each warp gets the start of its own run, warps in order.
// Every thread of the block calls it (two barriers).  s_a and s_b are shared
// arrays of blockDim.x / 32 entries; callers alternate between two pairs on
// consecutive calls, which makes a third barrier before their reuse
// unnecessary.
struct BlockSlots {
  int a;
  unsigned long long b;
};

__device__ __forceinline__ BlockSlots block_reserve(int* ca, int wa, unsigned long long* cb, unsigned long long wb,
                                                    int* s_a, unsigned long long* s_b) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  if (lane == 0) {
    s_a[warp] = wa;
    s_b[warp] = wb;
  }
  __syncthreads();
  if (warp == 0) {
    const int va = lane < nw ? s_a[lane] : 0;
    const unsigned long long vb = lane < nw ? s_b[lane] : 0ull;
    const int ia = warp_inclusive_scan(va);
    const unsigned long long ib = warp_inclusive_scan(vb);
    int ba = 0;
    unsigned long long bb = 0;
    if (lane == 31) {
      if (ia) ba = atomicAdd(ca, ia);
      if (ib) bb = atomicAdd(cb, ib);
    }
    ba = __shfl_sync(kFull, ba, 31);
    bb = __shfl_sync(kFull, bb, 31);
    if (lane < nw) {
      s_a[lane] = ba + ia - va;
      s_b[lane] = bb + ib - vb;
    }
  }
  __syncthreads();
  return BlockSlots{s_a[warp], s_b[warp]};
}

// Edge sweep over 32 tasks held one per lane (task start `st`, length `len`,
// a caller value `tag`): the tasks' edges are numbered 0..total-1 in lane
// order and handed out 32 * kSweepUnroll at a time, each lane taking
// kSweepUnroll edges.  For each edge, with w = col_idx[k] and the tag of the
// task owning it, gather(w, tag) is evaluated first (a load of per-vertex
// state) and fn(w, tag, gathered) after it.  All kSweepUnroll col_idx loads
// of a lane are issued before any gather, and all gathers before any fn, so
// that a lane has kSweepUnroll loads in flight at each step even where fn
// writes memory (which could keep the compiler from moving the next edge's
// gather ahead of it).
template <int kU = kSweepUnroll, class Gather, class Fn>
__device__ __forceinline__ void sweep_tile(long long st, int len, int tag, const int* __restrict__ col,
                                           Gather gather, Fn fn) {
  constexpr int kSweepUnroll = kU;  // edges per lane and step
  const int lane = threadIdx.x & 31;
  const int incl = warp_inclusive_scan(len);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - len;
  using G = decltype(gather(0, 0));
  for (int b = 0; b < total; b += 32 * kSweepUnroll) {
    int w[kSweepUnroll], own[kSweepUnroll];
#pragma unroll
    for (int u = 0; u < kSweepUnroll; ++u) {
      const int e = b + u * 32 + lane;
      int j = 0;  // owner: the largest lane j with excl_j <= e
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int c = j + step;
        if (__shfl_sync(kFull, excl, c) <= e) j = c;
      }
      const long long k = __shfl_sync(kFull, st, j) + (e - __shfl_sync(kFull, excl, j));
      const int tg = __shfl_sync(kFull, tag, j);
      own[u] = e < total ? tg : -1;
      w[u] = e < total ? __ldg(col + k) : -1;
    }
    G gv[kSweepUnroll];
#pragma unroll
    for (int u = 0; u < kSweepUnroll; ++u) gv[u] = w[u] >= 0 ? gather(w[u], own[u]) : G{};
#pragma unroll
    for (int u = 0; u < kSweepUnroll; ++u)
      if (w[u] >= 0) fn(w[u], own[u], gv[u]);
  }
}

// Random tie-break rho_R of the JP-ADG priority (Section 4.1): the upper 32
// bits of the (v+1)-th output of SplitMix64 (Steele, Lea & Flood, OOPSLA
// 2014) started from state `seed`.  The state advances by the golden-ratio
// increment 0x9e3779b97f4a7c15 and each output is mixed by the finaliser
// z ^= z>>30; z *= 0xbf58476d1ce4e5b9; z ^= z>>27; z *= 0x94d049bb133111eb;
// z ^= z>>31.
__device__ __forceinline__ unsigned tie_hash(unsigned long long seed, unsigned v) {
  unsigned long long z = seed + (static_cast<unsigned long long>(v) + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return static_cast<unsigned>(z >> 32);
}

}  // namespace gc
#endif
