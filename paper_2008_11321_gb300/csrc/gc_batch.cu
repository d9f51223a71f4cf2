// gc_color_batch: JP-ADG on many graphs at once.
//
// The graphs arrive packed as one CSR, their disjoint union: graph g owns the
// vertices [graph_off[g], graph_off[g+1]) and its edges stay inside that
// range.  ADG (Algorithm 1, Section 3) keeps its state per graph -- degree
// sum, |U|, threshold, its own eps -- while one set of launches per round
// serves every graph still running: all graphs start in round 1 together, so a
// graph that is still running is always in the global round, and a graph
// whose U is empty drops out.  JP (Algorithm 3, Section 4.1) then runs once on
// the union with each vertex's tie-break computed from its own graph's seed
// and its id inside that graph; as no edge joins two graphs, each graph's
// colouring is exactly the one gc_color_graph gives it alone.
#include <climits>
#include <cstring>
#include <vector>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kBThreads = 256;

// Per-graph ADG state (device).
struct BGraph {
  unsigned long long sigma;  // sum of D over the graph's U
  unsigned long long sum_R;  // this round: sum of D over the graph's R
  unsigned long long cut;    // this round: decrements inside the graph
  int size_U;                // |U| of the graph (0: finished)
  int size_Unext;            // this round: survivors
  int T;                     // threshold of the current round
  int rounds;                // rounds the graph needed (set when U empties)
  unsigned p, q;             // the graph's eps = p / q
  unsigned long long seed;   // the graph's tie-break seed
};

struct BCtl {
  int round;        // global round (the round of every graph still running)
  int size_Unext;   // survivors over all graphs
  int size_U;       // |U| over all graphs in the current round (from round 2 on)
  int err;          // a round that removed no vertex (cannot happen)
  unsigned long long ntasks;
  unsigned long long total_U;    // sum over graphs and rounds of |U|
  unsigned long long total_dec;  // sum over graphs and rounds of the cut
};

__device__ __forceinline__ int threshold_of(unsigned long long sigma, int size_u, unsigned p, unsigned q) {
  if (size_u <= 0) return 0;
  unsigned __int128 num = static_cast<unsigned __int128>(static_cast<unsigned long long>(q) + p) * sigma;
  unsigned __int128 den = static_cast<unsigned __int128>(q) * static_cast<unsigned>(size_u);
  unsigned __int128 t = num / den;
  return t > static_cast<unsigned __int128>(INT_MAX) ? INT_MAX : static_cast<int>(t);
}

__global__ void batch_init_kernel(BGraph* __restrict__ gs, const gc_job* __restrict__ jobs, int G,
                                  const long long* __restrict__ off, const long long* __restrict__ row_ptr,
                                  BCtl* ctl, unsigned long long* __restrict__ seeds, long long n_total) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    seeds[g] = jobs[g].seed;
    BGraph b{};
    const long long n = off[g + 1] - off[g];
    b.sigma = static_cast<unsigned long long>(row_ptr[off[g + 1]] - row_ptr[off[g]]);
    b.size_U = static_cast<int>(n);
    b.p = jobs[g].eps_p;
    b.q = jobs[g].eps_q;
    b.seed = jobs[g].seed;
    b.T = threshold_of(b.sigma, b.size_U, b.p, b.q);
    b.rounds = 0;
    gs[g] = b;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    BCtl c{};
    c.round = 1;
    c.size_U = static_cast<int>(n_total);
    *ctl = c;
  }
}

// Graph id of every vertex (one block per graph writes its range), so that
// the kernels below read a vertex's graph instead of searching graph_off.
__global__ void batch_gid_kernel(const long long* __restrict__ off, int G, int* __restrict__ gid) {
  for (int g = blockIdx.x; g < G; g += gridDim.x)
    for (long long v = off[g] + threadIdx.x; v < off[g + 1]; v += blockDim.x) gid[v] = g;
}

// Sum of `x` over the lanes of `group` (a __match_any_sync class), 64-bit.
__device__ __forceinline__ unsigned long long group_sum(unsigned group, unsigned long long x) {
  const unsigned lo = __reduce_add_sync(group, static_cast<unsigned>(x & 0xffffu));
  const unsigned mid = __reduce_add_sync(group, static_cast<unsigned>((x >> 16) & 0xffffu));
  const unsigned hi = __reduce_add_sync(group, static_cast<unsigned>(x >> 32));
  return static_cast<unsigned long long>(lo) + (static_cast<unsigned long long>(mid) << 16) +
         (static_cast<unsigned long long>(hi) << 32);
}

// One block step of the batched partition, K vertices per thread (vertex
// i = base + j * blockDim.x + threadIdx.x for j < K): all K vertices' loads
// first, then the survivors and UPDATE tasks of the whole block appended with
// one atomic per list (block_reserve); the per-graph counts stay per warp and
// graph (__match_any_sync groups).
template <int K>
__device__ __forceinline__ void batch_partition_steps(
    BCtl* __restrict__ ctl, BGraph* __restrict__ gs, const int* __restrict__ gid,
    const long long* __restrict__ row_ptr, int* __restrict__ D, int* __restrict__ batch,
    const int* __restrict__ u_in, int* __restrict__ u_out, long long* __restrict__ task_start,
    int* __restrict__ task_len, int* __restrict__ task_g, long long size_u, unsigned* __restrict__ live, int round,
    bool first) {
  __shared__ int s_keep[2][kBThreads / 32];
  __shared__ unsigned long long s_task[2][kBThreads / 32];
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const long long span = static_cast<long long>(blockDim.x) * K;
  const long long stride = static_cast<long long>(gridDim.x) * span;
  int par = 0;
  // base is the same for every thread of the block: the barriers inside
  // block_reserve are reached by all of them on every step
  for (long long base = static_cast<long long>(blockIdx.x) * span; base < size_u; base += stride, par ^= 1) {
    int u[K], d[K], g[K], nt[K], incl[K];
    long long rs[K], re[K];
    bool in_r[K], keep[K];
    unsigned km[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long i = base + static_cast<long long>(j) * blockDim.x + threadIdx.x;
      const bool active = i < size_u;
      u[j] = 0;
      d[j] = 0;
      g[j] = -1;
      rs[j] = 0;
      re[j] = 0;
      if (active) {
        u[j] = first ? static_cast<int>(i) : u_in[i];
        g[j] = gid[u[j]];
        if (first) {
          rs[j] = row_ptr[u[j]];
          re[j] = row_ptr[u[j] + 1];
          d[j] = static_cast<int>(re[j] - rs[j]);
        } else {
          d[j] = D[u[j]];
        }
      }
      const int T = active ? gs[g[j]].T : 0;
      in_r[j] = active && d[j] <= T;
      keep[j] = active && !in_r[j];
    }
    if (!first) {  // removed vertices' rows -> UPDATE tasks of at most kChunk edges
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (in_r[j]) {
          rs[j] = row_ptr[u[j]];
          re[j] = row_ptr[u[j] + 1];
        }
    }
    int wkeep = 0;
    unsigned long long wtask = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      km[j] = __ballot_sync(kFull, keep[j]);
      wkeep += __popc(km[j]);
      nt[j] = (!first && in_r[j]) ? static_cast<int>((re[j] - rs[j] + kChunk - 1) / kChunk) : 0;
      incl[j] = warp_inclusive_scan(nt[j]);
      wtask += static_cast<unsigned>(__shfl_sync(kFull, incl[j], 31));
    }
    const BlockSlots slot = block_reserve(&ctl->size_Unext, wkeep, &ctl->ntasks, wtask, s_keep[par], s_task[par]);
    int kb = slot.a;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long i = base + static_cast<long long>(j) * blockDim.x + threadIdx.x;
      const bool active = i < size_u;
      // survivors -> U', counted per graph
      if (keep[j]) u_out[kb + __popc(km[j] & lt)] = u[j];
      kb += __popc(km[j]);
      const unsigned grp = __match_any_sync(kFull, g[j]);
      const unsigned kgrp = grp & km[j];
      if (keep[j] && (kgrp & lt) == 0) atomicAdd(&gs[g[j]].size_Unext, __popc(kgrp));
      // removed -> batch id, per-graph sum of D
      const unsigned rm = __ballot_sync(kFull, in_r[j]);
      const unsigned rgrp = grp & rm;
      // liveness bitmap: round 1 writes the warp's word (vertices 32 w ..
      // 32 w + 31: every run starts at a multiple of 32), later rounds clear
      // bits
      if (first) {
        if (lane == 0 && active) live[i >> 5] = km[j];
        if (active) D[u[j]] = d[j];
      } else if (in_r[j]) {
        atomicAnd(&live[u[j] >> 5], ~(1u << (u[j] & 31)));
      }
      const unsigned long long dsum = group_sum(grp, in_r[j] ? static_cast<unsigned long long>(d[j]) : 0ull);
      if (in_r[j]) {
        batch[u[j]] = round;
        if ((rgrp & lt) == 0) atomicAdd(&gs[g[j]].sum_R, dsum);
      }
    }
    if (first) continue;  // round 1 sweeps vertex tiles
    unsigned long long tb = slot.b;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int tot = __shfl_sync(kFull, incl[j], 31);
      const int excl = incl[j] - nt[j];
      for (int b = 0; b < tot; b += 32) {
        const int x = b + lane;
        int o = 0;  // owner: the largest lane o with excl_o <= x
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int c = o + step;
          if (__shfl_sync(kFull, excl, c) <= x) o = c;
        }
        const long long st = __shfl_sync(kFull, rs[j], o) +
                             static_cast<long long>(x - __shfl_sync(kFull, excl, o)) * kChunk;
        const long long rej = __shfl_sync(kFull, re[j], o);
        const int gj = __shfl_sync(kFull, g[j], o);
        if (x < tot) {
          task_start[tb + x] = st;
          task_len[tb + x] = static_cast<int>(rej - st < kChunk ? rej - st : kChunk);
          task_g[tb + x] = gj;
        }
      }
      tb += static_cast<unsigned long long>(tot);
    }
  }
}

// Vertices per thread and block step on rounds large enough to give every
// thread of the grid that many.
constexpr int kBPartItems = 4;

__global__ void __launch_bounds__(kBThreads, 4)  // 64 registers: 4 blocks per SM
batch_partition_kernel(BCtl* __restrict__ ctl, BGraph* __restrict__ gs, const int* __restrict__ gid,
                       const long long* __restrict__ row_ptr, int* __restrict__ D,
                       int* __restrict__ batch, const int* __restrict__ u_in, int* __restrict__ u_out,
                       long long* __restrict__ task_start, int* __restrict__ task_len,
                       int* __restrict__ task_g, long long size_u, unsigned* __restrict__ live) {
  const int round = ctl->round;
  if (size_u < 0) size_u = ctl->size_U;  // the graph-launched rounds
  const bool first = round == 1;
  // the same choice in every block: size_u and the grid are the kernel's
  if (size_u >= static_cast<long long>(gridDim.x) * blockDim.x * kBPartItems)
    batch_partition_steps<kBPartItems>(ctl, gs, gid, row_ptr, D, batch, u_in, u_out, task_start, task_len, task_g,
                                       size_u, live, round, first);
  else
    batch_partition_steps<1>(ctl, gs, gid, row_ptr, D, batch, u_in, u_out, task_start, task_len, task_g, size_u,
                             live, round, first);
}

__global__ void __launch_bounds__(kBThreads)
batch_update_kernel(BCtl* __restrict__ ctl, BGraph* __restrict__ gs, const int* __restrict__ gid,
                    const long long* __restrict__ row_ptr, const int* __restrict__ col,
                    int* __restrict__ D, const int* __restrict__ batch,
                    const long long* __restrict__ task_start, const int* __restrict__ task_len,
                    const int* __restrict__ task_g, long long vertex_tiles_n, const unsigned* __restrict__ live) {
  const int round = ctl->round;
  const unsigned long long ntasks =
      vertex_tiles_n > 0 ? static_cast<unsigned long long>(vertex_tiles_n) : ctl->ntasks;
  const int lane = threadIdx.x & 31;
  const unsigned long long gwarp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = (static_cast<unsigned long long>(gridDim.x) * blockDim.x) >> 5;
  // decrements counted per graph; a lane flushes its count when the graph of
  // its edges changes (edges of one graph come in long runs)
  int cur_g = -1;
  unsigned long long cnt = 0;
  for (unsigned long long tile = gwarp; tile * 32 < ntasks; tile += nwarps) {
    const unsigned long long t = tile * 32 + lane;
    long long st = 0;
    int len = 0, tg = 0;
    if (t < ntasks) {
      if (vertex_tiles_n > 0) {
        if (batch[t] == round) {
          st = row_ptr[t];
          len = static_cast<int>(row_ptr[t + 1] - st);
          tg = gid[t];
        }
      } else {
        st = task_start[t];
        len = task_len[t];
        tg = task_g[t];
      }
    }
    sweep_tile<4>(
        st, len, tg, col, [&](int w, int) { return (__ldg(live + (w >> 5)) >> (w & 31)) & 1u; },
        [&](int w, int g, unsigned lw) {
      if (lw) {  // w is still in U
        atomicSub(&D[w], 1);
        if (g != cur_g) {
          if (cnt) atomicAdd(&gs[cur_g].cut, cnt);
          cur_g = g;
          cnt = 0;
        }
        ++cnt;
      }
    });
  }
  if (cnt) atomicAdd(&gs[cur_g].cut, cnt);
}

__global__ void batch_finalize_kernel(BCtl* ctl, BGraph* __restrict__ gs, int G) {
  const int round = ctl->round;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    BGraph c = gs[g];
    if (c.size_U == 0) continue;
    atomicAdd(&ctl->total_U, static_cast<unsigned long long>(c.size_U));
    if (c.cut) atomicAdd(&ctl->total_dec, c.cut);
    c.sigma = c.sigma - c.sum_R - c.cut;
    c.size_U = c.size_Unext;
    if (c.size_U == 0)
      c.rounds = round;
    else
      c.T = threshold_of(c.sigma, c.size_U, c.p, c.q);
    c.sum_R = 0;
    c.cut = 0;
    c.size_Unext = 0;
    gs[g] = c;
  }
}

// After a round: the survivors become U.  In the graph-launched loop the
// kernel also decides whether the loop goes on (a round whose U was already
// empty changed nothing and ends it; so does a round that removed no vertex,
// which cannot happen and is reported).
__device__ __forceinline__ bool next_round(BCtl* ctl) {
  const int prev = ctl->size_U, next = ctl->size_Unext;
  if (prev == 0) return false;
  if (next >= prev) {
    ctl->err = 1;
    ctl->size_U = 0;
    return false;
  }
  ctl->round += 1;
  ctl->size_U = next;
  ctl->size_Unext = 0;
  ctl->ntasks = 0;
  return next > 0;
}

__global__ void batch_next_round_kernel(BCtl* ctl) { next_round(ctl); }

__global__ void batch_next_round_graph_kernel(BCtl* ctl, cudaGraphConditionalHandle loop) {
  cudaGraphSetConditional(loop, next_round(ctl) ? 1u : 0u);
}

// rho_R of every vertex from its graph's seed and its id inside the graph.
__global__ void batch_tie_kernel(const BGraph* __restrict__ gs, const long long* __restrict__ off,
                                 const int* __restrict__ gid, long long n, unsigned* __restrict__ tiev) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int g = gid[v];
    tiev[v] = tie_hash(gs[g].seed, static_cast<unsigned>(v - off[g]));
  }
}

// Largest colour and round count per graph.
__global__ void batch_results_kernel(const BGraph* __restrict__ gs, const int* __restrict__ gid, int G,
                                     long long n, const int* __restrict__ color, int* __restrict__ ncol,
                                     int* __restrict__ nrounds) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < n;
       base += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long v = base + threadIdx.x;
    const bool active = v < n;
    const int g = active ? gid[v] : -1;
    const int c = active ? color[v] : 0;
    const unsigned grp = __match_any_sync(kFull, g);
    const int m = static_cast<int>(__reduce_max_sync(grp, static_cast<unsigned>(c)));
    if (active && (grp & lt) == 0 && ncol) atomicMax(&ncol[g], m);
    (void)lane;
  }
  if (nrounds)
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
      nrounds[g] = gs[g].rounds;
}

// The ADG rounds from round 2 on as one CUDA graph loop (gc_graph.cu): the
// body holds two rounds (partition, UPDATE, finalize, next round), the first
// reading U from ubuf[0] and writing U' to ubuf[1], the second the other way
// round, so every kernel argument is fixed; the partition reads |U| from the
// control block, and each round's last kernel sets the loop condition.  A
// round whose U is already empty is a no-op.
struct RoundArgs {
  BCtl* ctl;
  BGraph* gs;
  const int* gid;
  const long long* rp;
  const int* col;
  int* D;
  int* bat;
  int* ubuf[2];
  long long* task_start;
  int* task_len;
  int* task_g;
  unsigned* live;
  long long G, pblocks, upd_blocks;  // the key: all of the above
};

cudaError_t batch_round_graph(gc_context* ctx, const RoundArgs& r, cudaGraphExec_t* exec) {
  return loop_graph(&ctx->batch_graph, &r, sizeof(r), [&](cudaStream_t cs, cudaGraphConditionalHandle loop) {
    const int G = static_cast<int>(r.G);
    for (int half = 0; half < 2; ++half) {
      batch_partition_kernel<<<static_cast<int>(r.pblocks), kBThreads, 0, cs>>>(
          r.ctl, r.gs, r.gid, r.rp, r.D, r.bat, r.ubuf[half], r.ubuf[half ^ 1], r.task_start, r.task_len, r.task_g,
          -1, r.live);
      batch_update_kernel<<<static_cast<int>(r.upd_blocks), kBThreads, 0, cs>>>(
          r.ctl, r.gs, r.gid, r.rp, r.col, r.D, r.bat, r.task_start, r.task_len, r.task_g, 0, r.live);
      batch_finalize_kernel<<<(G + 255) / 256, 256, 0, cs>>>(r.ctl, r.gs, G);
      batch_next_round_graph_kernel<<<1, 1, 0, cs>>>(r.ctl, loop);
    }
  }, exec);
}

}  // namespace

size_t batch_adg_scratch_bytes(long long n, long long nnz, long long G) {
  const long long ntask = n + nnz / kChunk + 1;
  return 2 * (static_cast<size_t>(n) * 4 + 256) + static_cast<size_t>(ntask) * 16 + 1024 +
         static_cast<size_t>(G) * (sizeof(BGraph) + sizeof(gc_job)) + static_cast<size_t>((n + 31) / 32) * 4 + 256 +
         2048;
}

}  // namespace gc

namespace gc {

gc_status batch_color(gc_context* ctx, const gc_batch_csr* b, const gc_job* jobs, int32_t* color_out,
                      int32_t* batch_out, int32_t* num_colors_out, int32_t* num_rounds_out, cudaStream_t s) {
  const long long n = b->n, nnz = b->nnz;
  const int G = static_cast<int>(b->num_graphs);
  const long long* rp = reinterpret_cast<const long long*>(b->row_ptr);
  const long long* off = reinterpret_cast<const long long*>(b->graph_off);
  // state that lives through both phases: D, batch (if internal), rho_R per
  // vertex, and the per-graph ADG state and jobs
  const size_t vb = (static_cast<size_t>(n > 0 ? n : 1) * 4 + 255) & ~size_t(255);
  const size_t gb = (static_cast<size_t>(G) * sizeof(BGraph) + 255) & ~size_t(255);
  const size_t jb = (static_cast<size_t>(G) * sizeof(gc_job) + 255) & ~size_t(255);
  const size_t sb = (static_cast<size_t>(G) * sizeof(unsigned long long) + 255) & ~size_t(255);
  GC_TRY(ctx->reserve_vert(4 * vb + gb + jb + sb));
  char* vbase = static_cast<char*>(ctx->vbuf);
  int* D = reinterpret_cast<int*>(vbase);
  int* bat = batch_out ? batch_out : reinterpret_cast<int*>(vbase + vb);
  unsigned* tiev = reinterpret_cast<unsigned*>(vbase + 2 * vb);
  BGraph* gs = reinterpret_cast<BGraph*>(vbase + 3 * vb);
  gc_job* djobs = reinterpret_cast<gc_job*>(vbase + 3 * vb + gb);
  int* gid = reinterpret_cast<int*>(vbase + 3 * vb + gb + jb);
  unsigned long long* seeds = reinterpret_cast<unsigned long long*>(vbase + 4 * vb + gb + jb);
  GC_TRY_CUDA(cudaMemcpyAsync(djobs, jobs, sizeof(gc_job) * G, cudaMemcpyHostToDevice, s));
  // One persistent launch (a block per graph, gc_batch_persist.cu) when no
  // graph is too large for one block: at most 4 times an SM's share of the
  // batch's CSR entries, and at most 2^24 entries.
  if (ctx->opt.batch_mode != GC_BATCH_SEGMENTED && n > 0) {
    GC_TRY(ctx->reserve(batch_persistent_scratch_bytes(n, G)));
    Arena pa = ctx->arena();
    int* order = nullptr;
    long long max_n = 0, max_nnz = 0;
    GC_TRY(batch_order(ctx, pa, b, &order, &max_n, &max_nnz, s));
    // The persistent path's time is the largest graph's on one block (about
    // 18 M CSR entries/s: 90 ms for 4,096 graphs up to 200k vertices), the
    // segmented path's the whole batch at GPU rate (about 14 G entries/s:
    // 50 ms for the same batch): AUTO takes the persistent path while the
    // largest graph holds at most 1/1024 of the batch's entries.
    const bool fits = max_nnz <= (1ll << 24) && max_nnz * 1024 <= (nnz > 0 ? nnz : 1);
    if (ctx->opt.batch_mode == GC_BATCH_PERSISTENT || fits) {
      ctx->stats.batch_path = GC_BATCH_PERSISTENT;
      ctx->stats.adg_rounds = 0;
      return batch_color_persistent(ctx, pa, b, djobs, order, color_out, batch_out, num_colors_out, num_rounds_out,
                                    s);
    }
  }
  ctx->stats.batch_path = GC_BATCH_SEGMENTED;
  // the segmented path's scratch is taken only now: the check above may have
  // grown (reallocated) the scratch arena
  GC_TRY(ctx->reserve(batch_adg_scratch_bytes(n, nnz, G)));
  Arena a = ctx->arena();
  BCtl* ctl = a.take<BCtl>(1);
  int* ubuf[2] = {a.take<int>(n > 0 ? n : 1), a.take<int>(n > 0 ? n : 1)};
  const long long ntask = n + nnz / kChunk + 1;
  long long* task_start = a.take<long long>(ntask);
  int* task_len = a.take<int>(ntask);
  int* task_g = a.take<int>(ntask);
  unsigned* live = a.take<unsigned>((n + 31) / 32 + 1);
  if (!ctl || !ubuf[0] || !ubuf[1] || !task_start || !task_len || !task_g || !live) return GC_ERR_OOM;
  if (n > 0) GC_TRY_CUDA(cudaMemsetAsync(bat, 0, sizeof(int) * n, s));  // 0 = still in U
  const int blocks = ctx->num_sms * 8;
  const int upd_blocks = resident_grid(batch_update_kernel, kBThreads, ctx->num_sms);
  batch_init_kernel<<<(G + 255) / 256, 256, 0, s>>>(gs, djobs, G, off, rp, ctl, seeds, n);
  ++g_launches;
  batch_gid_kernel<<<G < 65535 ? G : 65535, 256, 0, s>>>(off, G, gid);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());

  // ADG: one set of launches per round for every graph still running
  ctx->timer_begin(gc_context::kTUpdate, s);
  long long size_u = n;
  int round = 0, cur = 0;
  int* pin = static_cast<int*>(ctx->pinned);
  while (size_u > 0) {
    ++round;
    if (round == 2 && ctx->opt.round_graph) {
      // rounds 2.. as one graph launch (no host round trip per round)
      RoundArgs ra{ctl,  gs,     gid,  rp,   b->col_idx, D,      bat, {ubuf[0], ubuf[1]}, task_start, task_len,
                   task_g, live, G, blocks, upd_blocks};
      cudaGraphExec_t ex = nullptr;
      if (cur == 1 && batch_round_graph(ctx, ra, &ex) == cudaSuccess) {
        GC_TRY_CUDA(cudaGraphLaunch(ex, s));
        GC_TRY_CUDA(cudaMemcpyAsync(pin, &ctl->round, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        GC_TRY_CUDA(cudaStreamSynchronize(s));
        if (pin[3]) return GC_ERR_CUDA;  // a round removed no vertex: cannot happen
        const int last = pin[0] - 1;     // each round that ran advanced the round number
        g_launches += 8ull * static_cast<unsigned long long>((last - 1 + 1) / 2);
        round = last;
        break;
      }
    }
    const long long want = (size_u + kBThreads - 1) / kBThreads;
    const int pblocks = static_cast<int>(want < blocks ? want : blocks);
    batch_partition_kernel<<<pblocks, kBThreads, 0, s>>>(ctl, gs, gid, rp, D, bat,
                                                         round == 1 ? nullptr : ubuf[cur ^ 1], ubuf[cur],
                                                         task_start, task_len, task_g, size_u, live);
    ++g_launches;
    batch_update_kernel<<<upd_blocks, kBThreads, 0, s>>>(ctl, gs, gid, rp, b->col_idx, D, bat, task_start,
                                                     task_len, task_g, round == 1 ? n : 0, live);
    ++g_launches;
    batch_finalize_kernel<<<(G + 255) / 256, 256, 0, s>>>(ctl, gs, G);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(cudaMemcpyAsync(pin, &ctl->size_Unext, sizeof(int), cudaMemcpyDeviceToHost, s));
    batch_next_round_kernel<<<1, 1, 0, s>>>(ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    const long long next = *pin;
    if (next >= size_u) return GC_ERR_CUDA;  // cannot happen: every running graph removes a vertex
    size_u = next;
    cur ^= 1;
  }
  ctx->timer_end(s);
  ctx->stats.adg_rounds = round;
  {
    unsigned long long* pl = static_cast<unsigned long long*>(ctx->pinned);
    GC_TRY_CUDA(cudaMemcpyAsync(pl, &ctl->total_U, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    ctx->stats.sum_U = static_cast<int64_t>(pl[0]);
    ctx->stats.sum_decrements = static_cast<int64_t>(pl[1]);
  }
  if (n == 0) return GC_OK;
  if (round > 255) {  // the fallback key reads rho_R per vertex
    batch_tie_kernel<<<blocks, 256, 0, s>>>(gs, off, gid, n, tiev);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }

  // JP on the union
  gc_csr u;
  u.n = n;
  u.nnz = nnz;
  u.row_ptr = b->row_ptr;
  u.col_idx = b->col_idx;
  GC_TRY(ctx->reserve(jpadg_scratch_bytes(n, nnz, round)));
  int colors = 0;
  GC_TRY(jp_run_packed(ctx, ctx->arena(), &u, bat, gid, seeds, off, tiev, D, round, color_out, &colors, s));

  if (num_colors_out || num_rounds_out) {
    if (num_colors_out) GC_TRY_CUDA(cudaMemsetAsync(num_colors_out, 0, sizeof(int) * G, s));
    batch_results_kernel<<<blocks, 256, 0, s>>>(gs, gid, G, n, color_out, num_colors_out, num_rounds_out);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(cudaStreamSynchronize(s));
  }
  return GC_OK;
}

}  // namespace gc

// ---------------------------------------------------------------------------
// gc_color_batch_list: graphs given as separate device CSRs are packed into
// the disjoint union on the device, coloured by batch_color, and the colours
// copied back to each graph's own output.
// ---------------------------------------------------------------------------
namespace gc {
namespace {

struct ListDesc {  // one graph of the list (device copy of the host array)
  const long long* row_ptr;
  const int* col_idx;
  int* color_out;
};

__device__ __forceinline__ int owner_of(const long long* __restrict__ off, int G, long long x) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void pack_rows_kernel(const ListDesc* __restrict__ d, const long long* __restrict__ voff,
                                 const long long* __restrict__ eoff, int G, long long n,
                                 long long* __restrict__ row_ptr) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v <= n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (v == n) {
      row_ptr[n] = eoff[G];
      continue;
    }
    const int g = owner_of(voff, G, v);
    row_ptr[v] = d[g].row_ptr[v - voff[g]] + eoff[g];
  }
}

__global__ void pack_cols_kernel(const ListDesc* __restrict__ d, const long long* __restrict__ voff,
                                 const long long* __restrict__ eoff, int G, long long nnz,
                                 int* __restrict__ col) {
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < nnz;
       k += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int g = owner_of(eoff, G, k);
    col[k] = d[g].col_idx[k - eoff[g]] + static_cast<int>(voff[g]);
  }
}

__global__ void unpack_colors_kernel(const ListDesc* __restrict__ d, const long long* __restrict__ voff, int G,
                                     long long n, const int* __restrict__ color) {
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int g = owner_of(voff, G, v);
    d[g].color_out[v - voff[g]] = color[v];
  }
}

}  // namespace

gc_status batch_color_list(gc_context* ctx, long long G, const gc_csr* graphs, const gc_job* jobs,
                           int32_t* const* color_out, cudaStream_t s) {
  std::vector<long long> voff(G + 1, 0), eoff(G + 1, 0);
  std::vector<ListDesc> desc(G);
  for (long long g = 0; g < G; ++g) {
    voff[g + 1] = voff[g] + graphs[g].n;
    eoff[g + 1] = eoff[g] + graphs[g].nnz;
    desc[g].row_ptr = reinterpret_cast<const long long*>(graphs[g].row_ptr);
    desc[g].col_idx = graphs[g].col_idx;
    desc[g].color_out = color_out[g];
  }
  const long long n = voff[G], nnz = eoff[G];
  if (n > static_cast<long long>(INT_MAX) - 1) return GC_ERR_OVERFLOW;
  // the packed union lives in the context's pack buffer:
  // desc | voff | eoff | row_ptr | col_idx | colours
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_desc = al(sizeof(ListDesc) * G), b_off = al(sizeof(long long) * (G + 1));
  const size_t b_rp = al(sizeof(long long) * (n + 1)), b_ci = al(sizeof(int) * (nnz > 0 ? nnz : 1));
  const size_t b_col = al(sizeof(int) * (n > 0 ? n : 1));
  GC_TRY(ctx->reserve_pack(b_desc + 2 * b_off + b_rp + b_ci + b_col));
  char* base = static_cast<char*>(ctx->pack);
  ListDesc* ddesc = reinterpret_cast<ListDesc*>(base);
  long long* dvoff = reinterpret_cast<long long*>(base + b_desc);
  long long* deoff = reinterpret_cast<long long*>(base + b_desc + b_off);
  long long* rp = reinterpret_cast<long long*>(base + b_desc + 2 * b_off);
  int* ci = reinterpret_cast<int*>(base + b_desc + 2 * b_off + b_rp);
  int* col = reinterpret_cast<int*>(base + b_desc + 2 * b_off + b_rp + b_ci);
  GC_TRY_CUDA(cudaMemcpyAsync(ddesc, desc.data(), sizeof(ListDesc) * G, cudaMemcpyHostToDevice, s));
  GC_TRY_CUDA(cudaMemcpyAsync(dvoff, voff.data(), sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, s));
  GC_TRY_CUDA(cudaMemcpyAsync(deoff, eoff.data(), sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, s));
  const int blocks = ctx->num_sms * 8;
  const int Gi = static_cast<int>(G);
  pack_rows_kernel<<<blocks, 256, 0, s>>>(ddesc, dvoff, deoff, Gi, n, rp);
  ++g_launches;
  if (nnz > 0) {
    pack_cols_kernel<<<blocks, 256, 0, s>>>(ddesc, dvoff, deoff, Gi, nnz, ci);
    ++g_launches;
  }
  GC_TRY_CUDA(cudaGetLastError());
  gc_batch_csr b;
  b.num_graphs = G;
  b.n = n;
  b.nnz = nnz;
  b.row_ptr = reinterpret_cast<const int64_t*>(rp);
  b.col_idx = ci;
  b.graph_off = reinterpret_cast<const int64_t*>(dvoff);
  GC_TRY(batch_color(ctx, &b, jobs, col, nullptr, nullptr, nullptr, s));
  if (n > 0) {
    unpack_colors_kernel<<<blocks, 256, 0, s>>>(ddesc, dvoff, Gi, n, col);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
  }
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  return GC_OK;
}

}  // namespace gc
