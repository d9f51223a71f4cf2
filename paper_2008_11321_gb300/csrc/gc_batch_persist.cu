// gc_color_batch in ONE persistent launch: every thread block takes whole
// graphs from a device-side queue (largest first) and runs JP-ADG on each
// graph alone, with block barriers as the only synchronisation -- no grid
// barrier, no host round trip between rounds, no waits between blocks.
//
// Per graph (vertex range [v0, v1) of the packed union; its edges stay in
// the range), inside one block:
//
//   ADG (Algorithm 1, Section 3): round l computes T = floor((q+p) Sigma /
//   (q |U|)) (the exact integer form of the threshold), partitions the list
//   U into R = {u : D[u] <= T} (batch[u] = l) and the survivors U', then
//   pushes the UPDATE: every edge (v, w) with v in R and w in U' (batch[w]
//   still 0) decrements D[w]; Sigma' = Sigma - Sigma_R - cut (Section 5,
//   "Caching Sums of Degrees").  Rounds repeat until U' is empty.
//
//   JP (Algorithm 3, Section 4.1) with priority <batch, rho_R, id>, rho_R the
//   graph's seeded hash of the local id: synchronous rounds in which every
//   uncoloured vertex whose predecessors are all coloured takes the smallest
//   colour none of them uses.  A colour word is written once, so a vertex
//   never acts on a wrong value: it either sees a predecessor's final colour
//   or waits for a later round.  The highest-priority uncoloured vertex is
//   always ready, so the rounds end (after the length of the longest path of
//   G_rho), and the colouring is Greedy's in decreasing priority -- the one
//   gc_color_graph gives the graph alone.  Vertices of degree <= 32 are
//   handled one per thread (their colour is at most 33: a 64-bit mask) and
//   resume where they stopped: a vertex that meets an uncoloured predecessor
//   keeps its row position (in D, free after ADG) and its colour mask, so
//   each row is read once over all rounds.  Larger vertices go one per warp
//   with a 1024-colour shared window.
//
// Per-vertex state lives in the union's arrays (graph g at offsets v0..v1),
// so a block's working set is one graph's and stays in L2.  Everything this
// kernel writes (D, batch, the lists, the colours) is read back with
// L2-coherent loads (ld.global.cg, or volatile for the colours), never
// through the SM's L1: a cache line at the boundary of two graphs may have
// been cached by an SM while another block was still writing the other
// graph's half of it.
//
// Both loops are bounded: an ADG round removes at least the vertex of
// smallest degree and a JP round colours at least the highest-priority
// uncoloured vertex; a round that makes no progress (impossible for a valid
// graph) sets the error word and the block moves on.
#include <climits>
#include <cstring>
#include <vector>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kPThreads = 512;
constexpr int kPWarps = kPThreads / kWarp;

struct PGraphArgs {
  const long long* row_ptr;  // union CSR
  const int* col;
  const long long* off;      // graph_off[G+1]
  const gc_job* jobs;        // per graph eps and seed (device)
  const int* order;          // graph ids, largest first
  int G;
  int* D;                    // n: degree in G[U], then degree at removal
  int* la;                   // n: lists (U, U', R; then JP's lists)
  int* lb;
  int* lc;
  int* ld;
  int* batch;                // n
  int* color;                // n
  unsigned long long* used;  // n: JP lane path, colours seen so far (D then holds the row position)
  int* ncol;                 // G or null
  int* nrounds;              // G or null
  unsigned long long* next;  // [0] queue position, [1] error word, [2] sum of |U|, [3] decrements
  int* err;                  // set if a round made no progress
};

__device__ __forceinline__ int p_threshold(unsigned long long sigma, int size_u, unsigned p, unsigned q) {
  if (size_u <= 0) return 0;
  const unsigned __int128 num = static_cast<unsigned __int128>(static_cast<unsigned long long>(q) + p) * sigma;
  const unsigned __int128 den = static_cast<unsigned __int128>(q) * static_cast<unsigned>(size_u);
  const unsigned __int128 t = num / den;
  return t > static_cast<unsigned __int128>(INT_MAX) ? INT_MAX : static_cast<int>(t);
}

// Appends x to list[base + ...] through the block counter *cnt, one atomic
// per warp (all lanes of the warp call it; `want` says who appends).
__device__ __forceinline__ void block_append(bool want, int x, int* list, int* cnt) {
  const unsigned m = __ballot_sync(kFull, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(m) - 1) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(kFull, base, __ffs(m) - 1);
  if (want) list[base + __popc(m & lanemask_lt())] = x;
}

__device__ __forceinline__ unsigned long long pkey(int bat, unsigned h) {
  return (static_cast<unsigned long long>(static_cast<unsigned>(bat)) << 32) | h;
}

__global__ void __launch_bounds__(kPThreads, 3)
batch_persistent_kernel(PGraphArgs A) {
  __shared__ unsigned long long s_sigma, s_sumR, s_cut;
  __shared__ int s_g, s_nU, s_nUn, s_nR, s_T, s_round, s_max;
  __shared__ int s_ns, s_nb, s_nsn, s_nbn;
  __shared__ unsigned s_win[kPWarps][kColorWin / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    if (tid == 0) {
      const unsigned long long k = atomicAdd(A.next, 1ull);
      s_g = k < static_cast<unsigned long long>(A.G) ? A.order[k] : -1;
    }
    __syncthreads();
    const int g = s_g;
    if (g < 0) return;
    const long long v0 = A.off[g], v1 = A.off[g + 1];
    const int n = static_cast<int>(v1 - v0);
    const unsigned p = A.jobs[g].eps_p, q = A.jobs[g].eps_q;
    const unsigned long long seed = A.jobs[g].seed;
    int* U = A.la + v0;
    int* Un = A.lb + v0;
    int* R = A.lc + v0;

    // ---- ADG -------------------------------------------------------------
    if (tid == 0) {
      s_sigma = static_cast<unsigned long long>(A.row_ptr[v1] - A.row_ptr[v0]);
      s_nU = n;
      s_round = 1;
    }
    __syncthreads();
    int rounds = 0;
    unsigned long long work_u = 0, work_dec = 0;  // (thread 0) sum of |U| and of the cuts
    while (n > 0) {
      if (tid == 0) {
        s_T = p_threshold(s_sigma, s_nU, p, q);
        s_nUn = 0;
        s_nR = 0;
        s_sumR = 0;
        s_cut = 0;
      }
      __syncthreads();
      const int round = s_round, T = s_T, nU = s_nU;
      const bool first = round == 1;
      unsigned long long sum_r = 0;
      for (int base = 0; base < nU; base += kPThreads) {
        const int i = base + tid;
        const bool active = i < nU;
        int u = 0, d = 0;
        if (active) {
          if (first) {
            u = static_cast<int>(v0) + i;
            d = static_cast<int>(A.row_ptr[u + 1] - A.row_ptr[u]);
            A.D[u] = d;
          } else {
            u = __ldcg(U + i);
            if (u < v0 || u >= v1) {  // not this graph's vertex: record it, skip it
              atomicExch(A.err, 2);
              u = static_cast<int>(v0);
            }
            d = __ldcg(A.D + u);
          }
        }
        const bool in_r = active && d <= T;
        if (in_r) {
          A.batch[u] = round;
          sum_r += static_cast<unsigned long long>(d);
        }
        block_append(in_r, u, R, &s_nR);
        block_append(active && !in_r, u, Un, &s_nUn);
      }
      sum_r = warp_sum(sum_r);
      if (lane == 0 && sum_r) atomicAdd(&s_sumR, sum_r);
      __syncthreads();
      rounds = round;
      const int nUn = s_nUn, nR = s_nR;
      work_u += static_cast<unsigned long long>(nU);
      if (nUn == 0) break;  // U is empty: nothing left to decrement
      if (nUn >= nU) {      // no vertex left U: cannot happen for a valid graph
        if (tid == 0) atomicExch(A.err, 1);
        break;
      }
      // push UPDATE over R's rows: 32 rows per warp, edges spread over lanes
      unsigned long long cut = 0;
      for (int tile = warp; tile * 32 < nR; tile += kPWarps) {
        const int t = tile * 32 + lane;
        long long st = 0;
        int len = 0;
        if (t < nR) {
          const int v = __ldcg(R + t);
          if (v >= v0 && v < v1) {
            st = A.row_ptr[v];
            len = static_cast<int>(A.row_ptr[v + 1] - st);
          } else {
            atomicExch(A.err, 2);
          }
        }
        sweep_tile(
            st, len, 0, A.col, [&](int w, int) { return __ldcg(A.batch + w); },
            [&](int w, int, int bw) {
              if (bw == 0) {  // w is in U'
                ++cut;
                atomicSub(&A.D[w], 1);
              }
            });
      }
      cut = warp_sum(cut);
      if (lane == 0 && cut) atomicAdd(&s_cut, cut);
      __syncthreads();
      if (tid == 0) {
        work_dec += s_cut;
        s_sigma = s_sigma - s_sumR - s_cut;
        s_nU = nUn;
        s_round = round + 1;
      }
      int* tmp = U;
      U = Un;
      Un = tmp;
      __syncthreads();
    }

    // ---- JP ----------------------------------------------------------------
    // lists: lane path (degree <= 32) in la/lb, warp path in lc/ld
    int* Ls = A.la + v0;
    int* Lsn = A.lb + v0;
    int* Lb = A.lc + v0;
    int* Lbn = A.ld + v0;
    if (tid == 0) {
      s_ns = 0;
      s_nb = 0;
      s_max = 0;
    }
    __syncthreads();
    int local_max = 0;
    for (int base = 0; base < n; base += kPThreads) {
      const int i = base + tid;
      const bool active = i < n;
      int v = 0;
      long long deg = 0;
      if (active) {
        v = static_cast<int>(v0) + i;
        deg = A.row_ptr[v + 1] - A.row_ptr[v];
        A.color[v] = deg == 0 ? 1 : 0;  // isolated: no predecessor, colour 1
        if (deg == 0) local_max = 1;
        if (deg > 0 && deg <= kSmallDeg) {  // lane path: start of the row, no colour seen
          A.D[v] = 0;
          A.used[v] = 0ull;
        }
      }
      block_append(active && deg > 0 && deg <= kSmallDeg, v, Ls, &s_ns);
      block_append(active && deg > kSmallDeg, v, Lb, &s_nb);
    }
    __syncthreads();
    volatile int* vcol = A.color;
    for (;;) {
      const int ns = s_ns, nb = s_nb;
      if (ns == 0 && nb == 0) break;
      if (tid == 0) {
        s_nsn = 0;
        s_nbn = 0;
      }
      __syncthreads();
      // lane path
      for (int base = 0; base < ns; base += kPThreads) {
        const int i = base + tid;
        bool pending = false;
        int v = 0;
        if (i < ns) {
          v = __ldcg(Ls + i);
          if (v < v0 || v >= v1) {  // not this graph's vertex: record it, skip it
            atomicExch(A.err, 2);
            v = static_cast<int>(v0);
          }
          const unsigned long long kv = pkey(__ldcg(A.batch + v), tie_hash(seed, static_cast<unsigned>(v - v0)));
          const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
          int pos = __ldcg(A.D + v);
          if (pos < 0 || pos > e - s) {  // a resume position outside the row: record it, restart
            atomicExch(A.err, 3);
            pos = 0;
          }
          unsigned long long used = pos > 0 ? __ldcg(A.used + v) : 0ull;
          long long k = s + pos;
          for (; k < e; ++k) {
            const int w = __ldg(A.col + k);
            const unsigned long long kw = pkey(__ldcg(A.batch + w), tie_hash(seed, static_cast<unsigned>(w - v0)));
            if (kw > kv || (kw == kv && w > v)) {
              const int c = vcol[w];
              if (c == 0) {
                pending = true;
                break;
              }
              if (c <= 64) used |= 1ull << (c - 1);
            }
          }
          if (pending) {  // resume here next round
            A.D[v] = static_cast<int>(k - s);
            A.used[v] = used;
          } else {
            const int c = __ffsll(static_cast<long long>(~used));
            vcol[v] = c;
            local_max = c > local_max ? c : local_max;
          }
        }
        block_append(pending, v, Lsn, &s_nsn);
      }
      // warp path: one vertex per warp
      unsigned* win = s_win[warp];
      for (int i = warp; i < nb; i += kPWarps) {
        int v = __ldcg(Lb + i);
        if (v < v0 || v >= v1) {
          if (lane == 0) atomicExch(A.err, 2);
          v = static_cast<int>(v0);
        }
        const unsigned long long kv = pkey(__ldcg(A.batch + v), tie_hash(seed, static_cast<unsigned>(v - v0)));
        const long long s = A.row_ptr[v], e = A.row_ptr[v + 1];
        int c = 0;
        bool pending = false;
        for (int wbase = 0; c == 0 && !pending; wbase += kColorWin) {
          win[lane] = 0u;
          __syncwarp();
          bool miss = false;
          for (long long k = s + lane; k < e; k += 32) {
            const int w = __ldg(A.col + k);
            const unsigned long long kw = pkey(__ldcg(A.batch + w), tie_hash(seed, static_cast<unsigned>(w - v0)));
            if (kw > kv || (kw == kv && w > v)) {
              const int cw = vcol[w];
              if (cw == 0) {
                miss = true;
              } else if (cw > wbase && cw <= wbase + kColorWin) {
                atomicOr(&win[(cw - wbase - 1) >> 5], 1u << ((cw - wbase - 1) & 31));
              }
            }
          }
          pending = __any_sync(kFull, miss);
          __syncwarp();
          if (!pending) {
            const unsigned freeb = ~win[lane];
            const unsigned fm = __ballot_sync(kFull, freeb != 0u);
            if (fm) {
              const int f = __ffs(fm) - 1;
              c = wbase + f * 32 + __ffs(__shfl_sync(kFull, freeb, f));
            }
          }
          __syncwarp();
        }
        if (lane == 0) {
          if (pending) {
            Lbn[atomicAdd(&s_nbn, 1)] = v;
          } else {
            vcol[v] = c;
            local_max = c > local_max ? c : local_max;
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (s_nsn + s_nbn >= ns + nb) {  // nothing coloured: cannot happen
          atomicExch(A.err, 1);
          s_nsn = s_nbn = 0;
        }
        s_ns = s_nsn;
        s_nb = s_nbn;
      }
      int* t1 = Ls;
      Ls = Lsn;
      Lsn = t1;
      int* t2 = Lb;
      Lb = Lbn;
      Lbn = t2;
      __syncthreads();
    }
    local_max = warp_max(local_max);
    if (lane == 0 && local_max) atomicMax(&s_max, local_max);
    __syncthreads();
    if (tid == 0) {
      if (A.ncol) A.ncol[g] = s_max;
      if (A.nrounds) A.nrounds[g] = rounds;
      if (work_u) atomicAdd(A.next + 2, work_u);
      if (work_dec) atomicAdd(A.next + 3, work_dec);
    }
    __syncthreads();
  }
}

// Graph ids by decreasing number of CSR entries (then increasing id): the
// sort key is ~nnz_g << 32 | g.
__global__ void batch_order_keys_kernel(const long long* __restrict__ off, const long long* __restrict__ row_ptr,
                                        int G, unsigned long long* __restrict__ keys, int* __restrict__ vals,
                                        long long* __restrict__ maxes) {
  long long mn = 0, mm = 0;
  for (long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < G;
       g += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long n = off[g + 1] - off[g];
    const long long m = row_ptr[off[g + 1]] - row_ptr[off[g]];
    keys[g] = (static_cast<unsigned long long>(~static_cast<unsigned>(m > 0xffffffffll ? 0xffffffffll : m)) << 32) |
              static_cast<unsigned>(g);
    vals[g] = static_cast<int>(g);
    mn = n > mn ? n : mn;
    mm = m > mm ? m : mm;
  }
  mn = warp_max(mn);
  mm = warp_max(mm);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned long long*>(&maxes[0]), static_cast<unsigned long long>(mn));
    atomicMax(reinterpret_cast<unsigned long long*>(&maxes[1]), static_cast<unsigned long long>(mm));
  }
}

}  // namespace

size_t batch_persistent_scratch_bytes(long long n, long long G) {
  const size_t vb = (static_cast<size_t>(n > 0 ? n : 1) * 4 + 255) & ~size_t(255);
  const size_t gb = static_cast<size_t>(G) + 1;
  // D, four lists, an internal batch array, JP's colour masks; the queue's
  // sort buffers
  return 6 * vb + (static_cast<size_t>(n > 0 ? n : 1) * 8 + 256) + 2 * (gb * 8 + 256) + 2 * (gb * 4 + 256) + sort_hist_elems(G) * 8 +
         (scan_temp_elems(static_cast<long long>(sort_hist_elems(G))) + 1) * 8 + 4096;
}

// The queue order and the largest graph (vertices, CSR entries): returns the
// sorted graph ids in *order_out (device) and the maxima on the host.
gc_status batch_order(gc_context* ctx, Arena& a, const gc_batch_csr* b, int** order_out, long long* max_n,
                      long long* max_nnz, cudaStream_t s) {
  const int G = static_cast<int>(b->num_graphs);
  SortBufs sb;
  sb.keys[0] = a.take<unsigned long long>(G);
  sb.keys[1] = a.take<unsigned long long>(G);
  sb.vals[0] = a.take<int>(G);
  sb.vals[1] = a.take<int>(G);
  sb.hist = a.take<long long>(sort_hist_elems(G));
  sb.temp = a.take<long long>(scan_temp_elems(static_cast<long long>(sort_hist_elems(G))) + 1);
  long long* maxes = a.take<long long>(2);
  if (!sb.keys[0] || !sb.keys[1] || !sb.vals[0] || !sb.vals[1] || !sb.hist || !sb.temp || !maxes) return GC_ERR_OOM;
  GC_TRY_CUDA(cudaMemsetAsync(maxes, 0, 2 * sizeof(long long), s));
  batch_order_keys_kernel<<<(G + 255) / 256 < 1024 ? (G + 255) / 256 : 1024, 256, 0, s>>>(
      reinterpret_cast<const long long*>(b->graph_off), reinterpret_cast<const long long*>(b->row_ptr), G,
      sb.keys[0], sb.vals[0], maxes);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  cudaError_t err = cudaSuccess;
  const int res = radix_sort_pairs(sb, G, 0xffu, s, &err);  // bytes 0..7: the whole key
  GC_TRY_CUDA(err);
  long long* pin = static_cast<long long*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, maxes, 2 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  *max_n = pin[0];
  *max_nnz = pin[1];
  *order_out = sb.vals[res];
  return GC_OK;
}

gc_status batch_color_persistent(gc_context* ctx, Arena a, const gc_batch_csr* b, const gc_job* djobs,
                                 const int* order, int32_t* color_out, int32_t* batch_out, int32_t* num_colors_out,
                                 int32_t* num_rounds_out, cudaStream_t s) {
  const long long n = b->n;
  const int G = static_cast<int>(b->num_graphs);
  PGraphArgs A{};
  A.row_ptr = reinterpret_cast<const long long*>(b->row_ptr);
  A.col = b->col_idx;
  A.off = reinterpret_cast<const long long*>(b->graph_off);
  A.jobs = djobs;
  A.order = order;
  A.G = G;
  const size_t cnt = static_cast<size_t>(n > 0 ? n : 1);
  A.D = a.take<int>(cnt);
  A.la = a.take<int>(cnt);
  A.lb = a.take<int>(cnt);
  A.lc = a.take<int>(cnt);
  A.ld = a.take<int>(cnt);
  A.batch = batch_out ? batch_out : a.take<int>(cnt);
  A.used = a.take<unsigned long long>(cnt);
  A.color = color_out;
  A.ncol = num_colors_out;
  A.nrounds = num_rounds_out;
  A.next = a.take<unsigned long long>(4);
  if (!A.D || !A.la || !A.lb || !A.lc || !A.ld || !A.batch || !A.used || !A.next) return GC_ERR_OOM;
  A.err = reinterpret_cast<int*>(A.next + 1);
  if (n > 0) GC_TRY_CUDA(cudaMemsetAsync(A.batch, 0, sizeof(int) * n, s));
  GC_TRY_CUDA(cudaMemsetAsync(A.next, 0, 4 * sizeof(unsigned long long), s));
  int per_sm = 0;
  GC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, kPThreads, 0));
  if (per_sm < 1) per_sm = 1;
  long long grid = static_cast<long long>(ctx->num_sms) * per_sm;
  if (grid > G) grid = G;
  ctx->timer_begin(gc_context::kTUpdate, s);
  batch_persistent_kernel<<<static_cast<int>(grid), kPThreads, 0, s>>>(A);
  ++g_launches;
  ctx->timer_end(s);
  GC_TRY_CUDA(cudaGetLastError());
  unsigned long long* pin = static_cast<unsigned long long*>(ctx->pinned);
  GC_TRY_CUDA(cudaMemcpyAsync(pin, A.next, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  ctx->stats.sum_U = static_cast<int64_t>(pin[2]);
  ctx->stats.sum_decrements = static_cast<int64_t>(pin[3]);
  // 1: a round without progress, 2: a list entry outside its graph, 3: a
  // resume position outside its row -- none can happen for a valid batch
  return *reinterpret_cast<int*>(pin + 1) ? GC_ERR_CUDA : GC_OK;
}

}  // namespace gc
