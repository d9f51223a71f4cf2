// ADG, Algorithm 1 (Section 3), as three kernels per round:
//
//   partition  R = {u in U : D[u] <= T}  (T = floor((q+p)*Sigma / (q*|U|)),
//              the exact integer form of D[u] <= (1+eps)*Sigma/|U|);
//              batch[R] = l; U' = U \ R compacted into the other U buffer
//              (the contiguous [R | U] layout of Section 5.1, kept as a list);
//              each removed vertex's adjacency is cut into UPDATE tasks of at
//              most kChunk edges; Sigma_R = sum of D over R is reduced.
//   update     push-style UPDATE: for every task edge (v, w) with w still in
//              U' (its bit in the liveness bitmap) an atomic decrement of D[w]
//              (DecrementAndFetch, Section 2.4); the number of decrements is
//              the cut (R, U').  Edges are spread over the lanes of a warp
//              across 32 tasks at a time, so short and long rows mix.
//   finalize   Sigma' = Sigma - Sigma_R - cut (Section 5, "Caching Sums of
//              Degrees"), |U| = |U'|, next T, l = l + 1.
//
// A round may pull instead of push (Section 5, "Push vs. Pull"; the CREW
// form of Algorithm 2): every survivor v in U' recounts D[v] as the number of
// its neighbours still live after the partition, so no two threads update
// the same word with contention, and Sigma' is the sum of the recounts (the
// cut follows as Sigma - Sigma_R - Sigma').  Push sweeps the rows of R, pull
// the rows of U'; the direction is chosen per round on the device
// (adg_pulls) from the two row sums, which the partition and finalize carry.
//
// Round 1 reads U = V implicitly (no list) and writes every vertex's D.
//
// Hubs.  Rounds 2-5 of a power-law graph send most decrements to a few
// thousand high-degree vertices, and atomics on one word serialise in its L2
// slice.  Before round 1 a degree histogram picks a power-of-two degree
// threshold that marks at most `update_hubs` vertices (gc_options) as hubs;
// their bit sits beside the liveness bit (one 8-byte gather per edge gives
// both), and UPDATE counts decrements aimed at hubs first per warp step
// (__match_any_sync), then per block in a shared-memory hash table, and adds
// each hub's count to D once per block at the end.  The decrements are the
// same, only merged: D, the cut and every result are unchanged.
//
// UPDATE tests "w still in U" on a bitmap (n bits) rather than on batch[]
// (n ints): the test is a random gather per edge, and a 2 MB bitmap for 2^24
// vertices stays in L2 next to the decremented D words, where a 64 MB array
// would not (random 4-byte gathers run several times faster from L2 than from
// HBM).  Round 1's partition visits the vertices in order and writes whole
// bitmap words; later rounds clear the bits of removed vertices.
// A host-driven round loop reads |U| after every round to stop; the number of
// rounds is O(log n) (the round-bound lemma of Section 3) and is single-digit
// on the power-law workloads.  A repeated call runs rounds 2 on as one CUDA
// graph whose finalize kernel decides on the device whether to go on
// (adg_round_graph below).
#include <climits>
#include <cstring>
#include <mutex>

#include "gc_internal.cuh"

namespace gc {
namespace {

constexpr int kAdgThreads = 256;
constexpr int kMaxHubs = 4096;  // gc_options.update_hubs at most

__device__ __forceinline__ int adg_threshold(unsigned long long sigma, int size_u, unsigned p,
                                             unsigned q) {
  if (size_u <= 0) return 0;
  unsigned __int128 num = static_cast<unsigned __int128>(static_cast<unsigned long long>(q) + p) * sigma;
  unsigned __int128 den = static_cast<unsigned __int128>(q) * static_cast<unsigned>(size_u);
  unsigned __int128 t = num / den;
  return t > static_cast<unsigned __int128>(INT_MAX) ? INT_MAX : static_cast<int>(t);
}

__global__ void adg_init_kernel(AdgCtl* ctl, long long n, long long nnz, unsigned p, unsigned q, int mode,
                                int pull_percent) {
  AdgCtl c{};
  c.sigma = static_cast<unsigned long long>(nnz);
  c.rows_U = static_cast<unsigned long long>(nnz);
  c.size_U = static_cast<int>(n);
  c.round = 1;
  c.p = p;
  c.q = q;
  c.mode = mode;
  c.pull_percent = pull_percent;
  c.hub_min_degree = INT_MAX;
  c.T = adg_threshold(c.sigma, c.size_U, p, q);
  *ctl = c;
}

// Hub threshold: counts of vertices by floor(log2 degree), then the smallest
// power of two 2^k >= 256 with at most max_hubs vertices of degree >= 2^k.
__global__ void adg_hub_hist_kernel(const long long* __restrict__ row_ptr, long long n,
                                    unsigned long long* __restrict__ hist) {
  __shared__ unsigned s_h[64];
  if (threadIdx.x < 64) s_h[threadIdx.x] = 0u;
  __syncthreads();
  for (long long v = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
       v += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long d = static_cast<unsigned long long>(row_ptr[v + 1] - row_ptr[v]);
    if (d >= 256) atomicAdd(&s_h[63 - __clzll(d)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 64 && s_h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_h[threadIdx.x]);
}

__global__ void adg_hub_pick_kernel(const unsigned long long* __restrict__ hist, int max_hubs, AdgCtl* ctl) {
  unsigned long long above = 0;
  int k = 64;
  while (k > 8 && above + hist[k - 1] <= static_cast<unsigned long long>(max_hubs)) {
    above += hist[k - 1];
    --k;
  }
  // vertices of degree >= 2^k number `above` <= max_hubs
  ctl->hub_min_degree = (k >= 31 || above == 0) ? INT_MAX : (1 << k);
  ctl->hub_cap = max_hubs;
}

// The partition's work on one block step of K vertices per thread (vertex
// i = base + j * blockDim.x + threadIdx.x for j < K, so each j is a coalesced
// run): all K vertices' loads are issued before any decision, and the step's
// survivors and UPDATE tasks are appended with one atomic per list for the
// whole block (block_reserve) rather than one per warp on the same word.
template <int K>
__device__ __forceinline__ void adg_partition_steps(
    AdgCtl* __restrict__ ctl, const long long* __restrict__ row_ptr, int* __restrict__ D, int* __restrict__ batch,
    const int* __restrict__ u_in, int* __restrict__ u_out, long long* __restrict__ task_start,
    int* __restrict__ task_len, uint2* __restrict__ live, bool first, long long size_u,
    const unsigned long long* __restrict__ mkeys, const unsigned long long* __restrict__ kstar,
    int* __restrict__ hub_base, int* __restrict__ hub_vertex, int round, int T, int hub_min,
    unsigned long long& sum_r, unsigned long long& rows_r, int& max_d) {
  __shared__ int s_keep[2][kAdgThreads / 32];
  __shared__ unsigned long long s_task[2][kAdgThreads / 32];
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt();
  const long long span = static_cast<long long>(blockDim.x) * K;
  const long long stride = static_cast<long long>(gridDim.x) * span;
  int par = 0;
  // base is the same for every thread of the block: the barriers inside
  // block_reserve are reached by all of them on every step
  for (long long base = static_cast<long long>(blockIdx.x) * span; base < size_u; base += stride, par ^= 1) {
    int u[K], d[K], nt[K], incl[K];
    long long rs[K], re[K];
    bool in_r[K], keep[K];
    unsigned km[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long i = base + static_cast<long long>(j) * blockDim.x + threadIdx.x;
      const bool active = i < size_u;
      u[j] = 0;
      d[j] = 0;
      rs[j] = 0;
      re[j] = 0;
      if (active) {
        if (first) {
          u[j] = static_cast<int>(i);
          rs[j] = row_ptr[u[j]];
          re[j] = row_ptr[u[j] + 1];
          d[j] = static_cast<int>(re[j] - rs[j]);
        } else {
          u[j] = u_in[i];
          d[j] = D[u[j]];
        }
      }
      // ADG: D[u] <= T; ADG-M: the key D[u] * 2^32 + u of list entry i is at
      // most the selected ceil(|U|/2)-th smallest key
      in_r[j] = active && (mkeys ? mkeys[i] <= *kstar : d[j] <= T);
      keep[j] = active && !in_r[j];
    }
    // removed vertices' rows (round 1 has them already) -> UPDATE tasks of at
    // most kChunk edges
    if (!first) {
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
    // survivors -> U'
    int kb = slot.a;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (keep[j]) u_out[kb + __popc(km[j] & lt)] = u[j];
      kb += __popc(km[j]);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const long long i = base + static_cast<long long>(j) * blockDim.x + threadIdx.x;
      const bool active = i < size_u;
      // liveness bitmap: round 1 writes the warp's word pair (vertices
      // i = 32 w .. 32 w + 31, since every run starts at a multiple of 32:
      // live bits, hub bits); later rounds clear live bits
      if (first) {
        const unsigned hm = __ballot_sync(kFull, active && d[j] >= hub_min);
        if (lane == 0 && active) live[i >> 5] = make_uint2(km[j], hm);
        // hub ranks: the word's hubs take consecutive ranks from
        // hub_base[word] on, in bit order (the hub of bit b has rank
        // hub_base + popc(hm & (2^b - 1)))
        if (hm && hub_base) {
          int hb = 0;
          if (lane == 0) {
            hb = atomicAdd(&ctl->n_hubs, __popc(hm));
            hub_base[i >> 5] = hb;
          }
          hb = __shfl_sync(kFull, hb, 0) + __popc(hm & lt);
          if (((hm >> lane) & 1u) && hb < ctl->hub_cap) hub_vertex[hb] = u[j];
        }
        // D[u] is written for every vertex in round 1; for a removed vertex
        // it then keeps its degree at removal, |{w in N(u) : batch(w) >=
        // batch(u)}|, which bounds u's predecessor count in JP.
        if (active) D[u[j]] = d[j];
      } else if (in_r[j]) {
        atomicAnd(&live[u[j] >> 5].x, ~(1u << (u[j] & 31)));
      }
      if (in_r[j]) {
        batch[u[j]] = round;
        sum_r += static_cast<unsigned long long>(d[j]);
        max_d = d[j] > max_d ? d[j] : max_d;
        rows_r += static_cast<unsigned long long>(re[j] - rs[j]);
      }
    }
    if (first) continue;  // round 1's UPDATE sweeps vertex tiles, no task list
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
        if (x < tot) {
          task_start[tb + x] = st;
          task_len[tb + x] = static_cast<int>(rej - st < kChunk ? rej - st : kChunk);
        }
      }
      tb += static_cast<unsigned long long>(tot);
    }
  }
}

// Vertices per thread and block step on rounds large enough to give every
// thread of the grid that many.
constexpr int kPartItems = 4;

__global__ void __launch_bounds__(kAdgThreads, 4)  // 64 registers: 4 blocks per SM
adg_partition_kernel(AdgCtl* __restrict__ ctl, const long long* __restrict__ row_ptr,
                     int* __restrict__ D, int* __restrict__ batch, const int* __restrict__ u_in,
                     int* __restrict__ u_out, long long* __restrict__ task_start,
                     int* __restrict__ task_len, uint2* __restrict__ live, int first_round_n,
                     const unsigned long long* __restrict__ mkeys = nullptr,
                     const unsigned long long* __restrict__ kstar = nullptr, int* __restrict__ hub_base = nullptr,
                     int* __restrict__ hub_vertex = nullptr) {
  const int round = ctl->round;
  const int T = ctl->T;
  const int hub_min = ctl->hub_min_degree;
  const bool first = first_round_n > 0;
  const long long size_u = first ? first_round_n : ctl->size_U;
  const int lane = threadIdx.x & 31;
  unsigned long long sum_r = 0, rows_r = 0;
  int max_d = 0;
  // the same choice in every block: size_u and the grid are the kernel's
  if (size_u >= static_cast<long long>(gridDim.x) * blockDim.x * kPartItems)
    adg_partition_steps<kPartItems>(ctl, row_ptr, D, batch, u_in, u_out, task_start, task_len, live, first, size_u,
                                    mkeys, kstar, hub_base, hub_vertex, round, T, hub_min, sum_r, rows_r, max_d);
  else
    adg_partition_steps<1>(ctl, row_ptr, D, batch, u_in, u_out, task_start, task_len, live, first, size_u, mkeys,
                           kstar, hub_base, hub_vertex, round, T, hub_min, sum_r, rows_r, max_d);
  sum_r = warp_sum(sum_r);
  rows_r = warp_sum(rows_r);
  if (lane == 0 && sum_r) atomicAdd(&ctl->sum_R, sum_r);
  if (lane == 0 && rows_r) atomicAdd(&ctl->rows_R, rows_r);
  max_d = warp_max(max_d);
  if (lane == 0 && max_d > 0) atomicMax(&ctl->max_removal_degree, max_d);
}

// Round 1 (vertex_tiles != 0): lane l of a warp owns vertex 32*tile + l and
// sweeps its row if it was removed in round 1 (degree <= T_1, no chunking
// needed since T_1 is the average degree bound).  Later rounds sweep the task
// list written by the partition.  With kHubs, decrements aimed at hubs (the
// second bit of the live word pair) are counted in the block's shared array
// at the hub's rank (hub_base[w / 32] + the hubs below w in its word) and
// reach D once per hub and block at the end.
template <bool kHubs>
__global__ void __launch_bounds__(kAdgThreads)
adg_update_kernel(AdgCtl* __restrict__ ctl, const long long* __restrict__ row_ptr,
                  const int* __restrict__ col, int* __restrict__ D, const int* __restrict__ batch,
                  const uint2* __restrict__ live, const long long* __restrict__ task_start,
                  const int* __restrict__ task_len, long long vertex_tiles_n, const int* __restrict__ hub_base,
                  const int* __restrict__ hub_vertex, long long vertex_lo = 0) {
  extern __shared__ int s_hub[];
  // The last round leaves U empty: no neighbour can still be in U, so there
  // is nothing to decrement (and the cut is not needed any more).  A pull
  // round recounts instead (adg_pull_*).
  if (ctl->size_Unext == 0 || adg_pulls(*ctl)) return;
  int nh = 0;
  if (kHubs) {
    nh = min(ctl->n_hubs, ctl->hub_cap);
    for (int i = threadIdx.x; i < nh; i += blockDim.x) s_hub[i] = 0;
    __syncthreads();
  }
  const int round = ctl->round;
  // round 1: the vertices [vertex_lo, vertex_tiles_n)
  const unsigned long long ntasks =
      vertex_tiles_n > 0 ? static_cast<unsigned long long>(vertex_tiles_n - vertex_lo) : ctl->ntasks;
  const int lane = threadIdx.x & 31;
  const unsigned long long gwarp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = (static_cast<unsigned long long>(gridDim.x) * blockDim.x) >> 5;
  unsigned long long cut = 0;
  for (unsigned long long tile = gwarp; tile * 32 < ntasks; tile += nwarps) {
    const unsigned long long t = tile * 32 + lane;
    long long st = 0;
    int len = 0;
    if (t < ntasks) {
      if (vertex_tiles_n > 0) {
        const long long x = vertex_lo + static_cast<long long>(t);
        if (batch[x] == round) {
          st = row_ptr[x];
          len = static_cast<int>(row_ptr[x + 1] - st);
        }
      } else {
        st = task_start[t];
        len = task_len[t];
      }
    }
    // gathered per neighbour w: bit 0 live, bit 1 hub, bits 2.. the hubs
    // below w in its word
    // the hub variant at 6 edges per lane and step stays at 40 registers
    sweep_tile<kHubs ? 6 : 8>(
        st, len, 0, col,
        [&](int w, int) {
          const uint2 lw = __ldg(live + (w >> 5));
          const unsigned b = static_cast<unsigned>(w) & 31u;
          unsigned r = (lw.x >> b) & 1u;
          if (kHubs) r |= (((lw.y >> b) & 1u) << 1) | (static_cast<unsigned>(__popc(lw.y & ((1u << b) - 1u))) << 2);
          return r;
        },
        [&](int w, int, unsigned g) {
          if (!(g & 1u)) return;  // w is no longer in U
          ++cut;
          if (kHubs && (g & 2u)) {
            const int h = __ldg(hub_base + (w >> 5)) + static_cast<int>(g >> 2);
            if (h < nh) {
              atomicAdd(&s_hub[h], 1);
              return;
            }
          }
          atomicSub(&D[w], 1);
        });
  }
  cut = warp_sum(cut);
  if (lane == 0 && cut) atomicAdd(&ctl->cut, cut);
  if (kHubs) {
    __syncthreads();
    for (int i = threadIdx.x; i < nh; i += blockDim.x) {
      const int c = s_hub[i];
      if (c) atomicSub(&D[hub_vertex[i]], c);
    }
  }
}

// Pull round, step 1: every survivor v of U' (the list the partition wrote)
// gets D[v] = 0 and its row cut into tasks of at most kChunk entries
// (vertex, start, length), appended warp by warp.
__global__ void __launch_bounds__(kAdgThreads)
adg_pull_tasks_kernel(AdgCtl* __restrict__ ctl, const long long* __restrict__ row_ptr, int* __restrict__ D,
                      const int* __restrict__ u_next, long long* __restrict__ task_start,
                      int* __restrict__ task_len, int* __restrict__ task_v) {
  if (!adg_pulls(*ctl)) return;
  const long long size_un = ctl->size_Unext;
  const int lane = threadIdx.x & 31;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x; base < size_un; base += stride) {
    const long long i = base + threadIdx.x;
    int v = 0, nt = 0;
    long long rs = 0, re = 0;
    if (i < size_un) {
      v = u_next[i];
      D[v] = 0;
      rs = row_ptr[v];
      re = row_ptr[v + 1];
      nt = static_cast<int>((re - rs + kChunk - 1) / kChunk);
    }
    const int incl = warp_inclusive_scan(nt);
    const int tot = __shfl_sync(kFull, incl, 31);
    const int excl = incl - nt;
    unsigned long long tbase = 0;
    if (lane == 31 && tot) tbase = atomicAdd(&ctl->ntasks_pull, static_cast<unsigned long long>(tot));
    tbase = __shfl_sync(kFull, tbase, 31);
    for (int b = 0; b < tot; b += 32) {
      const int x = b + lane;
      int j = 0;  // owner: the largest lane j with excl_j <= x
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int c = j + step;
        if (__shfl_sync(kFull, excl, c) <= x) j = c;
      }
      const long long st = __shfl_sync(kFull, rs, j) +
                           static_cast<long long>(x - __shfl_sync(kFull, excl, j)) * kChunk;
      const long long rej = __shfl_sync(kFull, re, j);
      const int vj = __shfl_sync(kFull, v, j);
      if (x < tot) {
        task_start[tbase + x] = st;
        task_len[tbase + x] = static_cast<int>(rej - st < kChunk ? rej - st : kChunk);
        task_v[tbase + x] = vj;
      }
    }
  }
}

// Pull round, step 2: each task counts its row's live neighbours (the
// bitmap already excludes this round's R); counts of the same task are
// merged by the warp in shared memory, then added to D[v] once per task.
// The sum of all counts is Sigma' = sum of D over U'.
__global__ void __launch_bounds__(kAdgThreads)
adg_pull_count_kernel(AdgCtl* __restrict__ ctl, const int* __restrict__ col, int* __restrict__ D,
                      const uint2* __restrict__ live, const long long* __restrict__ task_start,
                      const int* __restrict__ task_len, const int* __restrict__ task_v) {
  __shared__ int s_cnt[kAdgThreads / 32][32];
  if (!adg_pulls(*ctl)) return;
  const unsigned long long ntasks = ctl->ntasks_pull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long gwarp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = (static_cast<unsigned long long>(gridDim.x) * blockDim.x) >> 5;
  int* cnt = s_cnt[warp];
  unsigned long long total = 0;
  for (unsigned long long tile = gwarp; tile * 32 < ntasks; tile += nwarps) {
    const unsigned long long t = tile * 32 + lane;
    long long st = 0;
    int len = 0;
    if (t < ntasks) {
      st = task_start[t];
      len = task_len[t];
    }
    cnt[lane] = 0;
    __syncwarp();
    sweep_tile(
        st, len, lane, col, [&](int w, int) { return (__ldg(live + (w >> 5)).x >> (w & 31)) & 1u; },
        [&](int, int j, unsigned lv) {
          // lanes of this step holding edges of the same task add once
          const unsigned act = __activemask();
          const unsigned lm = __ballot_sync(act, lv != 0u);
          const unsigned grp = __match_any_sync(act, j);
          const unsigned mine = grp & lm;
          if (lv && (mine & lanemask_lt()) == 0) atomicAdd(&cnt[j], __popc(mine));
        });
    __syncwarp();
    const int c = cnt[lane];
    if (t < ntasks && c) {
      atomicAdd(&D[task_v[t]], c);
      total += static_cast<unsigned long long>(c);
    }
    __syncwarp();
  }
  total = warp_sum(total);
  if (lane == 0 && total) atomicAdd(&ctl->pull_sigma, total);
}

__device__ __forceinline__ void adg_finalize(AdgCtl* ctl) {
  AdgCtl c = *ctl;
  c.total_U += static_cast<unsigned long long>(c.size_U);
  if (adg_pulls(c)) {  // Sigma' is the recount; the cut follows from it
    c.cut = c.sigma - c.sum_R - c.pull_sigma;
    c.sigma = c.pull_sigma;
    ++c.pull_rounds;
  } else {
    c.sigma = c.sigma - c.sum_R - c.cut;
  }
  c.total_dec += c.cut;
  c.rows_U -= c.rows_R;
  c.size_U = c.size_Unext;
  c.round += 1;
  c.T = adg_threshold(c.sigma, c.size_U, c.p, c.q);
  c.sum_R = 0;
  c.rows_R = 0;
  c.cut = 0;
  c.pull_sigma = 0;
  c.ntasks = 0;
  c.ntasks_pull = 0;
  c.size_Unext = 0;
  *ctl = c;
}

__global__ void adg_finalize_kernel(AdgCtl* ctl) { adg_finalize(ctl); }

// The graph-launched loop's finalize: a round whose U was already empty is
// a no-op and ends the loop; so does a round that removed no vertex (cannot
// happen; reported); else the usual finalize, and the loop goes on while U
// holds vertices.
__global__ void adg_finalize_graph_kernel(AdgCtl* ctl, cudaGraphConditionalHandle loop) {
  const int prev = ctl->size_U;
  if (prev == 0) {
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  if (ctl->size_Unext >= prev) {
    ctl->graph_err = 1;
    ctl->size_U = 0;
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  adg_finalize(ctl);
  cudaGraphSetConditional(loop, ctl->size_U > 0 ? 1u : 0u);
}

// ADG's rounds from round 2 on as one CUDA graph loop (gc_graph.cu): the
// body holds two rounds (partition, UPDATE, the pull kernels unless the mode
// is PUSH, finalize), the first reading U from ubuf[0] and writing U' to
// ubuf[1], the second the other way round, so every kernel argument is
// fixed (the partition reads |U| from the control block).  Used when the
// context keeps no per-round timers.
struct AdgRoundArgs {
  AdgCtl* ctl;
  const long long* rp;
  const int* col;
  int* D;
  int* batch;
  int* ubuf[2];
  long long* task_start;
  int* task_len;
  int* task_v;
  uint2* live;
  int* hub_base;
  int* hub_vertex;
  long long mode, hubs, upd_blocks, pull_blocks, max_blocks, hub_smem;  // the key: all of the above
};

cudaError_t adg_round_graph(gc_context* ctx, const AdgRoundArgs& r, cudaGraphExec_t* exec) {
  return loop_graph(&ctx->adg_graph, &r, sizeof(r), [&](cudaStream_t cs, cudaGraphConditionalHandle loop) {
    for (int half = 0; half < 2; ++half) {
      int* u_in = r.ubuf[half];
      int* u_out = r.ubuf[half ^ 1];
      adg_partition_kernel<<<static_cast<int>(r.max_blocks), kAdgThreads, 0, cs>>>(
          r.ctl, r.rp, r.D, r.batch, u_in, u_out, r.task_start, r.task_len, r.live, 0, nullptr, nullptr,
          r.hub_base, r.hub_vertex);
      if (r.mode != GC_UPDATE_PULL) {
        if (r.hubs > 0)
          adg_update_kernel<true><<<static_cast<int>(r.upd_blocks), kAdgThreads, static_cast<size_t>(r.hub_smem),
                                    cs>>>(r.ctl, r.rp, r.col, r.D, r.batch, r.live, r.task_start, r.task_len, 0,
                                          r.hub_base, r.hub_vertex, 0);
        else
          adg_update_kernel<false><<<static_cast<int>(r.upd_blocks), kAdgThreads, 0, cs>>>(
              r.ctl, r.rp, r.col, r.D, r.batch, r.live, r.task_start, r.task_len, 0, nullptr, nullptr, 0);
      }
      if (r.mode != GC_UPDATE_PUSH) {
        adg_pull_tasks_kernel<<<static_cast<int>(r.max_blocks), kAdgThreads, 0, cs>>>(
            r.ctl, r.rp, r.D, u_out, r.task_start, r.task_len, r.task_v);
        adg_pull_count_kernel<<<static_cast<int>(r.pull_blocks), kAdgThreads, 0, cs>>>(
            r.ctl, r.col, r.D, r.live, r.task_start, r.task_len, r.task_v);
      }
      adg_finalize_graph_kernel<<<1, 1, 0, cs>>>(r.ctl, loop);
    }
  }, exec);
}

}  // namespace

// Excludes D (n ints), which the caller provides.
size_t adg_scratch_bytes(long long n, long long nnz) {
  const long long ntask = n + nnz / kChunk + 1;
  return 2 * (static_cast<size_t>(n) * 4 + 256) + static_cast<size_t>(ntask) * 16 + 3 * 256 +
         static_cast<size_t>((n + 31) / 32) * 8 + 256 + 64 * 8 + 256 + static_cast<size_t>((n + 31) / 32) * 4 +
         256 + kMaxHubs * 4 + 256 + 2048;
}

gc_status adg_run(gc_context* ctx, Arena a, const gc_csr* g, unsigned p, unsigned q, int* batch,
                  int* D, int* rounds_out, cudaStream_t s, const ColChunks* chunks) {
  const long long n = g->n, nnz = g->nnz;
  *rounds_out = 0;
  ctx->stats.adg_rounds = 0;
  ctx->adg_max_removal_degree = -1;
  if (n == 0) return GC_OK;
  AdgCtl* ctl = a.take<AdgCtl>(1);
  int* ubuf[2] = {a.take<int>(n), a.take<int>(n)};
  const long long ntask = n + nnz / kChunk + 1;
  long long* task_start = a.take<long long>(ntask);
  int* task_len = a.take<int>(ntask);
  int* task_v = a.take<int>(ntask);
  uint2* live = a.take<uint2>((n + 31) / 32);
  unsigned long long* hub_hist = a.take<unsigned long long>(64);
  int* hub_base = a.take<int>((n + 31) / 32);
  int* hub_vertex = a.take<int>(kMaxHubs);
  if (!ctl || !D || !ubuf[0] || !ubuf[1] || !task_start || !task_len || !task_v || !live || !hub_hist ||
      !hub_base || !hub_vertex)
    return GC_ERR_OOM;

  const int mode = ctx->opt.update_mode;
  GC_TRY_CUDA(cudaMemsetAsync(batch, 0, sizeof(int) * n, s));  // batch 0 = still in U
  adg_init_kernel<<<1, 1, 0, s>>>(ctl, n, nnz, p, q, mode, ctx->opt.pull_percent);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  // hubs: at most update_hubs vertices, one shared counter each
  const int hubs = ctx->opt.update_hubs > 0 && nnz > 0 ? min(ctx->opt.update_hubs, kMaxHubs) : 0;
  if (hubs > 0) {
    GC_TRY_CUDA(cudaMemsetAsync(hub_hist, 0, 64 * sizeof(unsigned long long), s));
    adg_hub_hist_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(row_ptr_of(g), n, hub_hist);
    adg_hub_pick_kernel<<<1, 1, 0, s>>>(hub_hist, ctx->opt.update_hubs, ctl);
    g_launches += 2;
    GC_TRY_CUDA(cudaGetLastError());
  }
  const size_t hub_smem = static_cast<size_t>(hubs) * sizeof(int);
  const int max_blocks = ctx->num_sms * 8;
  int per_sm = 0;
  const cudaError_t oe =
      hubs > 0
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adg_update_kernel<true>, kAdgThreads, hub_smem)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adg_update_kernel<false>, kAdgThreads, 0);
  if (oe != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int upd_blocks = ctx->num_sms * per_sm;
  const int pull_blocks = resident_grid(adg_pull_count_kernel, kAdgThreads, ctx->num_sms);
  long long size_u = n;
  int cur = 0;
  int* pinned = static_cast<int*>(ctx->pinned);
  int round = 0;
  while (size_u > 0) {
    ++round;
    if (round == 2 && cur == 1 && !ctx->timing && ctx->opt.round_graph) {
      // rounds 2.. as one graph launch (no host round trip per round)
      const AdgRoundArgs ra{ctl,        row_ptr_of(g), g->col_idx, D,        batch,    {ubuf[0], ubuf[1]},
                            task_start, task_len,      task_v,     live,     hub_base, hub_vertex,
                            mode,       hubs,          upd_blocks, pull_blocks, max_blocks,
                            static_cast<long long>(hub_smem)};
      cudaGraphExec_t ex = nullptr;
      if (adg_round_graph(ctx, ra, &ex) == cudaSuccess) {
        GC_TRY_CUDA(cudaGraphLaunch(ex, s));
        GC_TRY_CUDA(cudaMemcpyAsync(pinned, ctl, sizeof(AdgCtl), cudaMemcpyDeviceToHost, s));
        GC_TRY_CUDA(cudaStreamSynchronize(s));
        AdgCtl hc;
        memcpy(&hc, pinned, sizeof(hc));
        if (hc.graph_err) return GC_ERR_CUDA;  // a round removed no vertex: cannot happen
        const int last = hc.round - 1;         // each round that ran advanced the round number
        const unsigned long long per_round = 2ull + (mode != GC_UPDATE_PULL) + 2ull * (mode != GC_UPDATE_PUSH);
        g_launches += 2ull * per_round * static_cast<unsigned long long>(last / 2);
        round = last;
        break;
      }
    }
    long long want = (size_u + kAdgThreads - 1) / kAdgThreads;
    int blocks = static_cast<int>(want < max_blocks ? want : max_blocks);
    adg_partition_kernel<<<blocks, kAdgThreads, 0, s>>>(
        ctl, row_ptr_of(g), D, batch, round == 1 ? nullptr : ubuf[cur ^ 1], ubuf[cur], task_start,
        task_len, live, round == 1 ? static_cast<int>(n) : 0, nullptr, nullptr, hub_base, hub_vertex);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    ctx->timer_begin(gc_context::kTUpdate, s);
    // round 1 sweeps vertex ranges, each once its column indices are on the
    // device (one range: the whole graph, already there); later rounds sweep
    // the partition's task list
    const bool chunked = round == 1 && chunks != nullptr && chunks->k > 0;
    if (chunked && mode == GC_UPDATE_PULL)  // nothing of round 1 reads col_idx before the pull count
      for (int c = 0; c < chunks->k; ++c) GC_TRY_CUDA(cudaStreamWaitEvent(s, chunks->ready[c], 0));
    if (mode != GC_UPDATE_PULL) {  // each direction's kernels return at once if not chosen
      const int nr = chunked ? chunks->k : 1;
      for (int c = 0; c < nr; ++c) {
        const long long lo = chunked ? chunks->lo[c] : 0;
        const long long hi = chunked ? chunks->lo[c + 1] : (round == 1 ? n : 0);
        if (chunked) GC_TRY_CUDA(cudaStreamWaitEvent(s, chunks->ready[c], 0));
        if (round == 1 && hi <= lo) continue;
        if (hubs > 0)
          adg_update_kernel<true><<<upd_blocks, kAdgThreads, hub_smem, s>>>(
              ctl, row_ptr_of(g), g->col_idx, D, batch, live, task_start, task_len, hi, hub_base, hub_vertex, lo);
        else
          adg_update_kernel<false><<<upd_blocks, kAdgThreads, 0, s>>>(
              ctl, row_ptr_of(g), g->col_idx, D, batch, live, task_start, task_len, hi, nullptr, nullptr, lo);
        ++g_launches;
      }
    }
    if (mode != GC_UPDATE_PUSH) {
      const long long wantp = (size_u + kAdgThreads - 1) / kAdgThreads;
      adg_pull_tasks_kernel<<<static_cast<int>(wantp < max_blocks ? wantp : max_blocks), kAdgThreads, 0, s>>>(
          ctl, row_ptr_of(g), D, ubuf[cur], task_start, task_len, task_v);
      adg_pull_count_kernel<<<pull_blocks, kAdgThreads, 0, s>>>(ctl, g->col_idx, D, live, task_start, task_len,
                                                                 task_v);
      g_launches += 2;
    }
    ctx->timer_end(s);
    GC_TRY_CUDA(cudaGetLastError());
    adg_finalize_kernel<<<1, 1, 0, s>>>(ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    GC_TRY_CUDA(cudaMemcpyAsync(pinned, &ctl->size_U, sizeof(int), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    long long next = *pinned;
    if (next >= size_u) return GC_ERR_CUDA;  // cannot happen: every round removes a vertex
    size_u = next;
    cur ^= 1;
  }
  // statistics
  GC_TRY_CUDA(cudaMemcpyAsync(pinned, ctl, sizeof(AdgCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  AdgCtl h;
  memcpy(&h, pinned, sizeof(h));
  ctx->stats.sum_U = static_cast<int64_t>(h.total_U);
  ctx->stats.sum_decrements = static_cast<int64_t>(h.total_dec);
  ctx->stats.adg_pull_rounds = h.pull_rounds;
  ctx->adg_max_removal_degree = h.max_removal_degree;
  ctx->stats.adg_rounds = round;
  *rounds_out = round;
  return GC_OK;
}

// ---------------------------------------------------------------------------
// ADG-M (Section 5, "Degree Median Instead of Degree Average"): each round
// removes the ceil(|U|/2) vertices of U with the smallest degree in U (the
// median degree is the threshold, and R is limited to half of U, one more if
// |U| is odd), vertices of equal degree in increasing id order.  Each round
// writes the keys D[u] * 2^32 + u of U (unique), selects the k-th smallest,
// k = ceil(|U|/2), by MSD radix selection (per 8-bit digit from the top: a
// histogram of the keys that match the digits chosen so far, then one block
// picks the digit holding the k-th key), and partitions U on it; UPDATE, the
// cut and the bookkeeping are ADG's.  floor(log2 n) + 1 rounds.
// ---------------------------------------------------------------------------
namespace {

struct SelState {
  unsigned long long prefix;  // digits chosen so far
  unsigned long long mask;    // their bit positions
  long long k;                // rank (1-based) still sought among the matching keys
  long long pad;
};

__global__ void adg_m_init_kernel(const long long* __restrict__ row_ptr, long long n, int* __restrict__ D,
                                  int* __restrict__ U, uint2* __restrict__ live) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  const long long t0 = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (long long v = t0; v < n; v += stride) {
    D[v] = static_cast<int>(row_ptr[v + 1] - row_ptr[v]);
    U[v] = static_cast<int>(v);
  }
  for (long long w = t0; w < (n + 31) / 32; w += stride) {
    const long long left = n - 32 * w;
    live[w] = make_uint2(left >= 32 ? ~0u : ((1u << left) - 1u), 0u);  // no hubs in ADG-M
  }
}

// keys of this round's U, and the selection state (k = ceil(|U|/2))
__global__ void adg_m_keys_kernel(const int* __restrict__ U, const AdgCtl* __restrict__ ctl,
                                  const int* __restrict__ D, unsigned long long* __restrict__ keys,
                                  SelState* __restrict__ st, unsigned* __restrict__ hist) {
  const long long size_u = ctl->size_U;
  const long long t0 = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  for (long long i = t0; i < size_u; i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int u = U[i];
    keys[i] = (static_cast<unsigned long long>(static_cast<unsigned>(D[u])) << 32) | static_cast<unsigned>(u);
  }
  if (t0 == 0) *st = SelState{0ull, 0ull, (size_u + 1) / 2, 0};
  if (t0 < 256) hist[t0] = 0u;
}

__global__ void __launch_bounds__(256)
adg_m_hist_kernel(const unsigned long long* __restrict__ keys, const AdgCtl* __restrict__ ctl,
                  const SelState* __restrict__ st, int shift, unsigned* __restrict__ hist) {
  __shared__ unsigned sh[256];
  sh[threadIdx.x] = 0u;
  __syncthreads();
  const long long size_u = ctl->size_U;
  const unsigned long long prefix = st->prefix, mask = st->mask;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < size_u;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned long long key = keys[i];
    if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// one block of 256 threads: the digit value whose bin holds the k-th key
__global__ void __launch_bounds__(256) adg_m_pick_kernel(SelState* __restrict__ st, int shift,
                                                         unsigned* __restrict__ hist) {
  __shared__ long long cum[256];
  const int t = threadIdx.x;
  cum[t] = hist[t];
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {  // inclusive scan
    const long long add = t >= o ? cum[t - o] : 0;
    __syncthreads();
    cum[t] += add;
    __syncthreads();
  }
  const long long k = st->k;
  const long long before = t > 0 ? cum[t - 1] : 0;
  __syncthreads();
  if (before < k && k <= cum[t]) {
    st->prefix |= static_cast<unsigned long long>(t) << shift;
    st->mask |= 255ull << shift;
    st->k = k - before;
  }
  hist[t] = 0u;
}

}  // namespace

size_t adg_m_scratch_bytes(long long n, long long nnz) {
  return adg_scratch_bytes(n, nnz) + static_cast<size_t>(n) * 8 + 256 + sizeof(SelState) + 256 + 256 * 4 + 256;
}

gc_status adg_m_run(gc_context* ctx, Arena a, const gc_csr* g, int* batch, int* D, int* rounds_out,
                    cudaStream_t s) {
  const long long n = g->n, nnz = g->nnz;
  *rounds_out = 0;
  ctx->stats.adg_rounds = 0;
  ctx->adg_max_removal_degree = -1;
  if (n == 0) return GC_OK;
  AdgCtl* ctl = a.take<AdgCtl>(1);
  int* ubuf[2] = {a.take<int>(n), a.take<int>(n)};
  const long long ntask = n + nnz / kChunk + 1;
  long long* task_start = a.take<long long>(ntask);
  int* task_len = a.take<int>(ntask);
  a.take<int>(ntask);  // (ADG's pull task list; ADG-M only pushes)
  uint2* live = a.take<uint2>((n + 31) / 32);
  a.take<unsigned long long>(64);
  unsigned long long* keys = a.take<unsigned long long>(n);
  SelState* st = a.take<SelState>(1);
  unsigned* hist = a.take<unsigned>(256);
  if (!ctl || !D || !ubuf[0] || !ubuf[1] || !task_start || !task_len || !live || !keys || !st || !hist)
    return GC_ERR_OOM;

  // digits of the keys that can be non-zero: u < n and D[u] <= n - 1
  int nbits = 1;
  while (nbits < 62 && (1ll << nbits) < n) ++nbits;
  const int ndig = (nbits + 7) / 8;
  int shifts[8], nshift = 0;
  for (int d = ndig - 1; d >= 0; --d) shifts[nshift++] = 32 + 8 * d;  // D, from the top
  for (int d = ndig - 1; d >= 0; --d) shifts[nshift++] = 8 * d;       // then u

  const long long* rp = row_ptr_of(g);
  const int max_blocks = ctx->num_sms * 8;
  const int upd_blocks = resident_grid(adg_update_kernel<false>, kAdgThreads, ctx->num_sms);
  GC_TRY_CUDA(cudaMemsetAsync(batch, 0, sizeof(int) * n, s));
  adg_init_kernel<<<1, 1, 0, s>>>(ctl, n, nnz, 0, 1, GC_UPDATE_PUSH, 0);  // (its threshold is not used here)
  ++g_launches;
  adg_m_init_kernel<<<max_blocks, kAdgThreads, 0, s>>>(rp, n, D, ubuf[0], live);
  ++g_launches;
  GC_TRY_CUDA(cudaGetLastError());
  long long size_u = n;
  int cur = 0, round = 0;
  int* pinned = static_cast<int*>(ctx->pinned);
  while (size_u > 0) {
    ++round;
    const long long want = (size_u + kAdgThreads - 1) / kAdgThreads;
    const int blocks = static_cast<int>(want < max_blocks ? want : max_blocks);
    adg_m_keys_kernel<<<blocks, kAdgThreads, 0, s>>>(ubuf[cur], ctl, D, keys, st, hist);
    ++g_launches;
    for (int j = 0; j < nshift; ++j) {
      adg_m_hist_kernel<<<blocks, 256, 0, s>>>(keys, ctl, st, shifts[j], hist);
      adg_m_pick_kernel<<<1, 256, 0, s>>>(st, shifts[j], hist);
      g_launches += 2;
    }
    GC_TRY_CUDA(cudaGetLastError());
    adg_partition_kernel<<<blocks, kAdgThreads, 0, s>>>(ctl, rp, D, batch, ubuf[cur], ubuf[cur ^ 1], task_start,
                                                        task_len, live, 0, keys, &st->prefix);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    ctx->timer_begin(gc_context::kTUpdate, s);
    adg_update_kernel<false><<<upd_blocks, kAdgThreads, 0, s>>>(ctl, rp, g->col_idx, D, batch, live, task_start,
                                                                 task_len, 0, nullptr, nullptr);
    ++g_launches;
    ctx->timer_end(s);
    GC_TRY_CUDA(cudaGetLastError());
    adg_finalize_kernel<<<1, 1, 0, s>>>(ctl);
    ++g_launches;
    GC_TRY_CUDA(cudaGetLastError());
    size_u /= 2;  // each round removes ceil(|U|/2): no read-back needed
    cur ^= 1;
  }
  // one read-back at the end: the totals, and |U| = 0 as a check
  GC_TRY_CUDA(cudaMemcpyAsync(pinned, ctl, sizeof(AdgCtl), cudaMemcpyDeviceToHost, s));
  GC_TRY_CUDA(cudaStreamSynchronize(s));
  AdgCtl h;
  memcpy(&h, pinned, sizeof(h));
  if (h.size_U != 0) return GC_ERR_CUDA;  // cannot happen
  ctx->stats.sum_U = static_cast<int64_t>(h.total_U);
  ctx->stats.sum_decrements = static_cast<int64_t>(h.total_dec);
  ctx->stats.adg_pull_rounds = 0;
  ctx->adg_max_removal_degree = h.max_removal_degree;
  ctx->stats.adg_rounds = round;
  *rounds_out = round;
  return GC_OK;
}

}  // namespace gc

// ---------------------------------------------------------------------------
// gc_adg_partition_noalloc: the same ADG rounds on a fixed scratch area that
// is compiled into the library, for callers that cannot allocate device
// memory when they call in.  It has no context: it runs on the calling
// thread's current device and launches the kernels above in the same order
// as adg_run.
// ---------------------------------------------------------------------------
namespace {

constexpr long long kNoAllocMaxN = 1ll << 18;     // vertices
constexpr long long kNoAllocMaxNnz = 1ll << 23;   // directed CSR entries
constexpr long long kNoAllocTasks = kNoAllocMaxN + kNoAllocMaxNnz / gc::kChunk + 1;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// layout: control block | D | U list 0 | U list 1 | task starts | task lengths
//         | liveness bitmap
constexpr size_t kNaOffD = align256(sizeof(gc::AdgCtl));
constexpr size_t kNaOffU0 = kNaOffD + align256(kNoAllocMaxN * sizeof(int));
constexpr size_t kNaOffU1 = kNaOffU0 + align256(kNoAllocMaxN * sizeof(int));
constexpr size_t kNaOffTs = kNaOffU1 + align256(kNoAllocMaxN * sizeof(int));
constexpr size_t kNaOffTl = kNaOffTs + align256(kNoAllocTasks * sizeof(long long));
constexpr size_t kNaOffLive = kNaOffTl + align256(kNoAllocTasks * sizeof(int));
constexpr size_t kNoAllocBytes = kNaOffLive + align256(kNoAllocMaxN / 32 * sizeof(uint2));  // about 6.5 MB

constexpr int kNoAllocDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_scratch[kNoAllocDevices];  // device address of the array, per device
int g_noalloc_sms[kNoAllocDevices];

}  // namespace

// One copy per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_adg_noalloc_scratch[kNoAllocBytes];

extern "C" gc_status gc_adg_partition_noalloc(const gc_csr* g, uint32_t eps_p, uint32_t eps_q,
                                              int32_t* batch_out, int32_t* num_rounds_out,
                                              gc_stream stream) {
  using namespace gc;
  if (!g || !num_rounds_out) return GC_ERR_INVALID_ARG;
  if (g->n < 0 || g->nnz < 0 || (g->n > 0 && !g->row_ptr) || (g->nnz > 0 && !g->col_idx))
    return GC_ERR_INVALID_ARG;
  if (eps_q == 0 || eps_q > (1u << 20) || eps_p > (1u << 20)) return GC_ERR_INVALID_ARG;
  if (g->n > kNoAllocMaxN || g->nnz > kNoAllocMaxNnz) return GC_ERR_OVERFLOW;
  if (g->n > 0 && !batch_out) return GC_ERR_INVALID_ARG;
  *num_rounds_out = 0;
  const long long n = g->n, nnz = g->nnz;
  if (n == 0) return GC_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // Set-up, once per device with that device current: the array's device
  // address (its host-side name is not a device address).
  int dev = -1;
  GC_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocDevices) return GC_ERR_CUDA;
  char* base = nullptr;
  int num_sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_scratch[dev]) {
      void* p = nullptr;
      GC_TRY_CUDA(cudaGetSymbolAddress(&p, g_adg_noalloc_scratch));
      int sms = 0;
      GC_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      g_noalloc_sms[dev] = sms;
      g_noalloc_scratch[dev] = p;
    }
    base = static_cast<char*>(g_noalloc_scratch[dev]);
    num_sms = g_noalloc_sms[dev];
  }
  AdgCtl* ctl = reinterpret_cast<AdgCtl*>(base);
  int* D = reinterpret_cast<int*>(base + kNaOffD);
  int* ubuf[2] = {reinterpret_cast<int*>(base + kNaOffU0), reinterpret_cast<int*>(base + kNaOffU1)};
  long long* task_start = reinterpret_cast<long long*>(base + kNaOffTs);
  int* task_len = reinterpret_cast<int*>(base + kNaOffTl);
  uint2* live = reinterpret_cast<uint2*>(base + kNaOffLive);

  // Every buffer above is written before it is read within a call; the
  // control block, the only state carried between kernels, is reset here.
  GC_TRY_CUDA(cudaMemsetAsync(batch_out, 0, sizeof(int) * n, s));
  adg_init_kernel<<<1, 1, 0, s>>>(ctl, n, nnz, eps_p, eps_q, GC_UPDATE_PUSH, 0);
  GC_TRY_CUDA(cudaGetLastError());
  const int max_blocks = num_sms * 8;
  const int upd_blocks = gc::resident_grid(gc::adg_update_kernel<false>, gc::kAdgThreads, num_sms);
  const long long* rp = reinterpret_cast<const long long*>(g->row_ptr);
  long long size_u = n;
  int cur = 0, round = 0;
  while (size_u > 0) {
    ++round;
    const long long want = (size_u + kAdgThreads - 1) / kAdgThreads;
    const int blocks = static_cast<int>(want < max_blocks ? want : max_blocks);
    adg_partition_kernel<<<blocks, kAdgThreads, 0, s>>>(ctl, rp, D, batch_out,
                                                        round == 1 ? nullptr : ubuf[cur ^ 1], ubuf[cur],
                                                        task_start, task_len, live,
                                                        round == 1 ? static_cast<int>(n) : 0);
    GC_TRY_CUDA(cudaGetLastError());
    adg_update_kernel<false><<<upd_blocks, kAdgThreads, 0, s>>>(ctl, rp, g->col_idx, D, batch_out, live,
                                                                 task_start, task_len, round == 1 ? n : 0, nullptr,
                                                                 nullptr);
    GC_TRY_CUDA(cudaGetLastError());
    adg_finalize_kernel<<<1, 1, 0, s>>>(ctl);
    GC_TRY_CUDA(cudaGetLastError());
    int next = 0;  // |U| of the next round, read into ordinary host memory
    GC_TRY_CUDA(cudaMemcpyAsync(&next, &ctl->size_U, sizeof(int), cudaMemcpyDeviceToHost, s));
    GC_TRY_CUDA(cudaStreamSynchronize(s));
    if (next >= size_u) return GC_ERR_CUDA;  // cannot happen: every round removes a vertex
    size_u = next;
    cur ^= 1;
  }
  *num_rounds_out = round;
  return GC_OK;
}
