/*
 * gcolor.h -- C ABI of the GB300 (sm_103a) graph-colouring library.
 *
 * The library computes the two data-parallel steps of JP-ADG from Besta et
 * al., "High-Performance Parallel Graph Coloring with Strong Guarantees on
 * Work, Depth, and Quality" (SC'20):
 *
 *   ADG     (Algorithm 1, Section 3): the approximate degeneracy ordering.
 *           Round after round it removes every remaining vertex whose degree
 *           in the remaining subgraph is at most (1+eps) times that
 *           subgraph's average degree; the round number is the vertex's batch.
 *   JP-ADG  (Algorithm 3, Section 4.1): Jones-Plassmann colouring with the
 *           priority rho(v) = <rho_ADG(v), rho_R(v)>, where rho_R is a seeded
 *           random tie-break.
 *
 * Graph model (Section 2.1): an undirected simple graph in CSR.  Both
 * directions of every edge are stored, rows are sorted ascending, there are
 * no self-loops and no duplicate edges.  Vertex ids are 0..n-1.
 *
 * Conventions for every call below:
 *  - Pointers documented "device" must be device memory of the context's GPU
 *    (cudaMalloc, or a PyTorch CUDA tensor's data pointer); "host" pointers
 *    are ordinary or page-locked host memory.  The CALLER owns every input
 *    and output buffer.  The context owns only its scratch memory, which it
 *    grows on demand and frees in gc_destroy().
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    stream-ordered.  Calls that return host scalars (num_rounds, num_colors)
 *    synchronise the stream before returning, so those scalars and the device
 *    outputs are ready when the call returns.
 *  - Exact integer arithmetic throughout: eps = eps_p / eps_q with
 *    eps_q >= 1, eps_p >= 0 and eps_p, eps_q <= 2^20 (GC_ERR_INVALID_ARG
 *    otherwise).  The ADG test "D[u] <= (1+eps) * Sigma/|U|" is evaluated as
 *    D[u] <= floor((q+p)*Sigma / (q*|U|)) without floating point.
 *  - Output numbering: batch ids start at 1 (Algorithm 1 starts its round
 *    counter at 1); colours start at 1 (Algorithm 3: 0 means uncoloured).
 *  - Results are deterministic: for a fixed seed the batches are unique and
 *    the colouring equals the sequential Greedy colouring in decreasing
 *    priority order (with vertex id as the final tie-break), whatever the
 *    thread schedule.
 *  - No call aborts, traps or hangs: every device-side wait is bounded and a
 *    wait that runs out is reported as GC_ERR_TIMEOUT.  After any error the
 *    context stays usable; device outputs are then unspecified.
 *  - A context may be used by one host thread at a time.
 */
#ifndef GCOLOR_H_
#define GCOLOR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GC_OK = 0,
  GC_ERR_INVALID_ARG = 1,   /* null pointer, bad size, eps out of range      */
  GC_ERR_INVALID_GRAPH = 2, /* CSR breaks the graph model (gc_validate_csr)  */
  GC_ERR_OOM = 3,           /* device or pinned-host allocation failed       */
  GC_ERR_CUDA = 4,          /* a CUDA runtime call failed                    */
  GC_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out            */
  GC_ERR_OVERFLOW = 6       /* a count would not fit the documented range    */
} gc_status;

/* Same type as cudaStream_t, spelled without the CUDA headers. */
typedef struct CUstream_st *gc_stream;

typedef struct gc_context gc_context;

/* A CSR graph resident on the device: row_ptr has n+1 int64 entries with
 * row_ptr[0] = 0 and row_ptr[n] = nnz; col_idx has nnz int32 entries.
 * n <= 2^31 - 2; nnz = 2m (both directions of each undirected edge). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t *row_ptr; /* device */
  const int32_t *col_idx; /* device */
} gc_csr;

/* Per-call statistics of the last completed call on a context. */
typedef struct {
  int32_t adg_rounds;      /* rho-bar: number of ADG rounds                    */
  int32_t num_colors;      /* largest colour used                              */
  int64_t sum_U;           /* sum over rounds of |U_l| (partition work)        */
  int64_t sum_decrements;  /* degree decrements performed by ADG's UPDATE      */
  int64_t jp_spins;        /* polls of uncoloured predecessors (diagnostic)    */
  float ms_adg;            /* device time of the ADG phase (0 if not timed)    */
  float ms_jp;             /* device time of the JP phase (0 if not timed)     */
  float ms_jp_color;       /* JP's bulk colouring launches, summed             */
  int32_t launches;        /* kernels this library launched in the last call   */
  float ms_adg_update;     /* ADG's UPDATE launches (one per round), summed     */
  float ms_core_solve;     /* the JP-ADG core cluster                          */
  float ms_core_preds;     /* extraction of the core's predecessor lists       */
  int32_t bulk_launches;   /* JP bulk launches (one per ADG batch outside core) */
  int64_t core_vertices;   /* vertices coloured by the core cluster            */
  int64_t core_preds;      /* predecessor entries of the core                  */
  int64_t core_degree_sum; /* degree sum of the core vertices                  */
  int32_t core_ctas;       /* CTAs (one cluster) that coloured the core        */
  int64_t sim_iterations;  /* DEC-ADG-ITR: SIM-COL iterations, summed over the
                              partitions (0 for the JP calls)                  */
  int64_t dec_internal_edges; /* DEC-ADG-ITR: CSR entries inside a partition
                              of vertices with such an entry (edges of G(l))   */
  float ms_dec_extract;    /* DEC-ADG-ITR: per-partition extraction launches   */
  float ms_dec_iterate;    /* DEC-ADG-ITR: the later SIM-COL iterations        */
  int64_t dec_tail_partitions; /* DEC-ADG-ITR: partitions finished by the
                              single-cluster tail (gc_options.dec_tail)      */
  int32_t adg_pull_rounds; /* ADG rounds whose UPDATE pulled (update_mode)     */
  int32_t jp_state_bits;   /* JP-ADG state word of the last call: 16 or 32     */
  int32_t batch_path;      /* gc_color_batch: GC_BATCH_SEGMENTED or _PERSISTENT */
} gc_stats;

/* Human-readable name of a status code (static storage). */
const char *gc_status_str(gc_status s);

/* Where the last CUDA call that failed inside this library on the calling
 * host thread was made, and the CUDA error ("file:line: name (message)");
 * "" if none has failed.  Thread-local storage, valid until the thread's
 * next library call. */
const char *gc_last_error(void);

/* ADG's UPDATE direction (gc_options.update_mode).  Push (Algorithm 1's
 * UPDATE): every vertex removed this round decrements the degree of each
 * neighbour still in U.  Pull (Section 5, "Push vs. Pull", the CREW variant
 * of Algorithm 2): every vertex still in U subtracts the number of its
 * neighbours removed this round, with no contended atomics.  AUTO chooses per
 * round from the edges each direction must sweep (see pull_percent).  The
 * results are identical in every mode. */
enum { GC_UPDATE_AUTO = 0, GC_UPDATE_PUSH = 1, GC_UPDATE_PULL = 2 };

/* Tunables of a context.  Fill one with gc_options_init(), change fields,
 * and pass it to gc_create() (NULL there means every default).  Each field
 * changes speed only: every call gives identical results for every valid
 * setting.  struct_size versions the struct: a caller built against an
 * older, shorter gc_options sets its own size and the library takes defaults
 * for the fields it does not have. */
typedef struct {
  uint32_t struct_size;    /* sizeof(gc_options) as the caller knows it      */
  int32_t core_target;     /* JP core size in vertices, 0..32768; 0: no core
                              (default 16384)                                */
  int32_t core_cluster;    /* at most this many CTAs in the core's thread-block
                              cluster, 1..16 (default 16; fewer if the device
                              cannot place them)                             */
  int32_t core_warps;      /* warps per core CTA, 1..32 (default 12)          */
  int32_t dec_tail;        /* DEC-ADG-ITR: 1 finishes a partition's last
                              SIM-COL iterations in one cluster launch
                              (default), 0 runs every iteration GPU-wide     */
  int32_t update_mode;     /* GC_UPDATE_AUTO (default), _PUSH or _PULL       */
  int32_t pull_percent;    /* AUTO pulls a round when the rows of U' hold at
                              most pull_percent % of the entries the rows of
                              R hold, 0..100000 (default 25)                 */
  int32_t bulk_blocks_per_sm; /* resident blocks per SM of JP's bulk colouring
                              kernel, 0 = as many as fit (default), 1..32    */
  uint32_t wait_limit_ms;  /* bound of every device-side wait, 1..600000 ms
                              (default 4000); a wait that runs out ends the
                              call with GC_ERR_TIMEOUT, context usable       */
  int32_t jp_state16;      /* 1: JP-ADG keeps each vertex's batch and colour in
                              a 16-bit word when both fit (the colour bound
                              is 1 + the largest degree at removal); 0
                              (default): always a 32-bit word                */
  int32_t batch_mode;      /* gc_color_batch: GC_BATCH_AUTO (default),
                              GC_BATCH_SEGMENTED or GC_BATCH_PERSISTENT      */
  int32_t update_hubs;     /* ADG's push UPDATE counts the decrements aimed at
                              up to this many highest-degree vertices (degree
                              >= a power of two >= 256) in a shared-memory
                              array per thread block, added to their degree
                              words once per block, 0..4096 (default 512; 0:
                              every decrement is an atomic on its word)      */
  int32_t host_upload;     /* gc_color_graph_host: 1 (default) has the SMs
                              read page-locked, mapped host buffers directly
                              (16-byte aligned; others use the copy engine);
                              0 copies the graph with the copy engine.
                              From 2^22 entries on, col_idx is copied in 8
                              vertex ranges on a stream of the context and
                              ADG's first round sweeps each range once it
                              has arrived                                    */
  int32_t round_graph;     /* 1 (default) runs ADG's rounds from round 2 on
                              as one CUDA graph launch (a device-side loop,
                              no host round trip per round) in the segmented
                              batch path and, while the context keeps no
                              timers (gc_set_timing), in the calls that run
                              ADG (gc_color_graph, _host, gc_adg_partition,
                              gc_color_graph_dec_itr, gc_color_graph_o);
                              built on the second call in a row with the
                              same buffers and shapes, kept by the context
                              while they stay the same; 0 launches each
                              round from the host                            */
} gc_options;

/* How gc_color_batch runs (gc_options.batch_mode, gc_stats.batch_path):
 * SEGMENTED runs ADG's rounds for all graphs together, one set of GPU-wide
 * launches per round, then one JP over the union; PERSISTENT is one launch
 * in which each thread block takes whole graphs from a queue (largest first)
 * and runs ADG and JP on each graph alone.  AUTO takes PERSISTENT only
 * while every graph holds at most 1/1024 of the batch's CSR entries (and at
 * most 2^24): one block colours a graph at a small fraction of the GPU's
 * rate, so a large graph sets the persistent launch's time.  Results are
 * identical. */
enum { GC_BATCH_AUTO = 0, GC_BATCH_SEGMENTED = 1, GC_BATCH_PERSISTENT = 2 };

/* Fill *opt with the defaults (and struct_size = sizeof(gc_options)). */
gc_status gc_options_init(gc_options *opt);

/* Create a context bound to CUDA device `device` with options `opt` (NULL:
 * defaults; GC_ERR_INVALID_ARG if a field is out of range).  Allocates
 * nothing large until the first call needs scratch.  *ctx is NULL on
 * failure.
 *
 * The environment is read here only for failure injection, to test the
 * error paths:
 *   GC_INJECT_STALL   id of a vertex whose colour is never published, so
 *                     that the waits of its successors run out (inside or
 *                     outside the JP core);
 *   GC_INJECT_OOM     non-zero: every scratch allocation fails (GC_ERR_OOM). */
gc_status gc_create(gc_context **ctx, int device, const gc_options *opt);

/* The options the context runs with (defaults filled in). */
gc_status gc_get_options(const gc_context *ctx, gc_options *out);

/* Replace the context's options (range-checked as in gc_create; the context
 * is unchanged on GC_ERR_INVALID_ARG).  Scratch memory is kept. */
gc_status gc_set_options(gc_context *ctx, const gc_options *opt);

/* Autotuner (no counterpart in the paper, which tunes nothing): finds the
 * options under which gc_color_graph(g, eps, seed) runs fastest on this
 * device, by coordinate descent over the option fields -- UPDATE direction
 * and pull threshold, JP state word, JP core size, warps and cluster, bulk
 * blocks per SM -- each run timed with CUDA events on `stream` (median of
 * `reps` runs after one warm-up run).  Every candidate's colouring is
 * compared with the starting options' on the device; a difference is a
 * library defect and returns GC_ERR_CUDA.  The search stops early once the
 * timed runs add up to budget_ms (0: no limit).  On success the fastest
 * options are applied to the context and written to *best_out, with their
 * median time (ms) in *best_ms_out and the starting options' in
 * *start_ms_out (both may be NULL).  Allocates two n-int device buffers for
 * the comparison and frees them before returning. */
gc_status gc_autotune(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q, uint64_t seed,
                      int32_t reps, float budget_ms, gc_options *best_out, float *best_ms_out,
                      float *start_ms_out, gc_stream stream);


/* Release the context's scratch memory and the context itself (NULL ok). */
void gc_destroy(gc_context *ctx);

/* Statistics of the last successful colouring call on `ctx`. */
gc_status gc_get_stats(const gc_context *ctx, gc_stats *out);

/* When `enable` is non-zero, later calls time their ADG and JP phases and
 * their main kernel groups with CUDA events recorded on the call's stream
 * (reported in gc_stats); default off. */
gc_status gc_set_timing(gc_context *ctx, int enable);

/* Check that `g` satisfies the graph model of Section 2.1: row_ptr starts at
 * 0, is non-decreasing and ends at nnz; every id is in [0, n); rows are
 * strictly increasing (sorted, no duplicates); no self-loops; and the graph
 * is symmetric (w in N(u) <=> u in N(w)).  Returns GC_OK or
 * GC_ERR_INVALID_GRAPH.  O(nnz log Delta) work on the device.  The other
 * calls assume a valid graph and do not re-check it. */
gc_status gc_validate_csr(gc_context *ctx, const gc_csr *g, gc_stream stream);

/* ADG, Algorithm 1 (Section 3).  Writes batch_out[v] = rho_ADG(v) in
 * 1..num_rounds for every vertex (device, n int32) and the number of rounds
 * to *num_rounds_out (host).  Degrees are maintained by push-style UPDATE
 * (atomic decrements of the neighbours of each removed vertex) and the degree
 * sum is carried from round to round by subtracting the removed degrees and
 * the cut (Section 5, "Caching Sums of Degrees"). */
gc_status gc_adg_partition(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q,
                           int32_t *batch_out, int32_t *num_rounds_out, gc_stream stream);

/* gc_adg_partition without a context and without allocating anything.
 * The paper has no counterpart: this is an interface for callers that
 * cannot allocate device memory when they call in -- for example a process
 * that handed all of the GPU's memory to its own allocator at start-up (a
 * cudaMalloc would fail there), or code on a latency budget that cannot
 * afford cudaMalloc/cudaFree, which may block and synchronise the device.
 * Same inputs, outputs and results as gc_adg_partition; the caller still
 * provides batch_out (device, n int32).
 * Scratch is one fixed array of about 6.5 MB built into the library; every
 * GPU that loads the library holds its own copy until the process exits.  It
 * bounds the graph: n <= 262144 vertices and nnz <= 8388608 entries; larger
 * graphs return GC_ERR_OVERFLOW without touching the device.
 * Runs on the calling thread's current device (g and batch_out must live
 * there).  The first call on each device looks up the array's device
 * address; make that first call before any stream capture.  The address is
 * kept for the rest of the process: after cudaDeviceReset() on a device it is
 * stale, so do not call this entry point on that device again.  Each ADG
 * round ends by reading |U| back into host memory, which synchronises
 * `stream` once per round.  All calls share the one array and each call
 * starts by resetting the state it reads, so calls whose work could overlap
 * on the GPU (other streams, other threads) race with each other and must be
 * serialised by the caller. */
gc_status gc_adg_partition_noalloc(const gc_csr *g, uint32_t eps_p, uint32_t eps_q,
                                   int32_t *batch_out, int32_t *num_rounds_out, gc_stream stream);

/* JP-ADG priority (Section 4.1): key_out[v] = (batch[v] << 32) | h_seed(v)
 * (device, n uint64), where h_seed(v) is the upper 32 bits of the (v+1)-th
 * output of the SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014)
 * started from state `seed`.  batch is device, n int32, values >= 0. */
gc_status gc_make_priority(gc_context *ctx, int64_t n, const int32_t *batch, uint64_t seed,
                           uint64_t *key_out, gc_stream stream);

/* ADG-M (Section 5, "Degree Median Instead of Degree Average"): ADG with
 * the median degree of U as the threshold and R limited to half of U (one
 * more if |U| is odd), so each round removes the ceil(|U|/2) vertices of U
 * with the smallest degree in U; vertices of equal degree go in increasing
 * id order.  batch_out (device, n int32) receives rounds 1..*num_rounds_out
 * (= floor(log2 n) + 1 for n >= 1). */
gc_status gc_adg_m_partition(gc_context *ctx, const gc_csr *g, int32_t *batch_out, int32_t *num_rounds_out,
                             gc_stream stream);

/* JP-ADG-M: ADG-M, then JP with <rho_ADG-M, rho_R> (rho_R as in
 * gc_make_priority); at most 4d + 1 colours for degeneracy d.  Arguments as
 * in gc_color_graph (without eps). */
gc_status gc_color_graph_m(gc_context *ctx, const gc_csr *g, uint64_t seed, int32_t *color_out, int32_t *batch_out,
                           int32_t *num_colors_out, int32_t *num_rounds_out, gc_stream stream);

/* ADG-O (Algorithm 6; Section 5, "Explicit Ordering in R"): the iterations
 * of gc_adg_partition, each removed set R numbered in increasing order of its
 * vertices' degree D in G[U] at removal, equal degrees in increasing id (a
 * reading: the paper leaves ties open).  rho_out[v] (device, n int32) is
 * rho_ADG(v) = (vertices removed in earlier iterations) + (v's place in its
 * sorted R), a permutation of 0..n-1; batch_out (device, n int32, may be
 * NULL) the iteration as in gc_adg_partition; rank_out (device, n int32, may
 * be NULL) the number of neighbours with a higher rho (Algorithm 6's
 * UPDATEandPRIORITIZE); *num_rounds_out (host, may be NULL) the number of
 * iterations. */
gc_status gc_adg_o_order(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q, int32_t *batch_out,
                         int32_t *rho_out, int32_t *rank_out, int32_t *num_rounds_out, gc_stream stream);

/* JP-ADG-O: JP (Algorithm 3) with the total order rho_ADG-O as its priority
 * (a higher rho is coloured first); no random tie-break, so no seed.
 * Arguments as in gc_color_graph.  At most floor(2(1+eps)d) + 1 colours. */
gc_status gc_color_graph_o(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q, int32_t *color_out,
                           int32_t *batch_out, int32_t *num_colors_out, int32_t *num_rounds_out, gc_stream stream);

/* DEC-ADG-ITR colouring (Section 4.3) of given partitions
 * R(l) = {v : batch[v] = l}, l = 1..num_rounds (batch: device, n int32, any
 * partial order such as gc_adg_partition's or gc_adg_m_partition's):
 * Algorithm 4 colours R(num_rounds) first and R(1) last, each with SIM-COL
 * (Algorithm 5) in its ITR form, every vertex still in U drawing the
 * smallest colour not used by a coloured neighbour (its bitmap B_v).  Of two
 * adjacent vertices of U that drew the same colour in one iteration, the one
 * with the lower (h_seed(v), v) key gives it back (h_seed as in
 * gc_make_priority; the paper resets both, which never ends with
 * deterministic draws), so each SIM-COL call ends within |R(l)| iterations
 * and the result does not depend on the schedule.  color_out (device, n
 * int32) receives colours >= 1, each at most 1 + the number of neighbours in
 * the same or a higher partition; *num_colors_out (host, may be NULL) the
 * largest.  gc_stats.sim_iterations counts the SIM-COL iterations.
 * GC_ERR_INVALID_ARG if num_rounds < 1 (n > 0) or a batch lies outside
 * 1..num_rounds (then color_out is undefined).  Empty partitions cost no
 * launches (the non-empty ones are read back once).  Scratch: about
 * 4 nnz + 24 n + 132 num_rounds bytes. */
gc_status gc_dec_itr_color(gc_context *ctx, const gc_csr *g, const int32_t *batch, int32_t num_rounds,
                           uint64_t seed, int32_t *color_out, int32_t *num_colors_out, gc_stream stream);

/* DEC-ADG-ITR end to end: ADG with eps = eps_p/eps_q (as gc_adg_partition),
 * then gc_dec_itr_color on its partitions.  At most floor(2(1+eps)d) + 1
 * colours for degeneracy d.  Arguments as in gc_color_graph. */
gc_status gc_color_graph_dec_itr(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q, uint64_t seed,
                                 int32_t *color_out, int32_t *batch_out, int32_t *num_colors_out,
                                 int32_t *num_rounds_out, gc_stream stream);

/* Priorities of the other JP variants the paper compares (Section 4.1,
 * "combinations of JP and orderings"), as keys for gc_jp_color:
 *   GC_PRIO_R    JP-R:   rho_R                      key = h_seed(v)
 *   GC_PRIO_FF   JP-FF:  the natural vertex order   key = 2^32 - 1 - v
 *   GC_PRIO_LF   JP-LF:  <deg(v), rho_R>            key = deg(v) << 32 | h_seed(v)
 *   GC_PRIO_LLF  JP-LLF: <ceil(log2 deg(v)), rho_R> key = ceil(log2 deg(v)) << 32 | h_seed(v)
 *                        (0 for degree 0 and 1)
 *   GC_PRIO_SL   JP-SL:  smallest-last              key = the index at which v is
 *                        removed when the vertex of minimum (degree in the
 *                        remaining graph, id) is removed repeatedly
 *                        (Matula-Beck peeling; the paper leaves ties open);
 *                        the vertex removed last is coloured first; no seed.
 *                        Inherently sequential: one thread block removes a
 *                        vertex every few microseconds.  n <= 2^25, else
 *                        GC_ERR_OVERFLOW.
 * with h_seed as in gc_make_priority; equal keys fall back to the vertex id
 * in gc_jp_color.  key_out is device, n uint64.  GC_ERR_INVALID_ARG for an
 * unknown kind. */
enum { GC_PRIO_R = 0, GC_PRIO_FF = 1, GC_PRIO_LF = 2, GC_PRIO_LLF = 3, GC_PRIO_SL = 4 };
gc_status gc_make_priority_kind(gc_context *ctx, const gc_csr *g, int32_t kind, uint64_t seed,
                                uint64_t *key_out, gc_stream stream);

/* JP colouring, Algorithm 3 (Section 4.1), for an arbitrary priority:
 * vertex u precedes v (u is a predecessor of v in the DAG G_rho) iff
 * (priority[u], u) > (priority[v], v) lexicographically, so any array gives
 * a total order.  color_out[v] >= 1 (device, n int32) is the smallest colour
 * not used by v's predecessors; *num_colors_out (host) is the largest colour. */
gc_status gc_jp_color(gc_context *ctx, const gc_csr *g, const uint64_t *priority,
                      int32_t *color_out, int32_t *num_colors_out, gc_stream stream);

/* JP-ADG end to end: ADG with eps = eps_p/eps_q, then JP with the priority
 * of gc_make_priority(batch, seed), computed on the fly.  color_out (device,
 * n int32) is required; batch_out (device, n int32) may be NULL.  Both host
 * scalars may be NULL.  Same result as gc_adg_partition + gc_make_priority +
 * gc_jp_color. */
gc_status gc_color_graph(gc_context *ctx, const gc_csr *g, uint32_t eps_p, uint32_t eps_q,
                         uint64_t seed, int32_t *color_out, int32_t *batch_out,
                         int32_t *num_colors_out, int32_t *num_rounds_out, gc_stream stream);

/* gc_color_graph for a graph in HOST memory: copies row_ptr (n+1 int64) and
 * col_idx (nnz int32) to device buffers that the context owns and keeps for
 * reuse, colours the graph, and copies the colours (and, if batch_out is not
 * NULL, the batches) back to the host arrays of n int32.  Page-locked host
 * buffers make the copies asynchronous.  Returns after the results are on
 * the host. */
gc_status gc_color_graph_host(gc_context *ctx, int64_t n, int64_t nnz, const int64_t *row_ptr,
                              const int32_t *col_idx, uint32_t eps_p, uint32_t eps_q,
                              uint64_t seed, int32_t *color_out, int32_t *batch_out,
                              int32_t *num_colors_out, int32_t *num_rounds_out,
                              gc_stream stream);

/* A batch of graphs packed as one CSR: the disjoint union of the graphs.
 * Graph g owns the vertices [graph_off[g], graph_off[g+1]) and every edge of
 * a vertex stays inside its graph's range (not checked; edges across graphs
 * make the per-graph results undefined).  col_idx holds union ids.  The
 * graph_off array is device memory, non-decreasing, graph_off[0] = 0 and
 * graph_off[num_graphs] = n; empty graphs are allowed. */
typedef struct {
  int64_t num_graphs;
  int64_t n;                /* total vertices                       */
  int64_t nnz;              /* total CSR entries                    */
  const int64_t *row_ptr;   /* device, n+1                          */
  const int32_t *col_idx;   /* device, nnz (union ids)              */
  const int64_t *graph_off; /* device, num_graphs+1                 */
} gc_batch_csr;

/* Per-graph parameters of a batch: eps = eps_p / eps_q and the tie-break
 * seed, as in gc_color_graph. */
typedef struct {
  uint32_t eps_p;
  uint32_t eps_q;
  uint64_t seed;
} gc_job;

/* JP-ADG for every graph of a batch at once.  ADG (Algorithm 1) keeps its
 * degree sum, |U|, threshold and eps per graph, with one set of launches per
 * round serving all graphs still running; JP (Algorithm 3) runs once on the
 * union, each vertex's tie-break taken from its own graph's seed and its id
 * inside that graph.  Each graph's batches and colours are exactly those
 * gc_color_graph returns for it alone (batch ids and colours are local to the
 * graph, both starting at 1).  jobs: host array of num_graphs entries.
 * color_out: device, n int32 (required); batch_out: device, n int32, or NULL;
 * num_colors_out / num_rounds_out: device, num_graphs int32 each, or NULL. */
gc_status gc_color_batch(gc_context *ctx, const gc_batch_csr *b, const gc_job *jobs,
                         int32_t *color_out, int32_t *batch_out, int32_t *num_colors_out,
                         int32_t *num_rounds_out, gc_stream stream);

/* gc_color_batch for graphs held in separate device buffers: graphs[g] is a
 * gc_csr like gc_color_graph's (local ids 0..n_g-1, device pointers); jobs
 * and graphs are host arrays of num_graphs entries, color_out a host array
 * of num_graphs device pointers (n_g int32 each).  The graphs are packed
 * into their disjoint union inside a buffer the context owns (grown on
 * demand), coloured together, and each graph's colours written to its own
 * output; results equal gc_color_graph on each graph alone.  Returns after
 * the colours are written. */
gc_status gc_color_batch_list(gc_context *ctx, int64_t num_graphs, const gc_csr *graphs,
                              const gc_job *jobs, int32_t *const *color_out, gc_stream stream);

/* gc_autotune for gc_color_batch(b, jobs): also chooses between the
 * persistent and the segmented batch path (batch_mode). */
gc_status gc_autotune_batch(gc_context *ctx, const gc_batch_csr *b, const gc_job *jobs, int32_t reps,
                            float budget_ms, gc_options *best_out, float *best_ms_out, float *start_ms_out,
                            gc_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GCOLOR_H_ */
