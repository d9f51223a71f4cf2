/*
 * oracle.c -- plain, slow, obviously correct CPU reference for ADG and JP-ADG
 * (Besta et al., "High-Performance Parallel Graph Coloring with Strong
 * Guarantees on Work, Depth, and Quality", SC'20).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The CUDA library shares
 * no code, header, table or constant with it: the priority hash below is
 * written here from SplitMix64's published definition, independently of the
 * GPU side's own version.
 *
 * Single-threaded, exact integer arithmetic throughout.  Graph input is the
 * paper's CSR model (Section 2.1, "Graph Model and Representation"): n vertices, int64 row offsets row_ptr[n+1],
 * int32 neighbour ids col_idx[row_ptr[n]], undirected (both directions stored),
 * simple, rows sorted.
 *
 * Readings of the paper taken here:
 *  - R test uses "<=" (Algorithm 1, the definition of R; the proof of the
 *    round bound in Section 3 also uses <=), evaluated exactly in integers:
 *    D[u] <= (1+eps) * Sigma/|U|  with eps = p/q  <=>  q*|U|*D[u] <= (q+p)*Sigma
 *    <=> D[u] <= floor((q+p)*Sigma / (q*|U|)), computed in 128 bits.
 *  - Batch ids start at 1 (Algorithm 1 sets l = 1); 0 never appears in output.
 *  - Priority rho(v) = <rho_ADG(v), rho_R(v)> (Section 4.1), made a total
 *    order by the vertex id: key(v) = (batch(v), h_seed(v), v), compared
 *    lexicographically; a HIGHER key is coloured first (pred(v) = neighbours
 *    with higher rho, Algorithm 3).
 *  - h_seed(v) = upper 32 bits of the (v+1)-th output of SplitMix64 seeded
 *    with `seed` (Steele, Lea & Flood, OOPSLA 2014): the paper only says the
 *    tie-break is random.
 *  - Colours start at 1 (Algorithm 3 initialises C to 0 = uncoloured and
 *    GetColor draws from {1, ..., |pred|+1}).
 *  - JP with a total order produces exactly the sequential Greedy colouring
 *    in decreasing priority (Algorithm 3: GetColor of v reads only the colours
 *    of pred(v), which are all final when v is coloured).  So the colour
 *    oracle is Greedy (Section 1) in that order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Priority tie-break: SplitMix64.                                            */
/* The generator's state advances by the odd constant 0x9e3779b97f4a7c15 and */
/* each output is the state passed through the 64-bit finaliser with shifts   */
/* 30, 27, 31 and multipliers 0xbf58476d1ce4e5b9, 0x94d049bb133111eb.          */
/* ------------------------------------------------------------------------- */

uint64_t oracle_splitmix64_output(uint64_t seed, uint64_t k)
{
    /* k-th output (k >= 1) of SplitMix64 started from state `seed` */
    uint64_t z = seed + k * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    return z;
}

uint32_t oracle_tiebreak(uint64_t seed, int64_t v)
{
    return (uint32_t)(oracle_splitmix64_output(seed, (uint64_t)v + 1) >> 32);
}

/* ------------------------------------------------------------------------- */
/* ADG, Algorithm 1 (Section 3), step by step.                                */
/* ------------------------------------------------------------------------- */

/*
 * Inputs: CSR, eps = eps_p / eps_q.
 * Output: batch[v] = rho_ADG(v) in 1..num_rounds.
 * Optional per-round records (NULL to skip; at most max_log rounds written):
 *   log_U[l-1] = |U_l|, log_R[l-1] = |R_l|, log_sigma[l-1] = sum_{u in U_l} D[u],
 *   log_T[l-1] = floor((q+p)*Sigma / (q*|U|)).
 * Returns 0 on success, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_adg(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
               uint32_t eps_p, uint32_t eps_q, int32_t *batch, int32_t *num_rounds,
               int64_t *log_U, int64_t *log_R, int64_t *log_sigma, int64_t *log_T,
               int64_t max_log)
{
    if (n < 0 || eps_q == 0) return 1;
    int64_t *D = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    char *inU = (char *)malloc((size_t)(n > 0 ? n : 1));
    char *inR = (char *)malloc((size_t)(n > 0 ? n : 1));
    if (!D || !inU || !inR) { free(D); free(inU); free(inR); return 2; }

    /* D = [deg(v_1) ... deg(v_n)];  l = 1;  U = V */
    for (int64_t v = 0; v < n; ++v) {
        D[v] = row_ptr[v + 1] - row_ptr[v];
        inU[v] = 1;
        batch[v] = 0;
    }
    int64_t sizeU = n;
    int32_t l = 1;

    while (sizeU > 0) {
        /* |U| = Count(U);  cnt = Reduce(U) = sum of D over U (a fresh sum) */
        int64_t count = 0, cnt = 0;
        for (int64_t v = 0; v < n; ++v)
            if (inU[v]) { count += 1; cnt += D[v]; }

        /* R = {u in U : D[u] <= (1+eps) * cnt/|U|}, exactly in integers */
        unsigned __int128 num = (unsigned __int128)(eps_q + (uint64_t)eps_p) * (uint64_t)cnt;
        unsigned __int128 den = (unsigned __int128)eps_q * (uint64_t)count;
        unsigned __int128 T = num / den;
        int64_t sizeR = 0;
        for (int64_t v = 0; v < n; ++v) {
            inR[v] = (char)(inU[v] && (unsigned __int128)D[v] <= T);
            sizeR += inR[v];
        }

        if (l - 1 < max_log) {
            if (log_U) log_U[l - 1] = count;
            if (log_R) log_R[l - 1] = sizeR;
            if (log_sigma) log_sigma[l - 1] = cnt;
            if (log_T) log_T[l - 1] = T > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)T;
        }

        /* UPDATE(U, R, D): for v in R, for u in N_U(v): DecrementAndFetch(D[u]).
         * U still contains R here, as in the listing. */
        for (int64_t v = 0; v < n; ++v) {
            if (!inR[v]) continue;
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                int32_t u = col_idx[k];
                if (inU[u]) D[u] -= 1;
            }
        }

        /* U = U \ R;  rho_ADG(v) = l for v in R;  l = l + 1 */
        for (int64_t v = 0; v < n; ++v) {
            if (inR[v]) {
                inU[v] = 0;
                batch[v] = l;
            }
        }
        sizeU -= sizeR;
        if (sizeR == 0) { free(D); free(inU); free(inR); return 3; } /* cannot happen: min degree <= average */
        l += 1;
    }
    *num_rounds = l - 1;
    free(D);
    free(inU);
    free(inR);
    return 0;
}

/*
 * A second, deliberately naive ADG: every round recomputes each remaining
 * vertex's degree inside G[U] from scratch, D[u] = |N(u) cap U| (the quantity
 * Algorithm 1's UPDATE maintains).  O(rounds * nnz); tiny graphs only.
 */
int oracle_adg_naive(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     uint32_t eps_p, uint32_t eps_q, int32_t *batch, int32_t *num_rounds)
{
    if (n < 0 || eps_q == 0) return 1;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!deg) return 2;
    for (int64_t v = 0; v < n; ++v) batch[v] = 0;
    int64_t left = n;
    int32_t l = 0;
    while (left > 0) {
        ++l;
        int64_t sum = 0;
        for (int64_t v = 0; v < n; ++v) {
            deg[v] = 0;
            if (batch[v] != 0) continue;
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
                if (batch[col_idx[k]] == 0) deg[v] += 1;
            sum += deg[v];
        }
        /* threshold comparison by cross-multiplication, no division */
        int64_t removed = 0;
        for (int64_t v = 0; v < n; ++v) {
            if (batch[v] != 0) continue;
            unsigned __int128 lhs = (unsigned __int128)eps_q * (uint64_t)left * (uint64_t)deg[v];
            unsigned __int128 rhs = (unsigned __int128)(eps_q + (uint64_t)eps_p) * (uint64_t)sum;
            if (lhs <= rhs) deg[v] = -1; /* mark for removal */
        }
        for (int64_t v = 0; v < n; ++v)
            if (batch[v] == 0 && deg[v] == -1) { batch[v] = l; ++removed; }
        left -= removed;
        if (removed == 0) { free(deg); return 3; }
    }
    *num_rounds = l;
    free(deg);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* ADG-M (Section 5, "Degree Median Instead of Degree Average"): in each     */
/* round R is the set of vertices of U whose degree in U is at most the      */
/* median degree of U, limited to half of U (one more if |U| is odd).  With  */
/* the limit, R is exactly the ceil(|U|/2) vertices of U with the smallest   */
/* degree; vertices of equal degree are taken in increasing id order (the   */
/* paper leaves this tie open).  UPDATE is Algorithm 1's.                    */
/* ------------------------------------------------------------------------- */
static const int64_t *g_sort_D;
static int cmp_deg_id(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    if (g_sort_D[x] != g_sort_D[y]) return g_sort_D[x] < g_sort_D[y] ? -1 : 1;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_adg_m(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t *batch,
                 int32_t *num_rounds)
{
    if (n < 0) return 1;
    int64_t *D = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *U = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!D || !U) { free(D); free(U); return 2; }
    for (int64_t v = 0; v < n; ++v) {
        D[v] = row_ptr[v + 1] - row_ptr[v];
        U[v] = v;
        batch[v] = 0;
    }
    int64_t sizeU = n;
    int32_t l = 0;
    while (sizeU > 0) {
        ++l;
        /* the ceil(|U|/2) smallest (degree, id) of U */
        g_sort_D = D;
        qsort(U, (size_t)sizeU, sizeof(int64_t), cmp_deg_id);
        const int64_t sizeR = (sizeU + 1) / 2;
        for (int64_t i = 0; i < sizeR; ++i) batch[U[i]] = l;
        /* UPDATE: the degree in U of every remaining neighbour drops by one */
        for (int64_t i = 0; i < sizeR; ++i) {
            const int64_t v = U[i];
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
                if (batch[col_idx[k]] == 0) D[col_idx[k]] -= 1;
        }
        memmove(U, U + sizeR, sizeof(int64_t) * (size_t)(sizeU - sizeR));
        sizeU -= sizeR;
    }
    *num_rounds = l;
    free(D);
    free(U);
    return 0;
}

/* ADG-M with every degree recomputed from scratch in each round (O(n*m)):
 * a cross-check of the incremental UPDATE above, for tiny graphs. */
int oracle_adg_m_naive(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t *batch,
                       int32_t *num_rounds)
{
    if (n < 0) return 1;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    char *take = (char *)malloc((size_t)(n > 0 ? n : 1));
    if (!deg || !take) { free(deg); free(take); return 2; }
    for (int64_t v = 0; v < n; ++v) batch[v] = 0;
    int64_t left = n;
    int32_t l = 0;
    while (left > 0) {
        ++l;
        for (int64_t v = 0; v < n; ++v) {
            deg[v] = 0;
            take[v] = 0;
            if (batch[v] != 0) continue;
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
                if (batch[col_idx[k]] == 0) deg[v] += 1;
        }
        /* pick ceil(left/2) times the remaining vertex of smallest (deg, id) */
        const int64_t want = (left + 1) / 2;
        for (int64_t t = 0; t < want; ++t) {
            int64_t best = -1;
            for (int64_t v = 0; v < n; ++v) {
                if (batch[v] != 0 || take[v]) continue;
                if (best < 0 || deg[v] < deg[best]) best = v;
            }
            take[best] = 1;
        }
        for (int64_t v = 0; v < n; ++v)
            if (take[v]) batch[v] = l;
        left -= want;
    }
    *num_rounds = l;
    free(deg);
    free(take);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Greedy colouring in a given order (Section 1: each vertex in turn takes   */
/* the smallest colour not used by an already coloured neighbour).           */
/* ------------------------------------------------------------------------- */

int oracle_greedy(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                  const int64_t *order, int32_t *color, int32_t *num_colors)
{
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) {
        color[v] = 0;
        if (row_ptr[v + 1] - row_ptr[v] > maxdeg) maxdeg = row_ptr[v + 1] - row_ptr[v];
    }
    /* used[c] == stamp  <=>  colour c is taken by a coloured neighbour */
    int64_t *used = (int64_t *)calloc((size_t)(maxdeg + 2), sizeof(int64_t));
    if (!used) return 2;
    int32_t maxc = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = order[i];
        int64_t stamp = i + 1;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int32_t c = color[col_idx[k]];
            if (c > 0 && c <= maxdeg + 1) used[c] = stamp;
        }
        int32_t c = 1;
        while (used[c] == stamp) ++c;
        color[v] = c;
        if (c > maxc) maxc = c;
    }
    *num_colors = maxc;
    free(used);
    return 0;
}

/* ---- priority order: key(v) = (primary(v), secondary(v), v), descending ---- */

typedef struct {
    uint64_t primary;
    uint64_t secondary;
    int64_t v;
} okey;

static int okey_desc(const void *a, const void *b)
{
    const okey *x = (const okey *)a, *y = (const okey *)b;
    if (x->primary != y->primary) return x->primary > y->primary ? -1 : 1;
    if (x->secondary != y->secondary) return x->secondary > y->secondary ? -1 : 1;
    if (x->v != y->v) return x->v > y->v ? -1 : 1;
    return 0;
}

/* order[] = vertices sorted by (primary, secondary, id) descending */
static int order_desc(int64_t n, const uint64_t *primary, const uint64_t *secondary, int64_t *order)
{
    okey *k = (okey *)malloc(sizeof(okey) * (size_t)(n > 0 ? n : 1));
    if (!k) return 2;
    for (int64_t v = 0; v < n; ++v) {
        k[v].primary = primary ? primary[v] : 0;
        k[v].secondary = secondary ? secondary[v] : 0;
        k[v].v = v;
    }
    qsort(k, (size_t)n, sizeof(okey), okey_desc);
    for (int64_t i = 0; i < n; ++i) order[i] = k[i].v;
    free(k);
    return 0;
}

/* JP-ADG priority key as one 64-bit word: (batch << 32) | h_seed(v); ties on
 * the word are broken by the larger vertex id. */
void oracle_priority(int64_t n, const int32_t *batch, uint64_t seed, uint64_t *key)
{
    for (int64_t v = 0; v < n; ++v)
        key[v] = ((uint64_t)(uint32_t)batch[v] << 32) | (uint64_t)oracle_tiebreak(seed, v);
}

/* Priorities of the other JP variants (Section 4.1, "combinations of JP and
 * orderings"), as 64-bit keys compared in decreasing (key, id) order:
 *   kind 0, JP-R:   rho_R                             h(v)
 *   kind 1, JP-FF:  natural vertex order (v = 0 first) 2^32 - 1 - v
 *   kind 2, JP-LF:  <deg(v), rho_R>                   deg(v) * 2^32 + h(v)
 *   kind 3, JP-LLF: <ceil(log2 deg(v)), rho_R>        that * 2^32 + h(v)
 * where ceil(log2 d) is the smallest k with 2^k >= d (0 for d <= 1) and h is
 * oracle_tiebreak.  Returns 1 for an unknown kind. */
static uint64_t ceil_log2_u64(uint64_t d)
{
    uint64_t k = 0;
    while (d > 1 && ((uint64_t)1 << k) < d) ++k;
    return k;
}

int oracle_priority_kind(int64_t n, const int64_t *row_ptr, int kind, uint64_t seed, uint64_t *key)
{
    if (kind < 0 || kind > 3) return 1;
    for (int64_t v = 0; v < n; ++v) {
        const uint64_t h = (uint64_t)oracle_tiebreak(seed, v);
        const uint64_t d = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
        if (kind == 0)
            key[v] = h;
        else if (kind == 1)
            key[v] = 0xffffffffull - (uint64_t)v;
        else if (kind == 2)
            key[v] = (d << 32) | h;
        else
            key[v] = (ceil_log2_u64(d) << 32) | h;
    }
    return 0;
}

/* JP colouring (Algorithm 3) for an arbitrary priority array, via its
 * equivalent Greedy in decreasing (priority, id) order. */
int oracle_jp_color(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                    const uint64_t *priority, int32_t *color, int32_t *num_colors)
{
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!order) return 2;
    int rc = order_desc(n, priority, NULL, order);
    if (rc == 0) rc = oracle_greedy(n, row_ptr, col_idx, order, color, num_colors);
    free(order);
    return rc;
}

/* Full JP-ADG: ADG batches, then colouring in (batch, h_seed, id) order. */
int oracle_jp_adg(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                  uint32_t eps_p, uint32_t eps_q, uint64_t seed,
                  int32_t *batch, int32_t *color, int32_t *num_rounds, int32_t *num_colors)
{
    int rc = oracle_adg(n, row_ptr, col_idx, eps_p, eps_q, batch, num_rounds,
                        NULL, NULL, NULL, NULL, 0);
    if (rc) return rc;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!key) return 2;
    oracle_priority(n, batch, seed, key);
    rc = oracle_jp_color(n, row_ptr, col_idx, key, color, num_colors);
    free(key);
    return rc;
}

/* |pred(v)| = number of neighbours with a higher (priority, id) (Algorithm 3,
 * Part 1: count[v] = |pred[v]|). */
void oracle_pred_count(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const uint64_t *priority, int32_t *count)
{
    for (int64_t v = 0; v < n; ++v) {
        int32_t c = 0;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int64_t w = col_idx[k];
            if (priority[w] > priority[v] || (priority[w] == priority[v] && w > v)) ++c;
        }
        count[v] = c;
    }
}

/* Longest path (in vertices) of the DAG G_rho whose edges run from higher to
 * lower (priority, id); depth[v] = 1 + max depth over pred(v).  Returns the
 * maximum: the number of dependency steps JP needs. */
int64_t oracle_jp_depth(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                        const uint64_t *priority, int32_t *depth)
{
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!order) return -1;
    if (order_desc(n, priority, NULL, order)) { free(order); return -1; }
    int64_t best = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t v = order[i];
        int32_t dv = 1;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int64_t w = col_idx[k];
            if (priority[w] > priority[v] || (priority[w] == priority[v] && w > v))
                if (depth[w] + 1 > dv) dv = depth[w] + 1;
        }
        depth[v] = dv;
        if (dv > best) best = dv;
    }
    free(order);
    return best;
}

/* ------------------------------------------------------------------------- */
/* ADG-O (Algorithm 6; Section 5, "Explicit Ordering in R" and "Detailed     */
/* Algorithm Specifications"): ADG whose removed set R is sorted by           */
/* increasing D before it is numbered, so that rho is a total order.         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t d;
    int64_t v;
} dkey;

static int dkey_asc(const void *a, const void *b)
{
    const dkey *x = (const dkey *)a, *y = (const dkey *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/*
 * Inputs: CSR, eps = eps_p / eps_q.  Outputs: batch[v] = the iteration that
 * removed v (1-based, as in Algorithm 1), rho[v] in 0..n-1 = Algorithm 6's
 * rho_ADG (l + i for the i-th vertex of the sorted R, l = vertices removed
 * before), rank[v] = its count of neighbours with a higher rho (Algorithm 6's
 * UPDATEandPRIORITIZE), *num_rounds.
 * Readings: R is sorted by increasing D with equal D in increasing vertex id
 * (the paper leaves ties open; the sort is meant to make the order total);
 * the threshold is Algorithm 1's, evaluated exactly in integers.
 * Returns 0, 1 on bad arguments, 2 on allocation failure.
 */
int oracle_adg_o(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t eps_p,
                 uint32_t eps_q, int32_t *batch, int64_t *rho, int64_t *rank, int32_t *num_rounds)
{
    if (n < 0 || eps_q == 0) return 1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t *D = (int64_t *)malloc(sizeof(int64_t) * nn);
    char *inU = (char *)malloc(nn);
    dkey *R = (dkey *)malloc(sizeof(dkey) * nn);
    if (!D || !inU || !R) { free(D); free(inU); free(R); return 2; }
    /* D = degrees; U = V; l = 0; rho(v) = n for all v */
    for (int64_t v = 0; v < n; ++v) {
        D[v] = row_ptr[v + 1] - row_ptr[v];
        inU[v] = 1;
        rho[v] = n;
        rank[v] = 0;
        batch[v] = 0;
    }
    int64_t sizeU = n, l = 0;
    int32_t round = 0;
    while (sizeU > 0) {
        ++round;
        /* the average degree of U, as an exact threshold on D */
        int64_t count = 0, cnt = 0;
        for (int64_t v = 0; v < n; ++v)
            if (inU[v]) { count += 1; cnt += D[v]; }
        unsigned __int128 num = (unsigned __int128)(eps_q + (uint64_t)eps_p) * (uint64_t)cnt;
        unsigned __int128 den = (unsigned __int128)eps_q * (uint64_t)count;
        unsigned __int128 T = num / den;
        /* PARTITION: R = {u in U : D[u] <= (1+eps) * average} */
        int64_t sizeR = 0;
        for (int64_t v = 0; v < n; ++v)
            if (inU[v] && (unsigned __int128)D[v] <= T) { R[sizeR].d = D[v]; R[sizeR].v = v; ++sizeR; }
        if (sizeR == 0) { free(D); free(inU); free(R); return 3; } /* cannot happen */
        /* SORT(R, D) by increasing D */
        qsort(R, (size_t)sizeR, sizeof(dkey), dkey_asc);
        /* rho(r_i) = l + i */
        for (int64_t i = 0; i < sizeR; ++i) {
            rho[R[i].v] = l + i;
            batch[R[i].v] = round;
        }
        /* &U = &U + |R| */
        for (int64_t i = 0; i < sizeR; ++i) inU[R[i].v] = 0;
        sizeU -= sizeR;
        /* UPDATEandPRIORITIZE: for v in R, every neighbour w after v in the
         * order loses one from D[w]; rank(v) counts them */
        for (int64_t i = 0; i < sizeR; ++i) {
            const int64_t v = R[i].v;
            int64_t c = 0;
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                const int32_t w = col_idx[k];
                if (rho[w] > rho[v]) {
                    D[w] -= 1;
                    c += 1;
                }
            }
            rank[v] = c;
        }
        l += sizeR;
    }
    *num_rounds = round;
    free(D);
    free(inU);
    free(R);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* DEC-ADG-ITR (Section 4.3): DEC-ADG's partition-by-partition colouring     */
/* (Algorithm 4) with SIM-COL (Algorithm 5) changed to give every vertex of U */
/* the smallest colour not in B_v instead of a random one.                    */
/* ------------------------------------------------------------------------- */

/*
 * Inputs: CSR, batch[v] in 1..rounds (the partitions R(l) of an ADG run),
 * seed of the tie-break.  Readings taken here:
 *  - Partitions are coloured from l = rounds down to 1 (Algorithm 4).
 *  - B_v is the set of colours of v's coloured neighbours: before SIM-COL on
 *    R(l) it receives the colours of neighbours in R(rounds) .. R(l+1)
 *    (Algorithm 4), and after each SIM-COL iteration the colours of
 *    neighbours in U that kept theirs (Algorithm 5, Part 3).  It is stored as
 *    a bitmap of deg(v) + 1 bits: the smallest colour not in B_v is at most
 *    |B_v| + 1 <= deg(v) + 1, so larger colours never decide it.
 *  - Every step of a SIM-COL iteration reads the state the previous step
 *    left (a synchronous parallel step): Part 2 compares the colours all of
 *    U drew in Part 1.
 *  - Conflict rule: the paper resets every vertex of a monochromatic edge in
 *    U.  With deterministic choices that never ends (two adjacent vertices
 *    with equal B draw the same colour again), so only the endpoint with the
 *    lower key (h_seed(v), v) resets; the higher one keeps its colour.  The
 *    highest-key vertex of U therefore keeps its colour in every iteration
 *    and each SIM-COL call ends after at most |R(l)| iterations.
 * Outputs: color[v] >= 1, *num_colors, *iterations = SIM-COL iterations summed
 * over the partitions, and (if non-NULL) fixed_iter[v] = the iteration of
 * SIM-COL on R(batch[v]) in which v kept its colour (1-based).
 * Returns 0, 1 on bad arguments (a batch outside 1..rounds), 2 on allocation
 * failure.
 */
int oracle_dec_adg_itr(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const int32_t *batch, int32_t rounds, uint64_t seed,
                       int32_t *color, int32_t *fixed_iter, int32_t *num_colors,
                       int64_t *iterations)
{
    if (n < 0 || rounds < 0) return 1;
    for (int64_t v = 0; v < n; ++v)
        if (batch[v] < 1 || batch[v] > rounds) return 1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t *boff = (int64_t *)malloc(sizeof(int64_t) * (nn + 1));   /* bitmap offsets, in bytes */
    uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    char *inU = (char *)calloc(nn, 1);
    char *lose = (char *)calloc(nn, 1);
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *part_start = (int64_t *)calloc((size_t)rounds + 2, sizeof(int64_t));
    if (!boff || !h || !inU || !lose || !members || !part_start) {
        free(boff); free(h); free(inU); free(lose); free(members); free(part_start);
        return 2;
    }
    boff[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t bits = row_ptr[v + 1] - row_ptr[v] + 1;  /* colours 1 .. deg(v)+1 */
        boff[v + 1] = boff[v] + (bits + 7) / 8;
        h[v] = oracle_tiebreak(seed, v);
        color[v] = 0;
        if (fixed_iter) fixed_iter[v] = 0;
    }
    unsigned char *B = (unsigned char *)calloc((size_t)(boff[n] > 0 ? boff[n] : 1), 1);
    if (!B) {
        free(boff); free(h); free(inU); free(lose); free(members); free(part_start);
        return 2;
    }
    /* members[] lists the vertices partition by partition: R(l) is
     * members[part_start[l] .. part_start[l+1]) */
    for (int64_t v = 0; v < n; ++v) part_start[batch[v] + 1] += 1;
    for (int32_t l = 1; l <= rounds; ++l) part_start[l + 1] += part_start[l];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)rounds + 2));
        if (!fill) {
            free(B); free(boff); free(h); free(inU); free(lose); free(members); free(part_start);
            return 2;
        }
        memcpy(fill, part_start, sizeof(int64_t) * ((size_t)rounds + 2));
        for (int64_t v = 0; v < n; ++v) members[fill[batch[v]]++] = v;
        free(fill);
    }

#define B_HAS(v, c) ((B[boff[v] + ((c) - 1) / 8] >> (((c) - 1) % 8)) & 1)
#define B_ADD(v, c)                                                             \
    do {                                                                        \
        if ((int64_t)(c) <= row_ptr[(v) + 1] - row_ptr[(v)] + 1)                \
            B[boff[v] + ((c) - 1) / 8] |= (unsigned char)(1u << (((c) - 1) % 8)); \
    } while (0)

    int32_t maxc = 0;
    int64_t iters = 0;
    for (int32_t l = rounds; l >= 1; --l) {
        const int64_t *R = members + part_start[l];
        const int64_t sizeR = part_start[l + 1] - part_start[l];
        /* Algorithm 4: B_v gets the colours of v's neighbours in the
         * partitions coloured already (batch > l). */
        for (int64_t i = 0; i < sizeR; ++i) {
            const int64_t v = R[i];
            for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                const int32_t u = col_idx[k];
                if (batch[u] > l) B_ADD(v, color[u]);
            }
        }
        /* SIM-COL on G(l) with U = R(l) */
        int64_t sizeU = sizeR;
        for (int64_t i = 0; i < sizeR; ++i) inU[R[i]] = 1;
        int32_t it = 0;
        while (sizeU > 0) {
            ++it;
            /* Part 1: every v in U takes the smallest colour not in B_v */
            for (int64_t i = 0; i < sizeR; ++i) {
                const int64_t v = R[i];
                if (!inU[v]) continue;
                int32_t c = 1;
                while (B_HAS(v, c)) ++c;
                color[v] = c;
            }
            /* Part 2: v resets if a neighbour in U with a higher key drew the
             * same colour (decided for all of U before any reset) */
            for (int64_t i = 0; i < sizeR; ++i) {
                const int64_t v = R[i];
                if (!inU[v]) continue;
                lose[v] = 0;
                for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                    const int32_t u = col_idx[k];
                    if (!inU[u] || color[u] != color[v]) continue;
                    if (h[u] > h[v] || (h[u] == h[v] && u > v)) { lose[v] = 1; break; }
                }
            }
            for (int64_t i = 0; i < sizeR; ++i) {
                const int64_t v = R[i];
                if (inU[v] && lose[v]) color[v] = 0;
            }
            /* Part 3: B_v gets the colours of neighbours in U that kept theirs */
            for (int64_t i = 0; i < sizeR; ++i) {
                const int64_t v = R[i];
                if (!inU[v]) continue;
                for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                    const int32_t u = col_idx[k];
                    if (inU[u] && color[u] > 0) B_ADD(v, color[u]);
                }
            }
            /* U = U \ {v in U : C[v] > 0} */
            for (int64_t i = 0; i < sizeR; ++i) {
                const int64_t v = R[i];
                if (inU[v] && color[v] > 0) {
                    inU[v] = 0;
                    --sizeU;
                    if (fixed_iter) fixed_iter[v] = it;
                    if (color[v] > maxc) maxc = color[v];
                }
            }
        }
        iters += it;
    }
#undef B_HAS
#undef B_ADD
    *num_colors = maxc;
    *iterations = iters;
    free(B); free(boff); free(h); free(inU); free(lose); free(members); free(part_start);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exact degeneracy by smallest-last peeling (Matula & Beck; Section 2.2):   */
/* repeatedly remove a vertex of minimum remaining degree.  d is the largest */
/* degree seen at removal; order[] is the removal sequence (first removed    */
/* first).  Bucket queue, O(n + m).                                          */
/* ------------------------------------------------------------------------- */

int64_t oracle_degeneracy(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int64_t *order)
{
    if (n == 0) return 0;
    int64_t maxdeg = 0;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        if (deg[v] > maxdeg) maxdeg = deg[v];
    }
    /* doubly linked bucket lists */
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 1));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    char *gone = (char *)calloc((size_t)n, 1);
    for (int64_t d = 0; d <= maxdeg; ++d) head[d] = -1;
    for (int64_t v = 0; v < n; ++v) {
        prev[v] = -1;
        next[v] = head[deg[v]];
        if (head[deg[v]] >= 0) prev[head[deg[v]]] = v;
        head[deg[v]] = v;
    }
    int64_t d = 0, cur = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (cur > 0) cur -= 1; /* the minimum can drop by at most one per removal */
        while (head[cur] < 0) ++cur;
        int64_t v = head[cur];
        /* unlink v */
        head[cur] = next[v];
        if (next[v] >= 0) prev[next[v]] = -1;
        gone[v] = 1;
        order[i] = v;
        if (cur > d) d = cur;
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int64_t w = col_idx[k];
            if (gone[w]) continue;
            /* move w from bucket deg[w] to deg[w]-1 */
            if (prev[w] >= 0) next[prev[w]] = next[w]; else head[deg[w]] = next[w];
            if (next[w] >= 0) prev[next[w]] = prev[w];
            deg[w] -= 1;
            prev[w] = -1;
            next[w] = head[deg[w]];
            if (head[deg[w]] >= 0) prev[head[deg[w]]] = w;
            head[deg[w]] = w;
        }
    }
    free(deg); free(head); free(next); free(prev); free(gone);
    return d;
}

/* ------------------------------------------------------------------------- */
/* Chromatic number by exhaustive backtracking (n <= 16), a lower bound for  */
/* every proper colouring (Section 1).                                        */
/* ------------------------------------------------------------------------- */

static int try_color(int64_t v, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                     int32_t k, int32_t *c)
{
    if (v == n) return 1;
    for (int32_t col = 1; col <= k; ++col) {
        int ok = 1;
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (col_idx[e] < v && c[col_idx[e]] == col) { ok = 0; break; }
        if (!ok) continue;
        c[v] = col;
        if (try_color(v + 1, n, row_ptr, col_idx, k, c)) return 1;
    }
    c[v] = 0;
    return 0;
}

int32_t oracle_chromatic_number(int64_t n, const int64_t *row_ptr, const int32_t *col_idx)
{
    if (n == 0) return 0;
    if (n > 16) return -1;
    int32_t c[16];
    for (int32_t k = 1; k <= (int32_t)n; ++k) {
        memset(c, 0, sizeof(c));
        if (try_color(0, n, row_ptr, col_idx, k, c)) return k;
    }
    return (int32_t)n;
}

/* ------------------------------------------------------------------------- */
/* Smallest-last order for JP-SL (Section 4.1 lists SL among the orderings   */
/* JP is combined with; Matula-Beck peeling): repeatedly remove a vertex of  */
/* minimum degree in the remaining graph.  The paper fixes no tie rule; the  */
/* reading taken is the vertex of minimum (current degree, id).  A binary    */
/* heap of (degree, id) entries with lazy deletion: an entry is stale once   */
/* its vertex is gone or its degree has dropped.  order[i] = i-th removed.   */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t d;
    int64_t v;
} sl_ent;

static int sl_less(sl_ent a, sl_ent b)
{
    return a.d < b.d || (a.d == b.d && a.v < b.v);
}

static void sl_push(sl_ent *h, int64_t *size, sl_ent e)
{
    int64_t i = (*size)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!sl_less(h[i], h[p])) break;
        sl_ent t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static sl_ent sl_pop(sl_ent *h, int64_t *size)
{
    sl_ent top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *size && sl_less(h[l], h[m])) m = l;
        if (r < *size && sl_less(h[r], h[m])) m = r;
        if (m == i) break;
        sl_ent t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

int oracle_smallest_last(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int64_t *order)
{
    if (n == 0) return 0;
    const int64_t nnz = row_ptr[n];
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    char *gone = (char *)calloc((size_t)n, 1);
    /* every vertex enters once, then once more per decrement: n + nnz/2 entries at most */
    sl_ent *heap = (sl_ent *)malloc(sizeof(sl_ent) * (size_t)(n + nnz / 2 + 1));
    if (!deg || !gone || !heap) { free(deg); free(gone); free(heap); return 2; }
    int64_t size = 0;
    for (int64_t v = 0; v < n; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        sl_ent e = {deg[v], v};
        sl_push(heap, &size, e);
    }
    int64_t i = 0;
    while (i < n) {
        sl_ent e = sl_pop(heap, &size);
        if (gone[e.v] || e.d != deg[e.v]) continue;  /* stale entry */
        gone[e.v] = 1;
        order[i++] = e.v;
        for (int64_t k = row_ptr[e.v]; k < row_ptr[e.v + 1]; ++k) {
            int64_t w = col_idx[k];
            if (gone[w]) continue;
            deg[w] -= 1;
            sl_ent f = {deg[w], w};
            sl_push(heap, &size, f);
        }
    }
    free(deg); free(gone); free(heap);
    return 0;
}
