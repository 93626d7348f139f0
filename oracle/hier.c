/*
 * ORACLE -- test infrastructure only.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load this code.  It shares no
 * code with the CUDA library and must never be called by it.
 *
 * Plain, sequential C for the two integer-producing steps of the aggregation
 * hierarchy (Section 2.2):
 *
 *   oh_match:  the maximal-weight matching coarsening.  Vertices are visited
 *              in random order; an unaggregated vertex is paired with its
 *              heaviest unaggregated neighbour (Section 2.2, first paragraph).
 *              Vertices left over afterwards join the aggregate that holds
 *              their heaviest neighbour (Section 2.2 and Section 4, first
 *              paragraph).
 *   oh_coarse: the Galerkin coarse graph of one level, (P^{k+1}_k)^T L_k
 *              P^{k+1}_k with P the 0/1 aggregation matrix of Section 2.2:
 *              coarse edge (I,J) carries the summed weight of all fine edges
 *              between aggregates I and J.
 *
 * Readings of points the paper leaves open:
 *   - "random order": the visit order of level k is the vertices sorted by
 *     the key SplitMix64(seed, (k << 32 | u) + 1), ties by vertex id, where
 *     SplitMix64(seed, i) is the i-th output of Steele, Lea & Flood's
 *     SplitMix64 generator started at `seed`, i.e. mix64(seed + i*golden).
 *     randomise == 0 visits vertices in increasing id order.
 *   - ties between equally heavy neighbours go to the smallest vertex id.
 *   - aggregates are numbered in the order they are created.
 *   - coarse weights are summed in the order (fine vertex ascending, CSR
 *     position ascending), starting from 0.0, in IEEE double.
 *   - coarse CSR rows list their columns in ascending order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t oh_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i >= 1) of SplitMix64 seeded with `seed`. */
uint64_t oh_splitmix64(uint64_t seed, uint64_t i)
{
    return oh_mix64(seed + i * 0x9E3779B97F4A7C15ULL);
}

typedef struct { uint64_t key; int64_t id; } oh_keyed;

static int oh_cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int oh_cmp_keyed(const void *a, const void *b)
{
    const oh_keyed *x = (const oh_keyed *)a, *y = (const oh_keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Visit order of level `level` (1 = the input graph). */
void oh_visit_order(int64_t n, uint64_t seed, int32_t level, int32_t randomise, int64_t *order)
{
    int64_t u;
    if (!randomise) {
        for (u = 0; u < n; ++u) order[u] = u;
        return;
    }
    oh_keyed *k = (oh_keyed *)malloc((size_t)n * sizeof(oh_keyed));
    for (u = 0; u < n; ++u) {
        k[u].key = oh_splitmix64(seed, (((uint64_t)(uint32_t)level) << 32 | (uint64_t)u) + 1ULL);
        k[u].id = u;
    }
    qsort(k, (size_t)n, sizeof(oh_keyed), oh_cmp_keyed);
    for (u = 0; u < n; ++u) order[u] = k[u].id;
    free(k);
}

/*
 * Aggregate the level graph (n, rp, ci, w).  Writes agg[u] (aggregate id of
 * u) and, per aggregate j, pair_a[j] (the visited vertex that created it) and
 * pair_b[j] (its matched partner).  Returns the number of aggregates.
 */
int64_t oh_match(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                 uint64_t seed, int32_t level, int32_t randomise,
                 int32_t *agg, int32_t *pair_a, int32_t *pair_b)
{
    int64_t *order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t i, u, p, count = 0;
    oh_visit_order(n, seed, level, randomise, order);
    for (u = 0; u < n; ++u) agg[u] = -1;

    /* matching pass in visit order */
    for (i = 0; i < n; ++i) {
        u = order[i];
        if (agg[u] >= 0) continue;
        int64_t best = -1;
        double bw = 0.0;
        for (p = rp[u]; p < rp[u + 1]; ++p) {
            int64_t v = ci[p];
            if (v == u || agg[v] >= 0) continue;
            if (best < 0 || w[p] > bw || (w[p] == bw && v < best)) { best = v; bw = w[p]; }
        }
        if (best >= 0) {
            agg[u] = (int32_t)count;
            agg[best] = (int32_t)count;
            pair_a[count] = (int32_t)u;
            pair_b[count] = (int32_t)best;
            ++count;
        }
    }
    /* leftovers join the aggregate of their heaviest neighbour */
    for (u = 0; u < n; ++u) {
        if (agg[u] >= 0) continue;
        int64_t best = -1;
        double bw = 0.0;
        for (p = rp[u]; p < rp[u + 1]; ++p) {
            int64_t v = ci[p];
            if (v == u) continue;
            if (best < 0 || w[p] > bw || (w[p] == bw && v < best)) { best = v; bw = w[p]; }
        }
        /* every neighbour of a leftover was matched, so agg[best] >= 0 */
        agg[u] = (best >= 0) ? agg[best] : -1;
    }
    free(order);
    return count;
}

/*
 * Coarse graph of one level.  With crp == NULL only counts: returns the
 * number of stored coarse entries.  Otherwise fills crp[nc+1], cci, cw.
 */
int64_t oh_coarse(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                  const int32_t *agg, int64_t nc,
                  int64_t *crp, int32_t *cci, double *cw)
{
    /* members of each aggregate in ascending vertex order */
    int64_t *mptr = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    int64_t *mem = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    double *acc = (double *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    int64_t *mark = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    int64_t *touched = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    int64_t u, I, p, t, total = 0;

    for (u = 0; u < n; ++u) mptr[agg[u] + 1]++;
    for (I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
    for (I = 0; I < nc; ++I) fill[I] = mptr[I];
    for (u = 0; u < n; ++u) mem[fill[agg[u]]++] = u;
    for (I = 0; I < nc; ++I) mark[I] = -1;

    if (crp) crp[0] = 0;
    for (I = 0; I < nc; ++I) {
        int64_t nt = 0;
        for (t = mptr[I]; t < mptr[I + 1]; ++t) {
            u = mem[t];
            for (p = rp[u]; p < rp[u + 1]; ++p) {
                int64_t J = agg[ci[p]];
                if (J == I) continue;
                if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; touched[nt++] = J; }
                acc[J] += w[p];
            }
        }
        /* ascending column order */
        qsort(touched, (size_t)nt, sizeof(int64_t), oh_cmp_i64);
        if (crp) {
            for (t = 0; t < nt; ++t) {
                cci[total + t] = (int32_t)touched[t];
                cw[total + t] = acc[touched[t]];
            }
            crp[I + 1] = total + nt;
        }
        total += nt;
    }
    free(mptr); free(mem); free(fill); free(acc); free(mark); free(touched);
    return total;
}
