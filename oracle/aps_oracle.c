/*
 * aps_oracle.c -- plain CPU oracle for the All-Pairs similarity join.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline (and its reference arm) load this library. The CUDA product path shares no
 * code, header or table with it.
 *
 * Everything here is FP64 arithmetic on the FP32 input values, written to be read
 * against the paper (Ozkural & Aykanat, "1-D and 2-D Parallel Algorithms for All-Pairs
 * Similarity Problem"):
 *
 *   Sec. 2.1      problem definition: M = {(v_i, v_j) : i != j, dot(v_i, v_j) >= t}
 *                 for unit-norm vectors; pairs are unordered and reported once, i < j.
 *   Sec. 3.2.2    all-pairs-0 (Alg. 1 + Alg. 2), all-pairs-1 (partial indexing),
 *                 all-pairs-2 (minsize, remscore, upperbound).
 *   Sec. 4        all-pairs-0-array (dense score array) and all-pairs-bruteforce.
 *
 * Readings of passages that are ambiguous in the paper:
 *   - matches use ">= t" (the definition), not "> t";
 *   - dimensions are ranked by decreasing non-zero count, ties by ascending id;
 *   - with minsize, vectors are processed by decreasing maxweight(x), ties by id, so
 *     that t/maxweight(x) never decreases (the text orders them the other way round,
 *     which contradicts the pop-from-the-front argument it makes);
 *   - partial indexing indexes a component once the running bound b reaches t (b >= t);
 *   - with remscore, Find-Matches walks x's components from the sparsest dimension to
 *     the densest, and remscore still includes the component being processed when the
 *     admission test is made (this is the order in which the bound is sound together
 *     with partial indexing).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PARTIAL_INDEX 1u /* all-pairs-1: partial indexing */
#define OR_MINSIZE 2u       /* all-pairs-2: minsize */
#define OR_REMSCORE 4u      /* all-pairs-2: remscore */
#define OR_UPPERBOUND 8u    /* all-pairs-2: upperbound */
/* Planted mistake for tests only: remscore with x's components walked densest first.
 * Tests use it to show that the test inputs can tell the two orders apart. */
#define OR_REMSCORE_FORWARD 256u

/* ------------------------------------------------------------------ result list */

typedef struct or_result {
    int64_t n, cap;
    int32_t *i, *j;
    double *s;
} or_result;

or_result *or_result_new(void) { return (or_result *)calloc(1, sizeof(or_result)); }

void or_result_free(or_result *r) {
    if (!r) return;
    free(r->i);
    free(r->j);
    free(r->s);
    free(r);
}

int64_t or_result_count(const or_result *r) { return r->n; }

void or_result_copy(const or_result *r, int32_t *i, int32_t *j, double *s) {
    memcpy(i, r->i, sizeof(int32_t) * (size_t)r->n);
    memcpy(j, r->j, sizeof(int32_t) * (size_t)r->n);
    memcpy(s, r->s, sizeof(double) * (size_t)r->n);
}

static int push_raw(or_result *r, int32_t a, int32_t b, double s) {
    if (r->n == r->cap) {
        int64_t cap = r->cap ? 2 * r->cap : 1024;
        int32_t *ni = (int32_t *)realloc(r->i, sizeof(int32_t) * (size_t)cap);
        if (ni) r->i = ni;
        int32_t *nj = (int32_t *)realloc(r->j, sizeof(int32_t) * (size_t)cap);
        if (nj) r->j = nj;
        double *ns = (double *)realloc(r->s, sizeof(double) * (size_t)cap);
        if (ns) r->s = ns;
        if (!ni || !nj || !ns) return -1;
        r->cap = cap;
    }
    r->i[r->n] = a;
    r->j[r->n] = b;
    r->s[r->n] = s;
    r->n++;
    return 0;
}

/* unordered pair, reported once with the smaller id first (Sec. 2.1) */
static int push(or_result *r, int32_t a, int32_t b, double s) {
    return a < b ? push_raw(r, a, b, s) : push_raw(r, b, a, s);
}

/* ------------------------------------------------------------ brute force (Sec. 4) */

/* dot(x, y) = sum_i x[i] * y[i] (Sec. 2.1), rows given as lists sorted by dimension. */
static double dot_sorted(const int32_t *ia, const float *va, int64_t na, const int32_t *ib,
                         const float *vb, int64_t nb) {
    double s = 0.0;
    int64_t p = 0, q = 0;
    while (p < na && q < nb) {
        if (ia[p] == ib[q]) {
            s += (double)va[p] * (double)vb[q];
            p++;
            q++;
        } else if (ia[p] < ib[q]) {
            p++;
        } else {
            q++;
        }
    }
    return s;
}

/* all-pairs-bruteforce: every pair's dot product, no intermediate data structure.
 * Returns the number of matches, or -1 on allocation failure. */
int64_t or_bruteforce(int32_t n, const int64_t *indptr, const int32_t *idx, const float *val,
                      double t, or_result *out) {
    for (int32_t a = 0; a < n; a++) {
        for (int32_t b = a + 1; b < n; b++) {
            double s = dot_sorted(idx + indptr[a], val + indptr[a], indptr[a + 1] - indptr[a],
                                  idx + indptr[b], val + indptr[b], indptr[b + 1] - indptr[b]);
            if (s >= t && push(out, a, b, s)) return -1;
        }
    }
    return out->n;
}

/* Brute force restricted to a list of rows: every pair (r, j), j != r, with
 * dot >= t, for each listed r. Used to check large outputs row by row. */
int64_t or_bruteforce_rows(int32_t n, const int64_t *indptr, const int32_t *idx,
                           const float *val, double t, const int32_t *rows, int32_t nrows,
                           or_result *out) {
    for (int32_t k = 0; k < nrows; k++) {
        int32_t a = rows[k];
        for (int32_t b = 0; b < n; b++) {
            if (b == a) continue;
            double s = dot_sorted(idx + indptr[a], val + indptr[a], indptr[a + 1] - indptr[a],
                                  idx + indptr[b], val + indptr[b], indptr[b + 1] - indptr[b]);
            if (s >= t && push(out, a, b, s)) return -1;
        }
    }
    return out->n;
}

/* Query set against a vector set (the matching step of the horizontal algorithm, Alg. 6,
 * where gathered query vectors are matched against a local index): every (q, y) with
 * dot(q, y) >= t. Reported as (i = query row, j = vector id), not reordered. */
int64_t or_bruteforce_cross(int32_t nq, const int64_t *qptr, const int32_t *qidx,
                            const float *qval, int32_t n, const int64_t *indptr,
                            const int32_t *idx, const float *val, double t, or_result *out) {
    for (int32_t a = 0; a < nq; a++) {
        for (int32_t b = 0; b < n; b++) {
            double s = dot_sorted(qidx + qptr[a], qval + qptr[a], qptr[a + 1] - qptr[a],
                                  idx + indptr[b], val + indptr[b], indptr[b + 1] - indptr[b]);
            if (s >= t && push_raw(out, a, b, s)) return -1;
        }
    }
    return out->n;
}

/* ------------------------------------------------------- preprocessing (Sec. 3.2.2) */

/* |x| (list length), maxweight(x), per-dimension non-zero count and
 * maxweight_i(V) = largest weight of dimension i over the whole dataset. */
void or_stats(int32_t n, int32_t m, const int64_t *indptr, const int32_t *idx, const float *val,
              int32_t *len, float *mw, int32_t *nnz_d, float *mw_d) {
    for (int32_t d = 0; d < m; d++) {
        nnz_d[d] = 0;
        mw_d[d] = 0.0f;
    }
    for (int32_t x = 0; x < n; x++) {
        len[x] = (int32_t)(indptr[x + 1] - indptr[x]);
        float best = 0.0f;
        for (int64_t p = indptr[x]; p < indptr[x + 1]; p++) {
            if (val[p] > best) best = val[p];
            nnz_d[idx[p]]++;
            if (val[p] > mw_d[idx[p]]) mw_d[idx[p]] = val[p];
        }
        mw[x] = best;
    }
}

static const int32_t *g_nnz_for_cmp;
static int cmp_dim(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    /* decreasing number of non-zeroes; ties by ascending dimension id */
    if (g_nnz_for_cmp[a] != g_nnz_for_cmp[b]) return g_nnz_for_cmp[a] > g_nnz_for_cmp[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* all-pairs-1 orders the dimensions by decreasing number of non-zeroes:
 * rank[d] = position of dimension d in that order. */
void or_dim_rank(int32_t m, const int32_t *nnz_d, int32_t *rank) {
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    for (int32_t d = 0; d < m; d++) order[d] = d;
    g_nnz_for_cmp = nnz_d;
    qsort(order, (size_t)m, sizeof(int32_t), cmp_dim);
    for (int32_t r = 0; r < m; r++) rank[order[r]] = r;
    free(order);
}

/* A row's components sorted by dimension rank (the processing order of all-pairs-1). */
typedef struct {
    int32_t rank;
    float v;
} comp_t;

static int cmp_comp(const void *pa, const void *pb) {
    const comp_t *a = (const comp_t *)pa, *b = (const comp_t *)pb;
    return a->rank < b->rank ? -1 : (a->rank > b->rank);
}

/* Rows re-expressed over ranks: crank/cval hold each row's components sorted by rank. */
void or_rank_rows(int32_t n, const int64_t *indptr, const int32_t *idx, const float *val,
                  const int32_t *rank, int32_t *crank, float *cval) {
    for (int32_t x = 0; x < n; x++) {
        int64_t a = indptr[x], k = indptr[x + 1] - a;
        comp_t *tmp = (comp_t *)malloc(sizeof(comp_t) * (size_t)(k ? k : 1));
        for (int64_t p = 0; p < k; p++) {
            tmp[p].rank = rank[idx[a + p]];
            tmp[p].v = val[a + p];
        }
        qsort(tmp, (size_t)k, sizeof(comp_t), cmp_comp);
        for (int64_t p = 0; p < k; p++) {
            crank[a + p] = tmp[p].rank;
            cval[a + p] = tmp[p].v;
        }
        free(tmp);
    }
}

/* Partial indexing (all-pairs-1): walking x's components in rank order, accumulate
 * b += x[i] * maxweight_i(V); the components seen while b < t stay unindexed as x';
 * indexing starts at the component where b reaches t. split[x] = |x'|, and
 * mw_pre[x] = maxweight(x') (0 for an empty x'). mwr is maxweight_i(V) by rank. */
void or_prefix_split(int32_t n, const int64_t *indptr, const int32_t *crank, const float *cval,
                     const float *mwr, double t, int32_t *split, float *mw_pre) {
    for (int32_t x = 0; x < n; x++) {
        double b = 0.0;
        int32_t k = 0;
        float best = 0.0f;
        int64_t len = indptr[x + 1] - indptr[x];
        while (k < len) {
            int64_t p = indptr[x] + k;
            b += (double)cval[p] * (double)mwr[crank[p]];
            if (b >= t) break;
            if (cval[p] > best) best = cval[p];
            k++;
        }
        split[x] = k;
        mw_pre[x] = best;
    }
}

/* ------------------------------------------------ sequential All-Pairs (Alg. 1-2) */

typedef struct {
    int32_t y;
    float w;
} post_t;

typedef struct {
    post_t *e;
    int64_t len, cap, front; /* entries before `front` were popped by minsize */
} list_t;

static int list_push(list_t *L, int32_t y, float w) {
    if (L->len == L->cap) {
        int64_t cap = L->cap ? 2 * L->cap : 4;
        post_t *ne = (post_t *)realloc(L->e, sizeof(post_t) * (size_t)cap);
        if (!ne) return -1;
        L->e = ne;
        L->cap = cap;
    }
    L->e[L->len].y = y;
    L->e[L->len].w = w;
    L->len++;
    return 0;
}

/* dot(x, y') of two rank-sorted component lists */
static double dot_ranked(const int32_t *ra, const float *va, int64_t na, const int32_t *rb,
                         const float *vb, int64_t nb) {
    double s = 0.0;
    int64_t p = 0, q = 0;
    while (p < na && q < nb) {
        if (ra[p] == rb[q]) {
            s += (double)va[p] * (double)vb[q];
            p++;
            q++;
        } else if (ra[p] < rb[q]) {
            p++;
        } else {
            q++;
        }
    }
    return s;
}

static const float *g_mw_for_cmp;
static int cmp_vec(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_mw_for_cmp[a] != g_mw_for_cmp[b]) return g_mw_for_cmp[a] > g_mw_for_cmp[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/*
 * All-Pairs(V, t) with the paper's optimisation toggles.
 *   flags = 0                      all-pairs-0-array (Alg. 1-2 with an array A)
 *   OR_PARTIAL_INDEX               all-pairs-1
 *   OR_PARTIAL_INDEX|MINSIZE|REMSCORE|UPPERBOUND   all-pairs-2
 * and any other subset (the variants of Sec. 4).
 *
 * query_mask (may be NULL): when given, Find-Matches runs only for vectors with a
 * non-zero mask entry; every vector is still indexed. Used to time a bounded sample.
 *
 * counters[0] = multiplications in the accumulation loop (A[y] += x[i]*y[i]),
 * counters[1] = candidates (y with A[y] != 0 after accumulation),
 * counters[2] = dot(x, y') evaluations performed, counters[3] = matches,
 * counters[4] = similarity evaluations decided (sum over matched x of #earlier vectors).
 * Returns the number of matches, or -1 on allocation failure.
 */
int64_t or_all_pairs(int32_t n, int32_t m, const int64_t *indptr, const int32_t *idx,
                     const float *val, double t, uint32_t flags, const uint8_t *query_mask,
                     or_result *out, int64_t *counters) {
    const int partial = (flags & OR_PARTIAL_INDEX) != 0;
    const int minsize = (flags & OR_MINSIZE) != 0;
    const int remscore = (flags & (OR_REMSCORE | OR_REMSCORE_FORWARD)) != 0;
    const int forward = (flags & OR_REMSCORE_FORWARD) != 0;
    const int upperbound = (flags & OR_UPPERBOUND) != 0;
    int64_t nnz = indptr[n];
    int64_t ret = -1;
    for (int k = 0; k < 5; k++) counters[k] = 0;

    int32_t *len = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    float *mw = (float *)malloc(sizeof(float) * (size_t)(n + 1));
    int32_t *nnz_d = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    float *mw_d = (float *)malloc(sizeof(float) * (size_t)(m + 1));
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    float *mwr = (float *)malloc(sizeof(float) * (size_t)(m + 1));
    int32_t *crank = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    float *cval = (float *)malloc(sizeof(float) * (size_t)(nnz + 1));
    int32_t *split = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    float *mw_pre = (float *)calloc((size_t)(n + 1), sizeof(float));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    double *A = (double *)calloc((size_t)(n + 1), sizeof(double));
    list_t *I = (list_t *)calloc((size_t)(m + 1), sizeof(list_t));
    if (!len || !mw || !nnz_d || !mw_d || !rank || !mwr || !crank || !cval || !split ||
        !mw_pre || !order || !pos || !A || !I)
        goto done;

    /* preprocessing: maxweight_i(V), maxweight(x), |x|, dimension order */
    or_stats(n, m, indptr, idx, val, len, mw, nnz_d, mw_d);
    or_dim_rank(m, nnz_d, rank);
    for (int32_t d = 0; d < m; d++) mwr[rank[d]] = mw_d[d];
    or_rank_rows(n, indptr, idx, val, rank, crank, cval);

    /* vector processing order (minsize needs decreasing maxweight(x)) */
    for (int32_t x = 0; x < n; x++) order[x] = x;
    if (minsize) {
        g_mw_for_cmp = mw;
        qsort(order, (size_t)n, sizeof(int32_t), cmp_vec);
    }
    for (int32_t k = 0; k < n; k++) pos[order[k]] = k;

    for (int32_t k = 0; k < n; k++) {
        const int32_t x = order[k];
        const int64_t xa = indptr[x];
        const int32_t xl = len[x];

        /* Find-Matches(x, I, t) -- Alg. 2 plus the all-pairs-2 bounds */
        if (!query_mask || query_mask[x]) {
            counters[4] += k;
            double rem = 0.0;
            if (remscore)
                for (int32_t c = 0; c < xl; c++) rem += (double)cval[xa + c] * (double)mwr[crank[xa + c]];
            const double mins = minsize ? t / (double)mw[x] : 0.0;
            for (int32_t step = 0; step < xl; step++) {
                /* with remscore: sparsest dimension first, unless the planted mistake */
                const int32_t c = (remscore && !forward) ? xl - 1 - step : step;
                const int32_t r = crank[xa + c];
                const double xv = (double)cval[xa + c];
                list_t *L = &I[r];
                if (minsize) /* pop vectors smaller than minsize from the list front */
                    while (L->front < L->len && (double)len[L->e[L->front].y] < mins) L->front++;
                for (int64_t e = L->front; e < L->len; e++) {
                    const int32_t y = L->e[e].y;
                    if (!remscore || A[y] != 0.0 || rem >= t) {
                        A[y] += xv * (double)L->e[e].w;
                        counters[0]++;
                    }
                }
                if (remscore) rem -= xv * (double)mwr[r];
            }
            /* candidates: every y with a non-zero score in A (all-pairs-0-array) */
            for (int32_t y = 0; y < n; y++) {
                if (A[y] == 0.0) continue;
                counters[1]++;
                const int64_t ya = indptr[y];
                if (upperbound) {
                    const int32_t lp = split[y];
                    const double bound = A[y] + (double)(lp < xl ? lp : xl) * (double)mw[x] *
                                                    (double)mw_pre[y];
                    if (bound < t) continue;
                }
                double s = A[y];
                if (split[y] > 0) {
                    s += dot_ranked(crank + xa, cval + xa, xl, crank + ya, cval + ya, split[y]);
                    counters[2]++;
                }
                if (s >= t) {
                    if (push(out, x, y, s)) goto done;
                    counters[3]++;
                }
            }
            memset(A, 0, sizeof(double) * (size_t)n); /* zero the whole array */
        }

        /* index x: I_i <- I_i + (x, x[i]) (Alg. 1), only from the point where the partial
         * bound b reaches t when partial indexing is on (all-pairs-1) */
        {
            double b = 0.0;
            int32_t c0 = 0;
            float best = 0.0f;
            if (partial) {
                while (c0 < xl) {
                    b += (double)cval[xa + c0] * (double)mwr[crank[xa + c0]];
                    if (b >= t) break;
                    if (cval[xa + c0] > best) best = cval[xa + c0];
                    c0++;
                }
            }
            split[x] = c0;
            mw_pre[x] = best;
            for (int32_t c = c0; c < xl; c++)
                if (list_push(&I[crank[xa + c]], x, cval[xa + c])) goto done;
        }
    }
    ret = out->n;

done:
    if (I)
        for (int32_t d = 0; d < m; d++) free(I[d].e);
    free(I);
    free(A);
    free(pos);
    free(order);
    free(mw_pre);
    free(split);
    free(cval);
    free(crank);
    free(mwr);
    free(rank);
    free(mw_d);
    free(nnz_d);
    free(mw);
    free(len);
    return ret;
}
