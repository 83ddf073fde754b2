/*
 * aps.h -- C ABI of the GB300 All-Pairs similarity join library (libaps.so).
 *
 * The library finds every pair of unit-norm, non-negative sparse vectors whose inner
 * product reaches a threshold t (Ozkural & Aykanat, Sec. 2.1: M = {(v_i, v_j) : i != j,
 * dot(v_i, v_j) >= t}), with the inverted-index All-Pairs method of Sec. 3.2.2
 * (Alg. 1-2 plus partial indexing, minsize, remscore and upperbound), and a dense
 * variant for embeddings (the matrix view S = D.D^T of Sec. 2.1) on tensor cores.
 *
 * Conventions for every entry point:
 *   - Plain C types only; no exception crosses the ABI. Every call returns an
 *     aps_status; on failure aps_last_error() gives a message (thread-local).
 *   - Input pointers are borrowed for the duration of the call only. Unless the
 *     APS_DEVICE_PTRS flag is given they are host pointers; with it they must be
 *     device pointers on the current CUDA device.
 *   - Objects returned through out-parameters (aps_index, aps_pairs buffers,
 *     aps_server) are owned by the library and released with the matching *_free.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls are synchronous with respect to the host: when they return, results are
 *     complete (device results are written on `stream`).
 *   - Vector ids in results are the caller's row numbers. Pairs of a self-join are
 *     unordered and reported once as (i < j), sorted by (i, j).
 *   - Scores are float32 within 1e-5 of the float64 dot product of the float32 inputs.
 *     Pairs whose float32 score lies within a band of t (at least 1e-5 wide) are
 *     decided by a float64 re-evaluation, so the pair set equals the float64 one.
 */
#ifndef APS_H
#define APS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aps_status {
    APS_OK = 0,
    APS_EINVAL = 1,       /* invalid argument or malformed input */
    APS_ENOMEM = 2,       /* device or host allocation failed */
    APS_ECUDA = 3,        /* a CUDA call failed */
    APS_EOVERFLOW = 4,    /* a caller-sized buffer is too small; count holds the need */
    APS_EAGAIN = 5,       /* serving: request not finished yet */
    APS_ETIMEOUT = 6,     /* a bounded device or host wait ran out */
    APS_ECANCELED = 7,    /* serving: request cancelled or expired */
    APS_EUNSUPPORTED = 8  /* device or configuration not supported */
} aps_status;

/* ---- flags ---------------------------------------------------------------------- */
#define APS_DEVICE_PTRS 0x1u      /* input arrays are device pointers */
#define APS_NORMALIZE 0x2u        /* L2-normalise rows (float64 norm) instead of checking */
#define APS_QUERYABLE 0x4u        /* index prefixes split on ||y'||_2 < t so that vectors
                                     outside the set may query the index (aps_query) */
#define APS_NO_PARTIAL_INDEX 0x8u /* ablation: index every component (all-pairs-0-array) */
#define APS_NO_MINSIZE 0x10u      /* ablation: no minsize pruning */
#define APS_NO_REMSCORE 0x20u     /* ablation: no remscore admission bound */
#define APS_NO_UPPERBOUND 0x40u   /* ablation: no upperbound before dot(x, y') */
#define APS_HOST_OUTPUT 0x100u    /* results are copied to pinned host memory */
#define APS_SUBUNIT_NORMS 0x200u  /* rows may have L2 norm below 1 (at most 1 + 1e-3), e.g. the
                                     projection of unit vectors onto a block of dimensions; every
                                     pruning bound of the join holds for such rows */

/* The paper's sequential variants (Sec. 4; timed in Tables 2-3 of Sec. 7.3) as flag sets
 * for aps_build_index. The candidate map is always a dense array here, so each is the
 * paper's "-array" form; all-pairs-2 (every bound on) is the default. NO_UPPERBOUND also
 * turns off the ||y'||_2 pre-filter, the other bound that skips dot(x, y'). Every variant
 * returns the same pairs; they differ in work. */
#define APS_VARIANT_ALL_PAIRS_0 (APS_NO_PARTIAL_INDEX | APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_0_REMSCORE (APS_NO_PARTIAL_INDEX | APS_NO_MINSIZE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_0_MINSIZE (APS_NO_PARTIAL_INDEX | APS_NO_REMSCORE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_1 (APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_1_REMSCORE (APS_NO_MINSIZE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_1_UPPERBOUND (APS_NO_MINSIZE | APS_NO_REMSCORE)
#define APS_VARIANT_ALL_PAIRS_1_MINSIZE (APS_NO_REMSCORE | APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_1_REMSCORE_MINSIZE (APS_NO_UPPERBOUND)
#define APS_VARIANT_ALL_PAIRS_2 0u

/* ---- results -------------------------------------------------------------------- */
typedef struct aps_pairs {
    int64_t count;   /* number of pairs */
    int32_t *i;      /* [count] first vector id (self-join: i < j; query: query row) */
    int32_t *j;      /* [count] second vector id */
    float *score;    /* [count] float32 score */
    int32_t on_device; /* 1: the three arrays are device pointers; 0: pinned host memory */
    int32_t _reserved;
    void *_priv;     /* library bookkeeping; do not touch */
} aps_pairs;

/* The similarity graph G_S(V, t) = (V, M) of Sec. 2.1 (edge u <-> v for every match,
 * weight w(u, v) = u.v) as a CSR adjacency. */
typedef struct aps_graph {
    int32_t n;         /* vertices */
    int32_t on_device; /* 1: the arrays are device pointers; 0: pinned host memory */
    int64_t nnz;       /* adjacency entries = 2 x pairs */
    int64_t *row_ptr;  /* [n + 1] row v is col[row_ptr[v] .. row_ptr[v + 1]) */
    int32_t *col;      /* [nnz] neighbours of each vertex, in increasing id */
    float *w;          /* [nnz] edge weights (the pairs' scores) */
    void *_priv;       /* library bookkeeping; do not touch */
} aps_graph;

/* Work counters and phase times of the last aps_all_pairs / aps_query / batch call on
 * an index (all counts are exact; times are CUDA-event milliseconds). */
typedef struct aps_stats {
    int64_t visits;       /* posting-list entries Alg. 2 adds: on x's lists, y after x (self-join),
                             |y| >= minsize when minsize is on */
    int64_t candidates;   /* (x, y) pairs with a non-zero partial score */
    int64_t verified;     /* candidates that passed upperbound and got dot(x, y') */
    int64_t pairs;        /* pairs emitted */
    int64_t band;         /* pairs re-decided in float64 */
    int64_t evaluations;  /* similarity evaluations decided: sum over instances n(n-1)/2 */
    int64_t reruns;       /* join re-runs after the output staging buffer grew */
    float ms_build;       /* index build (aps_build_index / batch) */
    float ms_join;        /* join kernel launches only (last attempt) */
    float ms_sort;        /* output stage: count scan + gather into (i, j) order */
    float ms_total;       /* whole call */
    int64_t entries_read; /* posting-list entries loaded by the join (visits plus the entries it
                             reads and skips: minsize, and ids at or before x in x's first window) */
} aps_stats;

typedef struct aps_index aps_index;

/*
 * Build the inverted index of n sparse vectors over m dimensions for threshold t
 * (steps of Alg. 1 plus the all-pairs-1/2 preprocessing of Sec. 3.2.2):
 *   - per-vector |x| and maxweight(x), per-dimension non-zero counts and maxweight_i(V);
 *   - dimensions ranked by decreasing non-zero count (ties: ascending id);
 *   - each vector's components re-ordered by that rank;
 *   - partial indexing: the leading components whose bound
 *     b = sum x[i] * maxweight_i(V) stays below t are kept unindexed (x'), the rest go
 *     into the posting lists (with APS_QUERYABLE the bound is ||x'||_2 instead);
 *   - posting lists I_d of (vector id, weight).
 * Input: CSR with int64 indptr[n+1] (indptr[0] = 0), int32 idx[nnz] strictly increasing
 * within each row and in [0, m), float32 val[nnz] finite and > 0. Each row must have
 * L2 norm within 1e-3 of 1 unless APS_NORMALIZE is given. Empty rows are legal (they
 * match nothing). 0 < t <= 1. n >= 0, m >= 1, nnz < 2^31.
 * Errors: APS_EINVAL (message names the first offending row), APS_ENOMEM, APS_ECUDA.
 */
aps_status aps_build_index(const int64_t *indptr, const int32_t *idx, const float *val,
                           int32_t n, int32_t m, float t, uint32_t flags, void *stream,
                           aps_index **out);

/* Self-join of the indexed set at the build threshold: every pair (i < j) with
 * dot >= t (Alg. 1-2 with the all-pairs-2 bounds), sorted by (i, j).
 * flags: APS_NO_MINSIZE / APS_NO_REMSCORE / APS_NO_UPPERBOUND ablations and
 * APS_HOST_OUTPUT. Result buffers are allocated by the library; free with aps_pairs_free.
 * The first call on an index captures its join phase as a CUDA graph that later calls
 * replay; calls on one index must not overlap each other (aps_query may run meanwhile).
 * Errors: APS_EINVAL (NULL arguments or a batched index), APS_ENOMEM, APS_ECUDA,
 * APS_EOVERFLOW (the staging still overflowed after growing twice); *out is then empty. */
aps_status aps_all_pairs(aps_index *index, uint32_t flags, aps_pairs *out);

/* The self-join of aps_all_pairs with the vertical algorithm's local pruning inside the
 * join (Sec. 5.1: Par-All-Pairs-0-Vert, Lemma 1, local threshold t/p). The `heavy`
 * costliest vectors of the index (the front of its cost-ordered work list; all of them when
 * heavy exceeds the count) are each joined as nblk dimension blocks, on different CTAs: a
 * block walks every nblk-th of the vector's creating components (those remscore lets
 * create candidates) and all of its updating ones. A match scores A + dot(x, y') >= t and
 * the blocks that created y hold all of A between them, so one block has A_b >=
 * (t - ||y'||_2) / nblk; a block keeps y only then (local pruning), decides the kept
 * candidates by their float64 dot product over all of y, and the blocks' pairs are merged
 * (sorted, duplicates dropped) into the vectors' output runs. The result equals
 * aps_all_pairs' (i < j, sorted by (i, j)); only the work distribution differs.
 * 2 <= nblk <= 8, heavy >= 0 (0: the plain join). Errors: APS_EINVAL (NULL arguments, a
 * batched index, nblk or heavy out of range), APS_ENOMEM, APS_ECUDA, APS_EOVERFLOW. */
aps_status aps_all_pairs_split(aps_index *index, int32_t nblk, int64_t heavy, uint32_t flags,
                               aps_pairs *out);

/* Match nq external query vectors (CSR as in aps_build_index) against the index
 * (the local matching step of the horizontal algorithm, Alg. 6): every (q, y) with
 * dot(q, y) >= t, as i = query row, j = vector id, sorted by (i, j). The index must
 * have been built with APS_QUERYABLE, and t >= the build threshold.
 * Errors: APS_EINVAL (NULL arguments, an index not single-instance or not built with
 * APS_QUERYABLE, t outside [build threshold, 1], malformed query rows), APS_ENOMEM,
 * APS_ECUDA, APS_EOVERFLOW; *out is then empty. */
aps_status aps_query(aps_index *index, const int64_t *qptr, const int32_t *qidx,
                     const float *qval, int32_t nq, float t, uint32_t flags, aps_pairs *out);

/* Read back the index build results for verification of each step. Any pointer may be
 * NULL. Host arrays, caller-allocated, sizes: len/mw/split/qsplit/mw_pre [n],
 * rank_of_dim/nnz_d/mw_d [m], crank/cval [nnz] (components re-ordered by rank, the
 * CSR row pointers are the input's), list_ptr [m+1] (by rank), post_id/post_w [list_ptr[m]].
 * Errors: APS_EINVAL (NULL index), APS_ECUDA. */
aps_status aps_index_export(const aps_index *index, int32_t *len, float *mw, int32_t *nnz_d,
                            float *mw_d, int32_t *rank_of_dim, int32_t *crank, float *cval,
                            int32_t *split, int32_t *qsplit, float *mw_pre, int64_t *list_ptr,
                            int32_t *post_id, float *post_w);

/* Sizes of the index: n, m, nnz and the number of indexed components (any pointer may
 * be NULL). Errors: APS_EINVAL (NULL index). */
aps_status aps_index_info(const aps_index *index, int32_t *n, int32_t *m, int64_t *nnz,
                          int64_t *indexed);

/* Self-join of a single-instance index, as aps_all_pairs, without allocating memory.
 * The paper has no counterpart: this exists for callers that cannot allocate device
 * memory while they join -- a process whose memory is reserved up front by its own
 * allocator, or a latency-critical thread that must not take the allocator's locks or
 * trigger the implicit synchronisation an allocation can cause. The caller owns the
 * device arrays i, j, score (capacity pairs each); on APS_OK *count pairs sorted by
 * (i, j) are in them. All scratch comes from one fixed 64 MiB device array inside the
 * library (held by every GPU that loads this part of the library until exit) and the
 * join uses at most 32 CTAs. Limits: the index's (vector, window) slots must fit the
 * arena with room left to stage pairs (else APS_EINVAL, before any work), and the pairs
 * must fit both the staging room and `capacity` (else APS_EOVERFLOW with *count = the
 * number of pairs). The current device must be the index's device, and i, j and score
 * must be device memory of that device (else APS_EINVAL). The first call on a device
 * looks up the array's device address (once per device, with that device current).
 * Every call reads its counters back and synchronizes `stream` before it returns, so it
 * must not be called while `stream` (or the legacy default stream it may wait on) is
 * being captured into a CUDA graph. Every call shares the one array and keeps no state in
 * it between calls, but calls that overlap on the GPU (other streams, other host threads)
 * race on it: run them one at a time per device. The index's stats (aps_index_stats)
 * then report this join's counters, with zero timings. Calls no cudaMalloc/cudaFree or
 * allocating routine. */
aps_status aps_all_pairs_noalloc(aps_index *index, int32_t *i, int32_t *j, float *score,
                                 int64_t capacity, int64_t *count, void *stream);

/* Counters and timings of the last join or query batch on this index (see aps_stats).
 * Errors: APS_EINVAL (NULL index or out). */
aps_status aps_index_stats(const aps_index *index, aps_stats *out);

void aps_index_free(aps_index *index);

/* Release the buffers of a result (device or host). Safe on a zeroed aps_pairs. */
void aps_pairs_free(aps_pairs *pairs);

/* Copy a result's arrays into caller-owned buffers (host or device; any may be NULL) on
 * `stream`, and wait for the copies. Errors: APS_EINVAL (NULL pairs), APS_ECUDA. */
aps_status aps_pairs_copy_to(const aps_pairs *pairs, int32_t *i, int32_t *j, float *score,
                             void *stream);

/* ---- batched form --------------------------------------------------------------- */
typedef struct aps_instance {
    const int64_t *indptr; /* CSR of one instance, as in aps_build_index */
    const int32_t *idx;
    const float *val;
    int32_t n, m;
    float t;
    int32_t _reserved;
} aps_instance;

/* Self-join of k independent instances in one pass: all instances are indexed by one
 * set of kernels and joined by one persistent launch (the size classes in turn, tile
 * shapes from the table of aps_set_tuning / aps_autotune_batch_csr). outs[k] receives
 * instance k's pairs (i < j, local row ids, sorted); all k results share one allocation,
 * released by calling aps_pairs_free on every element. stats (may be NULL) gets the
 * totals. Errors: APS_EINVAL (k < 1, NULL arrays, an instance with n < 0, m < 1, t
 * outside (0, 1] or malformed rows), APS_ENOMEM, APS_ECUDA, APS_EOVERFLOW; every
 * outs[r] is then empty. */
aps_status aps_batch_all_pairs(int32_t k, const aps_instance *inst, uint32_t flags,
                               void *stream, aps_pairs *outs, aps_stats *stats);

/* The batched self-join over one concatenated CSR: instance r owns rows
 * [row_offsets[r], row_offsets[r+1]) (host array of k+1 entries, row_offsets[0] = 0);
 * indptr (row_offsets[k]+1 entries, global: indptr[0] = 0), idx, val as in
 * aps_build_index (device pointers with APS_DEVICE_PTRS, dimension ids local to each
 * instance, in [0, m[r])); m and t are host arrays of k entries. Results and ownership as
 * in aps_batch_all_pairs. Avoids per-instance copies when the batch is device-resident.
 * Errors as aps_batch_all_pairs (also row_offsets[0] != 0). */
aps_status aps_batch_all_pairs_csr(int32_t k, const int64_t *row_offsets, const int64_t *indptr,
                                   const int32_t *idx, const float *val, const int32_t *m,
                                   const float *t, uint32_t flags, void *stream, aps_pairs *outs,
                                   aps_stats *stats);

/* ---- join tile shapes and the autotuner ------------------------------------------ */
/* The join's tile shape for an instance of n vectors: G query groups per CTA (1, 2, 4 or
 * 8), each with a candidate window of 40960 / G ids in shared memory (the blocks of
 * Sec. 5.1.9 as CTA-level tiles). G is looked up by the instance's size bucket: bucket b
 * holds 1 + the previous bound <= n <= APS_TUNE_BOUND_b, with bounds 512, 1280, 2560,
 * 5120, 10240, 20480, 40960 and unbounded (aps_tune_bucket). The bucket bounds are the
 * work-split thresholds; the table is process-wide and read by every later index build
 * (aps_build_index and the batched calls). */
#define APS_TUNE_BUCKETS 8

typedef struct aps_tuning {
    int32_t groups[APS_TUNE_BUCKETS];       /* G per size bucket: 1, 2, 4 or 8 */
    int32_t query_groups[APS_TUNE_BUCKETS]; /* G for indexes built with APS_QUERYABLE */
} aps_tuning;

typedef struct aps_tune_report {
    int32_t instances[APS_TUNE_BUCKETS]; /* instances of the batch per bucket */
    int32_t sampled[APS_TUNE_BUCKETS];   /* of those, in the timed sample */
    float ms[APS_TUNE_BUCKETS][4];       /* sample join ms with G = 1, 2, 4, 8 (-1: not run) */
    float ms_default;                    /* whole-batch join ms with the default table */
    float ms_tuned;                      /* whole-batch join ms with the chosen table */
    int32_t kept_default;                /* 1: the measured table was not faster overall */
    int32_t _reserved;
} aps_tune_report;

/* The size bucket (0 .. APS_TUNE_BUCKETS-1) of an instance of n vectors. */
int32_t aps_tune_bucket(int64_t n);
/* The built-in table, the same in both columns: G = 8 up to 5120 vectors (one window),
 * 4 up to 10240, 2 above. (This and aps_get_tuning ignore a NULL out.) */
void aps_tuning_default(aps_tuning *out);
/* The table in force for this process. */
void aps_get_tuning(aps_tuning *out);
/* Replace the table in force (APS_EINVAL unless every entry of both columns is 1, 2, 4
 * or 8). Affects index builds that start afterwards; built indexes keep their shapes. */
aps_status aps_set_tuning(const aps_tuning *tuning);
/* Autotuner for a batch given as in aps_batch_all_pairs_csr. For each size bucket the
 * batch populates, a sample of its instances (whole instances, at most 2^18 vectors,
 * spread over the bucket) is indexed with each G in {1, 2, 4, 8} and joined three times;
 * the bucket takes the G with the least join time (the current entry unless another is
 * at least 2% faster). The chosen table is then timed against the default on the whole
 * batch (two joins each) and kept only if faster; the queryable column is left as it
 * is. The winner is installed
 * (aps_set_tuning) and returned in *out; *report (may be NULL) gets the measurements.
 * APS_QUERYABLE and APS_HOST_OUTPUT in flags are ignored (the self-join column is tuned).
 * Results of the batch do not depend on the table; only the join time does.
 * Errors: APS_EINVAL (arguments or rows, as aps_batch_all_pairs_csr), APS_ENOMEM,
 * APS_ECUDA; on any error the table in force is left unchanged. */
aps_status aps_autotune_batch_csr(int32_t k, const int64_t *row_offsets, const int64_t *indptr,
                                  const int32_t *idx, const float *val, const int32_t *m,
                                  const float *t, uint32_t flags, void *stream, aps_tuning *out,
                                  aps_tune_report *report);

/* ---- dense embeddings ----------------------------------------------------------- */
/* All pairs (i < j) of n unit vectors X[n, d] (float32, row-major) with X_i . X_j >= t:
 * the S = D.D^T view of Sec. 2.1 computed as a BF16 tensor-core product with float32
 * accumulation, a provable margin delta below t for candidates, float32 rescoring of
 * the candidates from X, float64 inside the band, sorted by (i, j). d must be a
 * multiple of 64 and at most 512. Needs an sm_103a device.
 * Errors: APS_EINVAL (d not a multiple of 64 in [64, 512], t outside (0, 1], a row whose
 * norm is off by more than 1e-3 without APS_NORMALIZE, a zero or non-finite row),
 * APS_EUNSUPPORTED (no sm_103 device, or no tensor-map encoder in the driver),
 * APS_ETIMEOUT (a pipeline wait of the tensor-core kernel ran out; the context stays
 * usable), APS_ENOMEM, APS_ECUDA; *out is then empty. */
aps_status aps_all_pairs_dense(const float *X, int32_t n, int32_t d, float t, uint32_t flags,
                               void *stream, aps_pairs *out, aps_stats *stats);
/* Measurement of the dense path's arithmetic: the float32 products S_ij = X_bf16,i . X_bf16,j
 * exactly as aps_all_pairs_dense's tensor-core kernel accumulates them (X rounded to BF16,
 * products summed in float32 in the tensor memory), written to raw[i * n + j] for every
 * computed entry: the 256-row blocks on and above the block diagonal (j's block >= i's
 * block); other entries are left as they were. X (n x d float32, row-major, 16-byte
 * aligned) and raw (n * n float32) are device pointers owned by the caller; rows are taken
 * as they are (no norm check). d as in aps_all_pairs_dense; n <= 16384. Synchronizes
 * stream. Errors: APS_EINVAL, APS_EUNSUPPORTED, APS_ETIMEOUT, APS_ENOMEM, APS_ECUDA. */
aps_status aps_dense_tensor_products(const float *X, int32_t n, int32_t d, float *raw, void *stream);

/* ---- the similarity graph -------------------------------------------------------- */
/* CSR adjacency of G_S (Sec. 2.1) from a pair list: each pair (i[p], j[p], s[p]) gives the
 * entries i -> j and j -> i of weight s[p]. The pairs must satisfy 0 <= i < j < n and be
 * strictly increasing in (i, j), the order aps_all_pairs returns (so a result's arrays
 * can be passed straight in with APS_DEVICE_PTRS when it is on the device); they are
 * host pointers without that flag. APS_HOST_OUTPUT copies the graph to pinned host
 * memory. Each row lists its neighbours in increasing id. count < 2^32.
 * Errors: APS_EINVAL for a pair out of range, out of order or repeated (nothing is
 * allocated then); APS_ENOMEM. Free with aps_graph_free. stream: cudaStream_t or NULL. */
aps_status aps_graph_csr(const int32_t *i, const int32_t *j, const float *s, int64_t count, int32_t n,
                         uint32_t flags, void *stream, aps_graph *out);
/* The k nearest neighbours of every vertex read off a device graph (the k-nn use of the
 * similarity graph, Sec. 2.2): row v of nbr[n * k] / wk[n * k] holds v's neighbours of
 * largest weight, ties by smaller id, in that order; rows with fewer than k neighbours
 * end in id -1, weight 0. nbr and wk are caller buffers, device pointers with
 * APS_DEVICE_PTRS and host pointers otherwise. 1 <= k <= 256.
 * Errors: APS_EINVAL (not a device graph from aps_graph_csr, k out of range, NULL
 * outputs), APS_ENOMEM, APS_ECUDA. */
aps_status aps_graph_knn(const aps_graph *g, int32_t k, int32_t *nbr, float *wk, uint32_t flags,
                         void *stream);
/* Copy a graph's arrays (device or host) into caller buffers of n + 1 / nnz / nnz
 * elements (any of them may be NULL). Synchronous. Errors: APS_EINVAL (a graph not from
 * aps_graph_csr), APS_ECUDA. */
aps_status aps_graph_copy_to(const aps_graph *g, int64_t *row_ptr, int32_t *col, float *w, void *stream);
void aps_graph_free(aps_graph *g);

/* ---- exact verification of candidate pairs --------------------------------------- */
/* The score merge of the vertical algorithm with local pruning (Sec. 5.1, Lemma 1 and
 * Eq. 2: a match has a partial score >= t/p on at least one of p dimension blocks): the
 * union of k candidate lists `lists[0..k)` (pairs i < j of the same n vectors, device or
 * host results, any order, duplicates allowed) is deduplicated, each pair's dot product is
 * recomputed in float64 from the rows of the CSR (indptr/idx/val as for aps_build_index,
 * device pointers with APS_DEVICE_PTRS; each row's ids strictly increasing), and the pairs
 * with dot >= t are returned in (i, j) order with float32 scores (free with aps_pairs_free).
 * *n_candidates (may be NULL) receives the size of the union. APS_HOST_OUTPUT as for
 * aps_all_pairs. Errors: APS_EINVAL for a pair outside 0 <= i < j < n or a malformed row. */
aps_status aps_pairs_verify(const aps_pairs *lists, int32_t k, const int64_t *indptr, const int32_t *idx,
                            const float *val, int32_t n, int32_t m, float t, uint32_t flags, void *stream,
                            aps_pairs *out, int64_t *n_candidates);

/* ---- serving -------------------------------------------------------------------- */
typedef struct aps_server aps_server;

typedef struct aps_query_req {
    const int64_t *qptr; /* host CSR of a query batch (copied at submit) */
    const int32_t *qidx;
    const float *qval;
    int32_t nq;
    float t;             /* >= the index build threshold */
} aps_query_req;

/* A request loop over a device-resident APS_QUERYABLE index. Submitted query batches
 * are admitted in arrival order when one of `slots` execution slots is free and their
 * estimated device footprint fits in mem_budget bytes; admitted batches run
 * concurrently on separate streams (continuous batching). The server borrows the index
 * until aps_server_free. Errors: APS_EINVAL (NULL arguments, slots outside [1, 64], an
 * index not single-instance or not built with APS_QUERYABLE), APS_ECUDA. */
aps_status aps_server_create(aps_index *index, size_t mem_budget, int32_t slots,
                             aps_server **out);
/* Queue a query batch; its rows are copied, so the request's arrays may be reused on
 * return. *ticket identifies it for poll and cancel. Errors: APS_EINVAL (NULL
 * arguments, malformed rows, t outside [build threshold, 1]). */
aps_status aps_stream_submit(aps_server *server, const aps_query_req *req, uint64_t *ticket);
/* Wait up to timeout_us (0 = just check) for a ticket. APS_EAGAIN if not done yet; on
 * APS_OK `out` receives the pairs (host memory) and the ticket is retired. Errors:
 * APS_EINVAL (NULL arguments, an unknown or retired ticket), APS_ECANCELED (cancelled;
 * the ticket is retired), or the batch's own error status (the ticket is retired). */
aps_status aps_stream_poll(aps_server *server, uint64_t ticket, int32_t timeout_us,
                           aps_pairs *out);
/* Cancel a ticket: a queued batch never runs, a running one completes and its result is
 * dropped; the next poll returns APS_ECANCELED. Errors: APS_EINVAL (NULL server, an
 * unknown ticket). */
aps_status aps_stream_cancel(aps_server *server, uint64_t ticket);
/* The device time line of a server's completed batches (continuous batching, Alg. 6's
 * matching step run for several query batches at once). Each batch's device work -- its
 * query upload, preparation, join and result download on its slot's stream -- lies between
 * two CUDA events; busy_ms is the device time with at least one batch in flight,
 * overlap_ms the time with two or more (admitted batches running side by side), span_ms
 * from the first batch's start to the last one's end, max_in_flight the most batches in
 * flight at once. Errors: APS_EINVAL (NULL arguments). */
typedef struct aps_timeline {
    int64_t batches;       /* completed batches (failed ones are not counted) */
    double busy_ms;
    double overlap_ms;
    double span_ms;
    int32_t max_in_flight;
    int32_t _reserved;
} aps_timeline;
aps_status aps_server_timeline(aps_server *server, aps_timeline *out);
void aps_server_free(aps_server *server);

/* ---- misc ----------------------------------------------------------------------- */
/* The message of this thread's last failed call (empty if none). */
const char *aps_last_error(void);
const char *aps_version(void);

/* Number of CUDA kernels this library has launched in this process (all devices). */
int64_t aps_launch_count(void);

/* Test hook: make the k-th next device allocation of the library fail with APS_ENOMEM
 * (k >= 1; 0 disables). Host-side only; no GPU fault is involved. */
void aps_debug_fail_alloc(int64_t k);

/* Test hook for the bounded waits of the dense tensor-core kernel: in the next `launches`
 * launches (0 disables) the MMA issuer waits for an accumulator release that never comes,
 * so the pipeline waits run out after wait_ns nanoseconds (0 = the default limit, 2 s).
 * The kernel then lets its MMAs and TMA copies settle, frees its tensor memory and
 * returns; aps_all_pairs_dense reports APS_ETIMEOUT and the context stays usable. No GPU
 * fault is involved. */
void aps_debug_dense_stall(int64_t launches, uint64_t wait_ns);

/* Test hook for the self-join's output staging: the next aps_all_pairs (or batched join)
 * starts with room for `pairs` staged pairs instead of its estimate (0 disables), so a
 * small value makes it overflow, grow the buffer and run the join again (stats.reruns).
 * Host-side only; the kernel never writes past the room it was given. */
void aps_debug_stage_cap(int64_t pairs);

#ifdef __cplusplus
}
#endif

#endif /* APS_H */
