// Device-resident inverted index (Alg. 1's I plus the all-pairs-1/2 per-vector data).
//
// Layout in HBM (N vectors over all instances, M = sum of instance dimension counts):
//   cptr[N+1]   row pointers (the caller's CSR row pointers, concatenated)
//   crank/cval  each row's components, re-ordered by dimension rank (rank local to the
//               instance; ranks sort dimensions by decreasing non-zero count)
//   len, mw, split, qsplit, mwpre [N]   |x|, maxweight(x), |x'| (unindexed prefix),
//               remscore boundary, maxweight(x')
//   mwr/nnzr[M] maxweight_i(V) and non-zero count by global rank
//   lptr[M+1]   posting-list start by global rank
//   crow[nnz]   the same rows interleaved as {int32 rank, float32 value} (8 bytes)
//   vmeta[N]    {int32 row offset, int32 |x|, int32 |x'|, float32 maxweight(x')} (16 bytes)
//   pnorm[N]    an upper bound of ||x'||_2 (with the 1e-3 norm tolerance of the queries):
//               dot(q, x') <= ||x'||_2 for any unit q
//   vcand[N]    what verification reads of a candidate y, in one 16-byte load: {int32 row
//               offset, int32 |y'|, float32 maxweight(y'), float32 ||y'||_2 bound}
//   pn4[]       ||y'||_2 rounded up to a 4-bit code (c * 1.01/15 >= ||y'||_2), eight codes
//               per 32-bit word, each instance from a 16-byte boundary (word pbase): the join
//               copies a window's codes into shared memory and rejects candidates with them
//   post[]      posting entries {int32 local vector id | min(|y|, 255) << 24, float32
//               weight} (8 bytes), in increasing id inside each list; the size class in
//               the top byte lets minsize skip an entry without another load (instances
//               with n >= 2^24 store the id only and skip no entry)
//   wptr[]      offsets of each candidate window (ids [w*W, (w+1)*W)) inside each list,
//               only for instances with > 1 window
#pragma once

#include <atomic>
#include <mutex>

#include "aps_internal.cuh"

namespace aps {

constexpr int JOIN_THREADS = 1024;
constexpr int JOIN_WMAX = 40960;  // accumulator slots of a whole CTA (160 KB)
constexpr int JOIN_RMAX = 1536;   // dense rank table for dot(x, y') lookups (6 KB)
constexpr int JOIN_XCAP = 1280;   // x's row kept in shared memory when |x| <= XCAP / G
// (so that every class layout of a CTA plus the join kernel's 1.5 KB of per-warp counters
// fits the 227 KB of shared memory a CTA can have)
// per-warp list of emitted pairs of one window: a warp scans at most W/NW slots rounded
// up to 128 (W/NW = 1280 for every group shape)
constexpr int JOIN_ECAP = JOIN_WMAX / (JOIN_THREADS / 32) + 128;
constexpr int JOIN_STAGE_SLAB = 4096;  // staging slots a query group reserves at a time
constexpr int JOIN_NCLS = 5;           // work-list classes: G = 1, 2, 4, 8 groups per CTA; vectors of <= 2 components
// ||y'||_2 bounds in 4 bits per vector: code c stands for c * PN4_STEP (PN4_STEP = 1.01 / 15,
// above any norm the index accepts), and PN4_UNIT = PN4_STEP in units of 2^-30, rounded up
constexpr float PN4_STEP = 1.01f / 15.f;
constexpr uint32_t PN4_UNIT = 72298617u;

struct InstDesc {
    int64_t vbase;   // first global vector id
    int64_t qwbase;  // first (vector, window) slot of the per-window pair counts
    int64_t wbase;   // first wptr entry (instances with nw > 1)
    int64_t ebase;   // first component (nnz offset)
    int64_t pbase;   // first 32-bit word of the instance's 4-bit ||y'||_2 codes (a multiple of 4)
    int32_t n;       // vectors
    int32_t m;       // dimensions
    int32_t rbase;   // first global rank
    int32_t nw;      // candidate windows
    int32_t W;       // window width
    int32_t G;       // query groups per CTA for this instance's class
    float t;         // threshold
    int32_t packed;  // 1: posting ids carry the size class in their top byte
};

struct Segment {      // the run of emitted pairs of one (x, window) slot qw, stored at segs[qw]
    int64_t src;      // offset in the staging buffer
    int32_t cnt;      // pairs (also in the per-slot counts; destination = scan(counts)[qw])
    int32_t i;        // local id of x
};

struct IndexArrays {
    DBuf<InstDesc> inst;
    DBuf<int32_t> vinst;  // instance of each vector
    DBuf<int64_t> cptr;
    DBuf<int32_t> crank;
    DBuf<float> cval;
    DBuf<int2> crow;
    DBuf<int4> vmeta;
    DBuf<int4> vcand;  // {row offset, |x'|, maxweight(x'), ||x'||_2 bound} per vector
    DBuf<uint32_t> pn4;  // 4-bit ||x'||_2 codes, eight per word, each instance 16-byte aligned
    DBuf<int32_t> len, split, qsplit;
    DBuf<float> mw, mwpre;
    DBuf<float> pnorm;  // ||x'||_2 of the unindexed prefix (rounded up, with the norm tolerance)
    DBuf<int32_t> rank_of_dim, dim_of_rank, nnz_d;
    DBuf<float> mw_d, mwr;
    DBuf<int64_t> lptr;
    DBuf<int32_t> wptr;
    DBuf<int2> post;
};

// The join phase of an index as a CUDA graph: the two workspace resets and the persistent
// join launch, captured on the index's first join; later joins update the nodes' pointers
// and launch parameters in the instantiated graph and replay it.
struct JoinGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t reset_ctr = nullptr, reset_cnt = nullptr, join = nullptr;
    int64_t launches = 0;
    JoinGraph() = default;
    JoinGraph(const JoinGraph &) = delete;
    JoinGraph &operator=(const JoinGraph &) = delete;
    ~JoinGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

}  // namespace aps

struct aps_index {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t flags = 0;
    int32_t k = 0;     // instances
    int64_t N = 0;     // vectors
    int64_t M = 0;     // dimensions (all instances)
    int64_t nnz = 0;
    int64_t nsuf = 0;  // indexed components
    int64_t nqw = 0;   // (vector, window) slots
    int64_t nwptr = 0;
    int64_t npw = 0;   // words of the 4-bit ||x'||_2 codes
    int32_t maxm = 0;
    float t = 0.f;     // single-instance threshold
    std::vector<aps::InstDesc> inst_h;
    aps::IndexArrays d;
    // join work list: vectors in decreasing estimated cost, grouped by class
    aps::DBuf<int32_t> items;
    int64_t class_begin[aps::JOIN_NCLS + 1] = {};  // classes G = 1, 2, 4, 8, then vectors of <= 2 components
    // output sizing from the previous join
    int64_t hint_pairs = 0;
    // pairs per query (times 16) that query batches on this index have needed at most: the
    // first staging of the next batch is sized from it, so that it rarely runs twice
    mutable std::atomic<int64_t> q_ppq16{64 * 16};
    aps::JoinGraph jgraph;  // the join phase, replayed by every join of this index
    aps_stats stats{};
    mutable std::mutex stats_mu;  // queries may run concurrently (serving slots)
};

namespace aps {

struct PairsAlloc {          // bookkeeping behind aps_pairs._priv
    void *block = nullptr;   // one allocation holding i, j and score
    size_t bytes = 0;        // its size (host blocks go back to the pinned cache)
    cudaStream_t stream = nullptr;
    int on_device = 1;
    int refs = 1;            // aps_pairs views sharing the block (batched results)
};

void pairs_release(aps_pairs *p);
// Replace device pairs by one pinned host copy.
aps_status pairs_to_host(aps_pairs *p, cudaStream_t s);

// External query rows prepared against an index: components re-expressed over the index's
// dimension ranks and sorted by rank, with |q|, maxweight(q) and the remscore boundary.
struct QueryArrays {
    DBuf<int2> crow;     // {rank, value} per component, rows in rank order
    DBuf<int4> vmeta;
    DBuf<int4> vcand;  // {row offset, |x'|, maxweight(x'), ||x'||_2 bound} per vector
    DBuf<uint32_t> pn4;  // 4-bit ||x'||_2 codes, eight per word, each instance 16-byte aligned    // {row offset, |q|, 0, 0}
    DBuf<int32_t> qsplit;
    DBuf<float> mw;
    int64_t nq = 0, nnz = 0;
};

// nnz_known: the number of components when the caller knows it from host row pointers
// (qptr[0] = 0 checked there), else -1 (both ends are then read back from the device).
aps_status prepare_queries(const aps_index *ix, const int64_t *qptr, const int32_t *qidx, const float *qval,
                           int32_t nq, float t, uint32_t flags, cudaStream_t s, QueryArrays &qa,
                           int64_t nnz_known = -1);

// Match prepared queries against every indexed vector: pairs (query row, vector id, score)
// with score >= t, sorted by (query, vector). Safe to call concurrently on different
// streams (it does not modify the index).
aps_status join_queries(const aps_index *ix, const QueryArrays &qa, float t, uint32_t flags, cudaStream_t s,
                        aps_pairs *out, aps_stats *stats);

// Build all index arrays for the instances whose CSRs are concatenated in (indptr, idx,
// val) with global row pointers (indptr[0] = 0). Inputs are device pointers.
aps_status build_index_device(aps_index *ix, const int64_t *indptr, const int32_t *idx,
                              const float *val, const std::vector<InstDesc> &inst_in,
                              cudaStream_t s, const aps_tuning *tune = nullptr);

// Join tile shapes (tune.cu): the size bucket of an instance, the process-wide table of
// query groups per bucket, and the autotuner (host arrays ro, hptr, m, t; device CSR).
int tune_bucket(int64_t n);
aps_tuning tuning_default();
aps_tuning tuning_current();
bool tuning_valid(const aps_tuning &tu);
void tuning_set(const aps_tuning &tu);
aps_status autotune_batch(int32_t k, const int64_t *ro, const int64_t *hptr, const int64_t *dp, const int32_t *di,
                          const float *dv, const int32_t *m, const float *t, uint32_t flags, cudaStream_t s,
                          aps_tuning *out, aps_tune_report *rep);

// Self-join of every instance of the index; fills a device aps_pairs (i, j, score)
// with per-instance ranges in pair_offsets_h (k+1 entries, may be null).
// nblk >= 2 and heavy > 0 (single-instance indexes): the vertical split with local pruning
// for the `heavy` costliest vectors, joined as nblk dimension blocks each (Sec. 5.1, Lemma 1).
aps_status join_all_pairs(aps_index *ix, uint32_t flags, aps_pairs *out,
                          std::vector<int64_t> *pair_offsets_h, int nblk = 0, int64_t heavy = 0);

// The self-join of a single-instance index with every buffer carved out of `arena`
// (arena_bytes, 256-byte aligned) and at most max_ctas CTAs; pairs land in the caller's
// arrays (capacity cap). *count receives the number of pairs, also on APS_EOVERFLOW.
aps_status join_noalloc(aps_index *ix, unsigned char *arena, size_t arena_bytes, int max_ctas, int32_t *oi,
                        int32_t *oj, float *os, int64_t cap, int64_t *count, cudaStream_t s);

// Dense all-pairs of X[n, d] (float32 rows; host or device per APS_DEVICE_PTRS) on the
// tensor cores with exact rescoring; d % 64 == 0, 64 <= d <= 512.
aps_status dense_all_pairs(const float *X, int32_t n, int32_t d, float t, uint32_t flags, cudaStream_t s,
                           aps_pairs *out, aps_stats *stats);
aps_status dense_all_pairs_device(const float *X, int32_t n, int32_t d, float t, cudaStream_t s, aps_pairs *out,
                                  aps_stats *stats, float *raw);
// The tensor cores' float32 products X_bf16 . X_bf16^T of the computed (upper) blocks into
// raw (row-major n x n, device memory); X on the device.
aps_status dense_tensor_products(const float *X, int32_t n, int32_t d, cudaStream_t s, float *raw);
double dense_margin(int d);
void dense_debug_stall(int64_t launches, uint64_t wait_ns);
void debug_stage_cap(int64_t pairs);

// The similarity graph G_S as a CSR adjacency from a pair list, its k nearest neighbours,
// and its release (graph.cu).
aps_status graph_csr(const int32_t *i, const int32_t *j, const float *s, int64_t count, int32_t n, uint32_t flags,
                     cudaStream_t st, aps_graph *out);
aps_status graph_knn(const aps_graph *g, int32_t k, int32_t *nbr, float *wk, uint32_t flags, cudaStream_t s);
void graph_release(aps_graph *g);

// Union of candidate pair lists, exact float64 rescoring from the rows, pairs >= t (verify.cu).
aps_status pairs_verify(const aps_pairs *lists, int32_t k, const int64_t *indptr, const int32_t *idx,
                        const float *val, int32_t n, int32_t m, float t, cudaStream_t s, aps_pairs *out,
                        int64_t *n_candidates);

}  // namespace aps
