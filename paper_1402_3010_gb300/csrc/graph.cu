// The similarity graph G_S(V, t) = (V, M) of the problem definition (Sec. 2.1): the
// undirected graph whose edges are the matches, edge weight w(u, v) = u.v, as a CSR
// adjacency, and the k nearest neighbours of every vertex read off it (the k-nn use of
// the graph in Sec. 2.2).
//
// Build, for pairs (i, j, s) strictly increasing in (i, j) with i < j:
//   1. a stable radix sort by j of keys (i << 32 | j) with the score as payload, so that
//      the pairs of each j come out in increasing i and carry everything the fill needs;
//   2. start_i[v] / start_j[v] = first position of v in the i-sorted input / in the
//      j-sorted keys (binary searches, no atomics); v's degree is the sum of its two run
//      lengths and row_ptr[v] = start_i[v] + start_j[v];
//   3. row v = its lower neighbours (the j-sorted run of v, increasing i) followed by its
//      upper neighbours (the input run of v, increasing j): every row is in increasing
//      neighbour id with no sort of the adjacency itself. Both fills read sequentially.
// Everything is deterministic.
#include <algorithm>
#include <cstring>

#include "index.cuh"

namespace aps {
namespace {

// Smallest index of a pair that is out of range, not i < j, or not after its predecessor.
__global__ void k_pairs_check(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t count,
                              int32_t n, unsigned long long *bad) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = pi[p], b = pj[p];
        bool ok = a >= 0 && a < b && b < n;
        if (ok && p > 0) {
            const int32_t a0 = pi[p - 1], b0 = pj[p - 1];
            ok = a0 < a || (a0 == a && b0 < b);
        }
        if (!ok) atomicMin(bad, (unsigned long long)p);
    }
}

__global__ void k_sort_keys(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                            const float *__restrict__ ps, int64_t count, uint64_t *keys, uint32_t *vals) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        keys[p] = ((uint64_t)(uint32_t)pi[p] << 32) | (uint64_t)(uint32_t)pj[p];
        vals[p] = __float_as_uint(ps[p]);
    }
}

// First position of each vertex v in [0, n] in the i-sorted pairs and in the j-sorted
// keys (= count for v = n); row_ptr[v] = start_i[v] + start_j[v].
__global__ void k_starts(const int32_t *__restrict__ pi, const uint64_t *__restrict__ keys, int64_t count, int32_t n,
                         int64_t *start_i, int64_t *start_j, int64_t *row_ptr) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = count;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (pi[mid] < v) lo = mid + 1; else hi = mid;
        }
        const int64_t a = lo;
        lo = 0;
        hi = count;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)(uint32_t)keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        start_i[v] = a;
        start_j[v] = lo;
        row_ptr[v] = a + lo;
    }
}

// Upper neighbours: pair p = (v, j) lands after v's lower neighbours.
__global__ void k_fill_upper(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                             const float *__restrict__ ps, int64_t count, const int64_t *__restrict__ row_ptr,
                             const int64_t *__restrict__ start_i, const int64_t *__restrict__ start_j, int32_t *col,
                             float *w) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = pi[p];
        const int64_t d = row_ptr[v] + (start_j[v + 1] - start_j[v]) + (p - start_i[v]);
        col[d] = pj[p];
        w[d] = ps[p];
    }
}

// Lower neighbours: the q-th key in j order, (i, v), is v's (q - start_j[v])-th.
__global__ void k_fill_lower(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t count,
                             const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ start_j, int32_t *col,
                             float *w) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[q];
        const int32_t v = (int32_t)(uint32_t)key;
        const int64_t d = row_ptr[v] + (q - start_j[v]);
        col[d] = (int32_t)(key >> 32);
        w[d] = __uint_as_float(vals[q]);
    }
}

// Rank key of a neighbour: larger weight first, then smaller id; distinct within a row.
__device__ __forceinline__ unsigned long long knn_key(float w, int32_t id) {
    uint32_t b = __float_as_uint(w);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // order-preserving map of the float
    return ((unsigned long long)b << 32) | (unsigned long long)(0xffffffffu - (uint32_t)id);
}

// One warp per vertex: k rounds, each taking the largest key below the previous one.
__global__ void k_knn(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                      const float *__restrict__ w, int32_t n, int32_t k, int32_t *nbr, float *wk) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += nw) {
        const int64_t b = row_ptr[v], e = row_ptr[v + 1];
        unsigned long long prev = ~0ull;
        for (int r = 0; r < k; r++) {
            unsigned long long best = 0ull;
            if (prev != 0ull) {
                for (int64_t q = b + lane; q < e; q += 32) {
                    const unsigned long long key = knn_key(w[q], col[q]);
                    if (key < prev && key > best) best = key;
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
                    best = y > best ? y : best;
                }
            }
            if (lane == 0) {
                int32_t id = -1;
                float wt = 0.f;
                if (best != 0ull) {
                    id = (int32_t)(0xffffffffu - (uint32_t)(best & 0xffffffffull));
                    uint32_t hb = (uint32_t)(best >> 32);
                    hb = (hb & 0x80000000u) ? (hb & 0x7fffffffu) : ~hb;
                    wt = __uint_as_float(hb);
                }
                nbr[v * (int64_t)k + r] = id;
                wk[v * (int64_t)k + r] = wt;
            }
            prev = best;
        }
    }
}

struct GraphAlloc {  // bookkeeping behind aps_graph._priv
    void *block = nullptr;
    cudaStream_t stream = nullptr;
    int on_device = 1;
};

size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

}  // namespace

aps_status graph_csr(const int32_t *i_in, const int32_t *j_in, const float *s_in, int64_t count, int32_t n,
                     uint32_t flags, cudaStream_t s, aps_graph *out) {
    memset(out, 0, sizeof(*out));
    if (n < 0 || count < 0 || (count > 0 && (!i_in || !j_in || !s_in))) {
        set_error("need n >= 0, count >= 0 and non-NULL pair arrays");
        return APS_EINVAL;
    }
    if (count > (int64_t)0xffffffffll || 2 * count >= (1ll << 62)) {
        set_error("%lld pairs exceed the 2^32 the graph build supports", (long long)count);
        return APS_EINVAL;
    }
    // the pairs on the device
    DBuf<int32_t> di, dj;
    DBuf<float> ds;
    const int32_t *pi = i_in, *pj = j_in;
    const float *ps = s_in;
    if (!(flags & APS_DEVICE_PTRS) && count > 0) {
        APS_TRY(di.alloc((size_t)count, s));
        APS_TRY(dj.alloc((size_t)count, s));
        APS_TRY(ds.alloc((size_t)count, s));
        APS_CUDA(cudaMemcpyAsync(di.p, i_in, 4 * (size_t)count, cudaMemcpyHostToDevice, s));
        APS_CUDA(cudaMemcpyAsync(dj.p, j_in, 4 * (size_t)count, cudaMemcpyHostToDevice, s));
        APS_CUDA(cudaMemcpyAsync(ds.p, s_in, 4 * (size_t)count, cudaMemcpyHostToDevice, s));
        pi = di.p;
        pj = dj.p;
        ps = ds.p;
    }
    if (count > 0) {
        DBuf<unsigned long long> bad;
        APS_TRY(bad.alloc(1, s));
        APS_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
        k_pairs_check<<<grid_for(count, 256), 256, 0, s>>>(pi, pj, count, n, bad.p);
        APS_LAUNCH_CHECK();
        unsigned long long b = 0;
        APS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(b), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        if (b != ~0ull) {
            set_error("pair %llu is out of range [0, n), not i < j, or not strictly after the previous pair in "
                      "(i, j) order",
                      b);
            return APS_EINVAL;
        }
    }
    // the graph: one allocation for row_ptr, col and w
    const int64_t nnz = 2 * count;
    const size_t o_col = align128(sizeof(int64_t) * ((size_t)n + 1));
    const size_t o_w = o_col + align128(sizeof(int32_t) * (size_t)nnz);
    const size_t bytes = o_w + align128(sizeof(float) * (size_t)nnz);
    GraphAlloc *ga = new GraphAlloc();
    ga->stream = s;
    aps_status st = dalloc(&ga->block, bytes, s);
    if (st != APS_OK) {
        delete ga;
        return st;
    }
    char *blk = static_cast<char *>(ga->block);
    int64_t *row_ptr = reinterpret_cast<int64_t *>(blk);
    int32_t *col = reinterpret_cast<int32_t *>(blk + o_col);
    float *w = reinterpret_cast<float *>(blk + o_w);
    out->n = n;
    out->on_device = 1;
    out->nnz = nnz;
    out->row_ptr = row_ptr;
    out->col = col;
    out->w = w;
    out->_priv = ga;
    auto fail = [&](aps_status e) {
        graph_release(out);
        return e;
    };
    {
        DBuf<int64_t> start;
        DBuf<uint64_t> keys;
        DBuf<uint32_t> vals;
        if ((st = start.alloc(2 * ((size_t)n + 1), s)) != APS_OK) return fail(st);
        if ((st = keys.alloc((size_t)count, s)) != APS_OK) return fail(st);
        if ((st = vals.alloc((size_t)count, s)) != APS_OK) return fail(st);
        int64_t *start_i = start.p, *start_j = start.p + n + 1;
        if (count > 0) {
            k_sort_keys<<<grid_for(count, 256), 256, 0, s>>>(pi, pj, ps, count, keys.p, vals.p);
            count_launch();
            if ((st = sort_pairs(keys.p, vals.p, count, bits_for((uint64_t)n), s)) != APS_OK) return fail(st);
        }
        k_starts<<<grid_for((int64_t)n + 1, 256), 256, 0, s>>>(pi, keys.p, count, n, start_i, start_j, row_ptr);
        count_launch();
        if (count > 0) {
            k_fill_upper<<<grid_for(count, 256), 256, 0, s>>>(pi, pj, ps, count, row_ptr, start_i, start_j, col, w);
            count_launch();
            k_fill_lower<<<grid_for(count, 256), 256, 0, s>>>(keys.p, vals.p, count, row_ptr, start_j, col, w);
            count_launch();
        }
        if (cudaGetLastError() != cudaSuccess) return fail(APS_ECUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(APS_ECUDA);
    }
    if (flags & APS_HOST_OUTPUT) {
        void *h = nullptr;
        if (cudaMallocHost(&h, bytes) != cudaSuccess) {
            set_error("cudaMallocHost of %zu bytes failed", bytes);
            return fail(APS_ENOMEM);
        }
        if (cudaMemcpyAsync(h, ga->block, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFreeHost(h);
            return fail(APS_ECUDA);
        }
        dfree(ga->block, s);
        ga->block = h;
        ga->on_device = 0;
        char *hb = static_cast<char *>(h);
        out->on_device = 0;
        out->row_ptr = reinterpret_cast<int64_t *>(hb);
        out->col = reinterpret_cast<int32_t *>(hb + o_col);
        out->w = reinterpret_cast<float *>(hb + o_w);
    }
    return APS_OK;
}

aps_status graph_knn(const aps_graph *g, int32_t k, int32_t *nbr, float *wk, uint32_t flags, cudaStream_t s) {
    if (!g || !g->_priv || !g->on_device) {
        set_error("the graph must be a device graph from aps_graph_csr");
        return APS_EINVAL;
    }
    if (k < 1 || k > 256 || !nbr || !wk) {
        set_error("need 1 <= k <= 256 and non-NULL output arrays");
        return APS_EINVAL;
    }
    const int64_t nk = (int64_t)g->n * k;
    if (nk == 0) return APS_OK;
    DBuf<int32_t> dn;
    DBuf<float> dw;
    int32_t *on = nbr;
    float *ow = wk;
    if (!(flags & APS_DEVICE_PTRS)) {
        APS_TRY(dn.alloc((size_t)nk, s));
        APS_TRY(dw.alloc((size_t)nk, s));
        on = dn.p;
        ow = dw.p;
    }
    k_knn<<<grid_for((int64_t)g->n * 32, 256, (int64_t)num_sms() * 64), 256, 0, s>>>(g->row_ptr, g->col, g->w, g->n,
                                                                                      k, on, ow);
    APS_LAUNCH_CHECK();
    if (!(flags & APS_DEVICE_PTRS)) {
        APS_CUDA(cudaMemcpyAsync(nbr, on, sizeof(int32_t) * (size_t)nk, cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaMemcpyAsync(wk, ow, sizeof(float) * (size_t)nk, cudaMemcpyDeviceToHost, s));
    }
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

void graph_release(aps_graph *g) {
    if (!g || !g->_priv) return;
    GraphAlloc *ga = static_cast<GraphAlloc *>(g->_priv);
    if (ga->on_device)
        dfree(ga->block, ga->stream);
    else
        cudaFreeHost(ga->block);
    delete ga;
    memset(g, 0, sizeof(*g));
}

}  // namespace aps
