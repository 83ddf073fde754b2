// Exact verification of candidate pairs: the score merge of the vertical algorithm with
// local pruning (Sec. 5.1, Lemma 1 / Eq. 2). The candidates of p dimension blocks (pairs
// whose partial score on some block reached t/p) are united, and each pair's full dot
// product is recomputed from the rows and compared with t.
//
//   1. keys i * n + j of every list, range-checked, into one buffer;
//   2. radix sort, then the first of each run of equal keys is kept (flag, scan, compact);
//   3. one thread per candidate: float64 dot of rows i and j by merging their sorted ids;
//   4. pairs with dot >= t compacted into (i, j, score), already in (i, j) order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "index.cuh"

namespace aps {
namespace {

__global__ void k_rows_check(const int64_t *__restrict__ indptr, const int32_t *__restrict__ idx, int32_t n,
                             int32_t m, unsigned long long *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = indptr[x], b = indptr[x + 1];
        bool ok = a >= 0 && b >= a;
        int prev = -1;
        for (int64_t p = a; ok && p < b; p++) {
            const int d = idx[p];
            ok = d > prev && d < m;
            prev = d;
        }
        if (!ok) atomicMin(bad, (unsigned long long)x);
    }
}

__global__ void k_list_keys(const int32_t *__restrict__ pi, const int32_t *__restrict__ pj, int64_t count, int32_t n,
                            uint64_t *keys, uint32_t *vals, unsigned long long *bad) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = pi[p], b = pj[p];
        if (a < 0 || a >= b || b >= n) {
            atomicMin(bad, (unsigned long long)p);
            keys[p] = 0;
        } else {
            keys[p] = (uint64_t)a * (uint64_t)n + (uint64_t)b;
        }
        vals[p] = 0u;
    }
}

__global__ void k_first_of_run(const uint64_t *__restrict__ keys, int64_t count, int32_t *first) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x)
        first[q] = (q == 0 || keys[q] != keys[q - 1]) ? 1 : 0;
}

__global__ void k_unique(const uint64_t *__restrict__ keys, const int32_t *__restrict__ first,
                         const int64_t *__restrict__ pos, int64_t count, uint64_t *ukeys) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x)
        if (first[q]) ukeys[pos[q]] = keys[q];
}

// float64 dot of rows i and j (ids strictly increasing in each row).
__global__ void k_pair_dot(const uint64_t *__restrict__ ukeys, int64_t nc, int32_t n,
                           const int64_t *__restrict__ indptr, const int32_t *__restrict__ idx,
                           const float *__restrict__ val, double t, int32_t *keep, float *score) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = ukeys[q];
        const int64_t i = (int64_t)(key / (uint64_t)n), j = (int64_t)(key % (uint64_t)n);
        int64_t a = indptr[i], ae = indptr[i + 1], b = indptr[j], be = indptr[j + 1];
        double acc = 0.0;
        while (a < ae && b < be) {
            const int32_t da = idx[a], db = idx[b];
            if (da == db) {
                acc += (double)val[a] * (double)val[b];
                a++;
                b++;
            } else if (da < db) {
                a++;
            } else {
                b++;
            }
        }
        keep[q] = acc >= t ? 1 : 0;
        score[q] = (float)acc;
    }
}

__global__ void k_emit_verified(const uint64_t *__restrict__ ukeys, const int32_t *__restrict__ keep,
                                const float *__restrict__ score, const int64_t *__restrict__ pos, int64_t nc,
                                int32_t n, int32_t *oi, int32_t *oj, float *os) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[q]) continue;
        const uint64_t key = ukeys[q];
        const int64_t d = pos[q];
        oi[d] = (int32_t)(key / (uint64_t)n);
        oj[d] = (int32_t)(key % (uint64_t)n);
        os[d] = score[q];
    }
}

}  // namespace

aps_status pairs_verify(const aps_pairs *lists, int32_t k, const int64_t *indptr, const int32_t *idx,
                        const float *val, int32_t n, int32_t m, float t, cudaStream_t s, aps_pairs *out,
                        int64_t *n_candidates) {
    memset(out, 0, sizeof(*out));
    int64_t total = 0;
    for (int r = 0; r < k; r++) total += std::max<int64_t>(lists[r].count, 0);
    DBuf<unsigned long long> bad;
    APS_TRY(bad.alloc(1, s));
    APS_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
    if (n > 0) {
        k_rows_check<<<grid_for(n, 256), 256, 0, s>>>(indptr, idx, n, m, bad.p);
        APS_LAUNCH_CHECK();
    }
    unsigned long long b = 0;
    APS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(b), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (b != ~0ull) {
        set_error("row %llu: ids not strictly increasing in [0, m) or a bad row pointer", b);
        return APS_EINVAL;
    }
    // 1. every list's keys in one buffer (host lists are brought over first)
    DBuf<uint64_t> keys;
    DBuf<uint32_t> vals;
    APS_TRY(keys.alloc((size_t)std::max<int64_t>(total, 1), s));
    APS_TRY(vals.alloc((size_t)std::max<int64_t>(total, 1), s));
    int64_t off = 0;
    for (int r = 0; r < k; r++) {
        const int64_t c = lists[r].count;
        if (c <= 0) continue;
        const int32_t *pi = lists[r].i, *pj = lists[r].j;
        DBuf<int32_t> hi, hj;
        if (!lists[r].on_device) {
            APS_TRY(hi.alloc((size_t)c, s));
            APS_TRY(hj.alloc((size_t)c, s));
            APS_CUDA(cudaMemcpyAsync(hi.p, pi, 4 * (size_t)c, cudaMemcpyHostToDevice, s));
            APS_CUDA(cudaMemcpyAsync(hj.p, pj, 4 * (size_t)c, cudaMemcpyHostToDevice, s));
            pi = hi.p;
            pj = hj.p;
        }
        k_list_keys<<<grid_for(c, 256), 256, 0, s>>>(pi, pj, c, n, keys.p + off, vals.p + off, bad.p);
        APS_LAUNCH_CHECK();
        off += c;
        APS_CUDA(cudaStreamSynchronize(s));  // host staging of this list may be released
    }
    APS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(b), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (b != ~0ull) {
        set_error("a candidate pair is outside 0 <= i < j < n");
        return APS_EINVAL;
    }
    // 2. sort and keep the first of each run
    if (total > 1) APS_TRY(sort_pairs(keys.p, vals.p, total, bits_for((uint64_t)n * (uint64_t)n), s));
    DBuf<int32_t> flag;
    DBuf<int64_t> pos;
    APS_TRY(flag.alloc((size_t)std::max<int64_t>(total, 1), s));
    APS_TRY(pos.alloc((size_t)total + 1, s));
    if (total > 0) {
        k_first_of_run<<<grid_for(total, 256), 256, 0, s>>>(keys.p, total, flag.p);
        APS_LAUNCH_CHECK();
    }
    APS_TRY(scan_exclusive(flag.p, pos.p, total, s));
    int64_t nc = 0;
    APS_CUDA(cudaMemcpyAsync(&nc, pos.p + total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (n_candidates) *n_candidates = nc;
    DBuf<uint64_t> ukeys;
    APS_TRY(ukeys.alloc((size_t)std::max<int64_t>(nc, 1), s));
    if (total > 0) {
        k_unique<<<grid_for(total, 256), 256, 0, s>>>(keys.p, flag.p, pos.p, total, ukeys.p);
        APS_LAUNCH_CHECK();
    }
    keys.release();
    vals.release();
    // 3. exact scores, 4. the pairs that reach t
    DBuf<int32_t> keep;
    DBuf<float> sc;
    DBuf<int64_t> kpos;
    APS_TRY(keep.alloc((size_t)std::max<int64_t>(nc, 1), s));
    APS_TRY(sc.alloc((size_t)std::max<int64_t>(nc, 1), s));
    APS_TRY(kpos.alloc((size_t)nc + 1, s));
    if (nc > 0) {
        k_pair_dot<<<grid_for(nc, 256), 256, 0, s>>>(ukeys.p, nc, n, indptr, idx, val, (double)t, keep.p, sc.p);
        APS_LAUNCH_CHECK();
    }
    APS_TRY(scan_exclusive(keep.p, kpos.p, nc, s));
    int64_t np = 0;
    APS_CUDA(cudaMemcpyAsync(&np, kpos.p + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    PairsAlloc *pa = new PairsAlloc();
    pa->stream = s;
    const size_t seg = ((size_t)np * 4 + 127) & ~(size_t)127;
    aps_status st = dalloc(&pa->block, std::max<size_t>(3 * seg, 256), s);
    if (st != APS_OK) {
        delete pa;
        return st;
    }
    char *blk = static_cast<char *>(pa->block);
    int32_t *oi = reinterpret_cast<int32_t *>(blk);
    int32_t *oj = reinterpret_cast<int32_t *>(blk + seg);
    float *os = reinterpret_cast<float *>(blk + 2 * seg);
    if (nc > 0) {
        k_emit_verified<<<grid_for(nc, 256), 256, 0, s>>>(ukeys.p, keep.p, sc.p, kpos.p, nc, n, oi, oj, os);
        APS_LAUNCH_CHECK();
    }
    APS_CUDA(cudaStreamSynchronize(s));
    out->count = np;
    out->i = oi;
    out->j = oj;
    out->score = os;
    out->on_device = 1;
    out->_reserved = 0;
    out->_priv = pa;
    return APS_OK;
}

}  // namespace aps
