// Index build: input statistics, dimension ranking, canonical rows, partial-indexing
// split and the suffix inverted index (the preprocessing of all-pairs-1/2 and the
// index-insertion step of Alg. 1, done for all vectors at once).
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "index.cuh"

namespace aps {
namespace {

constexpr int T256 = 256;

__device__ __forceinline__ int inst_of_vec(const InstDesc *inst, int k, int64_t x) {
    // last instance whose vbase <= x (instances with n == 0 share the next vbase)
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (inst[mid].vbase <= x) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

__device__ __forceinline__ int inst_of_rank(const InstDesc *inst, int k, int64_t r) {
    int lo = 0, hi = k;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int64_t)inst[mid].rbase <= r) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

__global__ void k_vinst(const InstDesc *inst, int k, int64_t N, int32_t *vinst) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N; x += (int64_t)gridDim.x * blockDim.x)
        vinst[x] = inst_of_vec(inst, k, x);
}

// Validation codes reported as (row << 8 | code) through atomicMin.
enum { E_PTR = 1, E_IDX_RANGE = 2, E_IDX_ORDER = 3, E_VALUE = 4, E_NORM = 5 };

// One warp per row: checks the row, records |x| and maxweight(x), and copies the values
// (scaled to unit norm with APS_NORMALIZE). The lanes read 32 components at a time; the
// error code is that of the row's first bad component (range before order before value,
// as for a sequential check). The float64 sum of squares is a warp tree sum.
__global__ void k_validate(const int64_t *__restrict__ indptr, const int32_t *__restrict__ idx,
                           const float *__restrict__ val, const int32_t *__restrict__ vinst,
                           const InstDesc *__restrict__ inst, int64_t N, int64_t nnz, uint32_t flags,
                           int32_t *__restrict__ erow, float *__restrict__ vout, int32_t *__restrict__ len,
                           float *__restrict__ mw, unsigned long long *err,
                           unsigned long long *longest_out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long longest = 0;  // the longest row this warp met (to *longest_out, when given)
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < N; x += nwarps) {
        const int64_t a = indptr[x], b = indptr[x + 1];
        if (a < 0 || b < a || b > nnz) {
            if (lane == 0) {
                atomicMin(err, ((unsigned long long)x << 8) | E_PTR);
                len[x] = 0;
                mw[x] = 0.f;
            }
            continue;
        }
        const int m = inst[vinst[x]].m;
        int code = 0, prev_last = -1;
        double ss = 0.0;
        for (int64_t base = a; base < b; base += 32) {
            const int64_t p = base + lane;
            const int cnt = (int)min((int64_t)32, b - base);
            int d = 0;
            float v = 1.f;
            if (p < b) {
                d = idx[p];
                v = val[p];
                erow[p] = (int32_t)x;
            }
            int prevd = __shfl_up_sync(0xffffffffu, d, 1);
            if (lane == 0) prevd = prev_last;
            int ec = 0;
            if (p < b) {
                if (d < 0 || d >= m) ec = E_IDX_RANGE;
                else if (d <= prevd) ec = E_IDX_ORDER;
                else if (!(v > 0.f) || !isfinite(v)) ec = E_VALUE;
            }
            const unsigned bad = __ballot_sync(0xffffffffu, ec != 0);
            if (!code && bad) code = __shfl_sync(0xffffffffu, ec, __ffs(bad) - 1);
            if (p < b) ss += (double)v * (double)v;
            prev_last = __shfl_sync(0xffffffffu, d, cnt - 1);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        float best = 0.f;
        if (b > a && !code) {
            const double nrm = sqrt(ss);
            if (!(flags & APS_NORMALIZE) && ((flags & APS_SUBUNIT_NORMS) ? nrm > 1.0 + 1e-3 : fabs(nrm - 1.0) > 1e-3))
                code = E_NORM;
            for (int64_t p = a + lane; p < b; p += 32) {
                const float v = (flags & APS_NORMALIZE) ? (float)((double)val[p] / nrm) : val[p];
                vout[p] = v;
                best = fmaxf(best, v);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
        }
        if (lane == 0) {
            if (code) atomicMin(err, ((unsigned long long)x << 8) | (unsigned long long)code);
            len[x] = (int32_t)(b - a);
            mw[x] = best;
            longest = max(longest, (unsigned long long)(b - a));
        }
    }
    if (lane == 0 && longest && longest_out) atomicMax(longest_out, longest);
}

// The rank-ordered rows when no row is longer than 64 components: one warp per row sorts
// the row's (rank, value) pairs by a bitonic network over the lanes, two per lane (element
// k = 2 * lane + h), instead of the global sort by (row, rank) that longer rows need.
__global__ void k_canon_rows64(const int64_t *__restrict__ cptr, const int32_t *__restrict__ idx,
                               const float *__restrict__ vout, const int32_t *__restrict__ vinst,
                               const InstDesc *__restrict__ inst, const int32_t *__restrict__ rank_of_dim,
                               int64_t N, int32_t *crank, float *cval) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < N; x += nwarps) {
        const int64_t a = cptr[x];
        const int L = (int)(cptr[x + 1] - a);  // <= 64
        const int64_t rb = inst[vinst[x]].rbase;
        const int k0 = 2 * lane, k1 = k0 + 1;
        int r0 = 0x7fffffff, r1 = 0x7fffffff;  // padding sorts last
        float v0 = 0.f, v1 = 0.f;
        if (k0 < L) {
            r0 = rank_of_dim[rb + idx[a + k0]];
            v0 = vout[a + k0];
        }
        if (k1 < L) {
            r1 = rank_of_dim[rb + idx[a + k1]];
            v1 = vout[a + k1];
        }
#pragma unroll
        for (int size = 2; size <= 64; size <<= 1) {
            // blocks of `size` elements ascending where bit `size` of k is 0, descending elsewhere
            const bool asc = (k0 & size) == 0;  // (k0 and k1 agree on it for size >= 2)
#pragma unroll
            for (int j = size >> 1; j > 0; j >>= 1) {
                if (j == 1) {  // elements k0, k1 of this lane
                    if ((r0 > r1) == asc) {
                        const int tr = r0;
                        r0 = r1;
                        r1 = tr;
                        const float tv = v0;
                        v0 = v1;
                        v1 = tv;
                    }
                } else {  // element k and k ^ j: the same slot of lane ^ (j / 2)
                    const int lm = j >> 1;
                    const int p0 = __shfl_xor_sync(0xffffffffu, r0, lm), p1 = __shfl_xor_sync(0xffffffffu, r1, lm);
                    const float q0 = __shfl_xor_sync(0xffffffffu, v0, lm), q1 = __shfl_xor_sync(0xffffffffu, v1, lm);
                    const bool keep_min = ((lane & lm) == 0) == asc;  // the lower element keeps the min when ascending
                    if (keep_min ? p0 < r0 : p0 > r0) {
                        r0 = p0;
                        v0 = q0;
                    }
                    if (keep_min ? p1 < r1 : p1 > r1) {
                        r1 = p1;
                        v1 = q1;
                    }
                }
            }
        }
        if (k0 < L) {
            crank[a + k0] = r0;
            cval[a + k0] = v0;
        }
        if (k1 < L) {
            crank[a + k1] = r1;
            cval[a + k1] = v1;
        }
    }
}

// Per-dimension non-zero count and maxweight_i(V) (positive floats order like ints).
__global__ void k_dimstats(const int32_t *__restrict__ idx, const float *__restrict__ vout,
                           const int32_t *__restrict__ erow, const int32_t *__restrict__ vinst,
                           const InstDesc *__restrict__ inst, int64_t nnz, int32_t *nnz_d, float *mw_d) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t D = (int64_t)inst[vinst[erow[p]]].rbase + idx[p];
        atomicAdd(&nnz_d[D], 1);
        atomicMax(reinterpret_cast<int *>(&mw_d[D]), __float_as_int(vout[p]));
    }
}

// The same for a batch of instances of at most DIMSTATS_DIMS dimensions each: one CTA per
// instance counts in shared memory (shared atomics instead of global ones on 25M
// dimensions), first the non-zeros, then the maxima, each written out once.
constexpr int DIMSTATS_DIMS = 56 * 1024;  // 224 KB of 32-bit counters
__global__ void __launch_bounds__(1024) k_dimstats_inst(const int64_t *__restrict__ cptr,
                                                        const int32_t *__restrict__ idx,
                                                        const float *__restrict__ vout,
                                                        const InstDesc *__restrict__ inst, int32_t *nnz_d,
                                                        float *mw_d) {
    extern __shared__ uint32_t dcnt[];  // [I.m]
    const InstDesc I = inst[blockIdx.x];
    const int64_t a = cptr[I.vbase], b = cptr[I.vbase + I.n];
    for (int pass = 0; pass < 2; pass++) {
        for (int d = threadIdx.x; d < I.m; d += blockDim.x) dcnt[d] = 0u;
        __syncthreads();
        for (int64_t p = a + threadIdx.x; p < b; p += blockDim.x) {
            if (pass == 0) atomicAdd(&dcnt[idx[p]], 1u);
            else atomicMax(&dcnt[idx[p]], __float_as_uint(vout[p]));  // positive floats order like their bits
        }
        __syncthreads();
        for (int d = threadIdx.x; d < I.m; d += blockDim.x) {
            if (pass == 0) nnz_d[(int64_t)I.rbase + d] = (int32_t)dcnt[d];
            else mw_d[(int64_t)I.rbase + d] = __uint_as_float(dcnt[d]);
        }
        __syncthreads();
    }
}

// Dimension order of all-pairs-1: decreasing non-zero count; the sort is stable and the
// input is in id order, so ties keep ascending dimension id.
__global__ void k_rank_keys(const int32_t *__restrict__ nnz_d, const InstDesc *__restrict__ inst, int k,
                            int64_t M, int nbits, uint64_t nmax, uint64_t *keys, uint32_t *vals) {
    for (int64_t D = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; D < M; D += (int64_t)gridDim.x * blockDim.x) {
        uint64_t ki = (uint64_t)inst_of_rank(inst, k, D);
        keys[D] = (ki << nbits) | (nmax - (uint64_t)nnz_d[D]);
        vals[D] = (uint32_t)D;
    }
}

__global__ void k_rank_scatter(const uint32_t *__restrict__ vals, const InstDesc *__restrict__ inst, int k,
                               int64_t M, const float *__restrict__ mw_d, int32_t *rank_of_dim,
                               int32_t *dim_of_rank, float *mwr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t D = vals[i];
        int ki = inst_of_rank(inst, k, i);
        rank_of_dim[D] = (int32_t)(i - inst[ki].rbase);
        dim_of_rank[i] = (int32_t)D;
        mwr[i] = mw_d[D];
    }
}

__global__ void k_canon_keys(const int32_t *__restrict__ idx, const int32_t *__restrict__ erow,
                             const int32_t *__restrict__ vinst, const InstDesc *__restrict__ inst,
                             const int32_t *__restrict__ rank_of_dim, int64_t nnz, int rb, uint64_t *keys,
                             uint32_t *vals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = erow[p];
        int32_t r = rank_of_dim[(int64_t)inst[vinst[x]].rbase + idx[p]];
        keys[p] = ((uint64_t)x << rb) | (uint64_t)r;
        vals[p] = (uint32_t)p;
    }
}

__global__ void k_canon_gather(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                               const float *__restrict__ vout, int64_t nnz, uint64_t rmask, int32_t *crank,
                               float *cval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        crank[q] = (int32_t)(keys[q] & rmask);
        cval[q] = vout[vals[q]];
    }
}

// Partial indexing (all-pairs-1): walking x's components in rank order, b accumulates
// x[i] * maxweight_i(V) in float64; qsplit = the first component where b >= t (the
// remscore boundary for x as a query). The index split is qsplit, or 0 without partial
// indexing, or, for a queryable index, the first component where ||x_prefix||_2 reaches
// t (with a margin for the 1e-3 norm tolerance). One warp per row: the lanes load 32
// components, form their products (exact in float64) and take the running sums by a warp
// prefix scan, carried from one 32-component step to the next. The scan associates the
// terms differently from a left-to-right sum, so where b comes within rounding of t the
// split may fall one component apart from a sequential one; either is a valid split (the
// bound of the unindexed prefix stays below t up to rounding, which the float64 band of
// the decisions covers).
__device__ __forceinline__ double warp_incl_scan_f64(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__global__ void k_split(const int64_t *__restrict__ cptr, const int32_t *__restrict__ crank,
                        const float *__restrict__ cval, const float *__restrict__ mwr,
                        const int32_t *__restrict__ vinst, const InstDesc *__restrict__ inst, int64_t N,
                        uint32_t flags, int32_t *split, int32_t *qsplit, float *mwpre, float *pnorm, int64_t M,
                        uint64_t *pkeys, uint32_t *pvals, unsigned long long *nsuf) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long nsuf_w = 0;  // this warp's indexed components (lane 0)
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < N; x += nwarps) {
        const InstDesc &I = inst[vinst[x]];
        const double t = (double)I.t;
        const int64_t a = cptr[x], b = cptr[x + 1];
        const int32_t L = (int32_t)(b - a);
        const bool need_cs = (flags & APS_QUERYABLE) != 0;  // the norm-bound split only for queryable indexes
        int32_t qs = L, cs = L;
        double bmw = 0.0, ss = 0.0;  // sums of the components before this step
        for (int64_t base = a; base < b && (qs == L || (need_cs && cs == L)); base += 32) {
            const int64_t p = base + lane;
            double pr = 0.0, sq = 0.0;
            if (p < b) {
                const double v = (double)cval[p];
                pr = v * (double)mwr[(int64_t)I.rbase + crank[p]];
                sq = v * v;
            }
            const double bi = bmw + warp_incl_scan_f64(pr, lane);
            const unsigned hit = __ballot_sync(0xffffffffu, p < b && bi >= t);
            if (qs == L && hit) qs = (int32_t)(base - a) + __ffs(hit) - 1;
            bmw = __shfl_sync(0xffffffffu, bi, 31);
            if (need_cs) {
                const double si = ss + warp_incl_scan_f64(sq, lane);
                const unsigned hc = __ballot_sync(0xffffffffu, p < b && si * (1.0 + 2e-3) >= t * t);
                if (cs == L && hc) cs = (int32_t)(base - a) + __ffs(hc) - 1;
                ss = __shfl_sync(0xffffffffu, si, 31);
            }
        }
        const int32_t sp = (flags & APS_NO_PARTIAL_INDEX) ? 0 : ((flags & APS_QUERYABLE) ? cs : qs);
        // maxweight(x') and an upper bound of ||x'||_2 (float32 with every operation rounded
        // up, so the bound can only come out above the exact norm; times 1 + 1.1e-3 for the
        // 1e-3 norm tolerance of the vectors it will be dotted with)
        float best = 0.f, pss = 0.f;
        for (int64_t p = a + lane; p < a + sp; p += 32) {
            const float c = cval[p];
            best = fmaxf(best, c);
            pss = __fmaf_ru(c, c, pss);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
            pss = __fadd_ru(pss, __shfl_xor_sync(0xffffffffu, pss, o));
        }
        if (lane == 0) {
            split[x] = sp;
            qsplit[x] = qs;
            mwpre[x] = best;
            pnorm[x] = sp ? __fmul_ru(__fsqrt_ru(pss), 1.0011f) : 0.f;
            nsuf_w += (unsigned long long)(L - sp);
        }
        // the row's posting keys: a suffix entry its global rank, a prefix entry a sentinel
        // past the last rank (it sorts last); the value is the entry's index. The sort is
        // stable and entries arrive in row order, so every list comes out in increasing id.
        for (int64_t p = a + lane; p < b; p += 32) {
            pkeys[p] = (p - a >= sp) ? (uint64_t)I.rbase + (uint64_t)crank[p] : (uint64_t)M;
            pvals[p] = (uint32_t)p;
        }
    }
    if (lane == 0 && nsuf_w) atomicAdd(nsuf, nsuf_w);
}

__global__ void k_post_fill(const uint32_t *__restrict__ vals, const int32_t *__restrict__ erow,
                            const float *__restrict__ cval, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ vinst, const InstDesc *__restrict__ inst, int64_t nsuf,
                            int2 *post) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nsuf; q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t p = vals[q];
        int64_t x = erow[p];
        const InstDesc &I = inst[vinst[x]];
        const int32_t lid = (int32_t)(x - I.vbase);
        const int32_t tag = I.packed ? (min(len[x], 255) << 24) : 0;
        post[q] = make_int2(lid | tag, __float_as_int(cval[p]));
    }
}

// List pointers from the sorted posting keys: lptr[R] = first suffix entry with key >= R
// (binary search; lptr[M] = nsuf).
__global__ void k_lptr(const uint64_t *__restrict__ keys, int64_t nsuf, int64_t M, int64_t *lptr) {
    for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R <= M; R += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nsuf;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < (uint64_t)R) lo = mid + 1; else hi = mid;
        }
        lptr[R] = lo;
    }
}

// Interleaved rows and per-vector metadata read by the join.
__global__ void k_pack(const int64_t *__restrict__ cptr, const int32_t *__restrict__ crank,
                       const float *__restrict__ cval, const int32_t *__restrict__ len,
                       const int32_t *__restrict__ split, const float *__restrict__ mwpre,
                       const float *__restrict__ pnorm, const int32_t *__restrict__ vinst,
                       const InstDesc *__restrict__ inst, int64_t N, int64_t nnz, int2 *crow, int4 *vmeta,
                       int4 *vcand, uint32_t *pn4) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += stride)
        crow[p] = make_int2(crank[p], __float_as_int(cval[p]));
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < N; x += stride) {
        vmeta[x] = make_int4((int32_t)cptr[x], len[x], split[x], __float_as_int(mwpre[x]));
        vcand[x] = make_int4((int32_t)cptr[x], split[x], __float_as_int(mwpre[x]), __float_as_int(pnorm[x]));
        // the smallest 4-bit code c with c * PN4_STEP >= ||x'||_2 (the bound stays a bound)
        const double pn = (double)pnorm[x];
        int c = (int)ceil(pn / (double)PN4_STEP);
        if ((double)c * (double)PN4_STEP < pn) c++;
        c = min(max(c, 0), 15);
        const InstDesc &I = inst[vinst[x]];
        const int64_t lx = x - I.vbase;
        if (c) atomicOr(&pn4[I.pbase + (lx >> 3)], (uint32_t)c << (4 * (lx & 7)));
    }
}

// Window offsets inside each list of a multi-window instance: w[i] = the offset in list R
// of its first entry with local id >= i * W (lists are in increasing id; binary search).
__global__ void k_wptr(const InstDesc *__restrict__ inst, int k, int64_t M, const int64_t *__restrict__ lptr,
                       const int2 *__restrict__ post, int32_t *wptr) {
    for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < M; R += (int64_t)gridDim.x * blockDim.x) {
        const InstDesc &I = inst[inst_of_rank(inst, k, R)];
        if (I.nw <= 1) continue;
        const int32_t idmask = I.packed ? 0x00ffffff : 0x7fffffff;
        const int64_t a = lptr[R], b = lptr[R + 1];
        int32_t *w = wptr + I.wbase + (R - I.rbase) * (I.nw + 1);
        int64_t lo = a;
        for (int i = 0; i <= I.nw; i++) {
            const int32_t bound = i * I.W;
            int64_t hi = b;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((post[mid].x & idmask) < bound) lo = mid + 1; else hi = mid;
            }
            w[i] = (int32_t)(lo - a);
        }
    }
}

// Join work list: every vector with later candidates in its instance, keyed by
// (class, decreasing estimated cost) so that the persistent join takes the most expensive
// queries first (least-loaded-first idea of the vertical algorithm's binning). Classes 0-3
// are the instance's tile shape (G = 1, 2, 4, 8 query groups per CTA); class 4 holds the
// vectors with one or two components, which the join streams one warp per vector.
__global__ void k_item_keys(const int64_t *__restrict__ cptr, const int32_t *__restrict__ crank,
                            const int64_t *__restrict__ lptr, const int32_t *__restrict__ vinst,
                            const InstDesc *__restrict__ inst, int64_t N, uint64_t *keys, uint32_t *vals,
                            unsigned long long *class_count) {
    // one warp per vector: the lanes read its ranks side by side and look up their lists;
    // the class counts go through shared memory (one global atomic per class and block)
    __shared__ unsigned long long ccount[JOIN_NCLS];
    if (threadIdx.x < JOIN_NCLS) ccount[threadIdx.x] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < N; x += nwarps) {
        const InstDesc &I = inst[vinst[x]];
        const int64_t lx = x - I.vbase;
        if (lx >= (int64_t)I.n - 1) {  // no later candidates: after every class
            if (lane == 0) {
                keys[x] = (uint64_t)JOIN_NCLS << 24;
                vals[x] = (uint32_t)x;
            }
            continue;
        }
        const int64_t a = cptr[x], b = cptr[x + 1];
        int64_t lsum = 0;  // total length of x's posting lists
        for (int64_t p = a + lane; p < b; p += 32) {
            const int64_t R = (int64_t)I.rbase + crank[p];
            lsum += lptr[R + 1] - lptr[R];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) {
            const double later = (double)(I.n - 1 - lx);
            const double cost = (double)lsum * later / (double)I.n + later / 8.0 + 32.0;
            // decreasing cost inside the class, in 24 bits (the costliest saturate together)
            const uint64_t c = cost >= 16777215.0 ? 0xffffffull : (uint64_t)cost;
            const int cls = b - a <= 2 ? 4 : I.G == 1 ? 0 : I.G == 2 ? 1 : I.G == 4 ? 2 : 3;
            keys[x] = ((uint64_t)cls << 24) | (0xffffffull - c);
            vals[x] = (uint32_t)x;
            atomicAdd(&ccount[cls], 1ull);
        }
    }
    __syncthreads();
    if (threadIdx.x < JOIN_NCLS && ccount[threadIdx.x]) atomicAdd(&class_count[threadIdx.x], ccount[threadIdx.x]);
}

__global__ void k_take_vals(const uint32_t *__restrict__ vals, int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)vals[i];
}

const char *code_name(int c) {
    switch (c) {
        case E_PTR: return "row pointers decrease or exceed nnz";
        case E_IDX_RANGE: return "dimension index out of [0, m)";
        case E_IDX_ORDER: return "dimension indices not strictly increasing";
        case E_VALUE: return "value not finite and > 0";
        case E_NORM: return "row L2 norm differs from 1 by more than 1e-3 (pass APS_NORMALIZE), or exceeds 1 + 1e-3 "
                            "with APS_SUBUNIT_NORMS";
        default: return "invalid input";
    }
}

}  // namespace

aps_status build_index_device(aps_index *ix, const int64_t *indptr, const int32_t *idx, const float *val,
                              const std::vector<InstDesc> &inst_in, cudaStream_t s, const aps_tuning *tune) {
    const int k = (int)inst_in.size();
    ix->k = k;
    ix->stream = s;
    // ---- host-side layout of instances: ranks, windows, classes
    std::vector<InstDesc> inst = inst_in;
    int64_t N = 0, M = 0, nqw = 0, nwptr = 0, npw = 0;
    int32_t maxm = 1, maxn = 1, maxnw = 1;
    // tile shape per instance: G query groups per CTA from the size-bucket table (its
    // queryable column for indexes built to answer queries)
    const aps_tuning tu = tune ? *tune : tuning_current();
    const int32_t *gtab = (ix->flags & APS_QUERYABLE) ? tu.query_groups : tu.groups;
    for (int i = 0; i < k; i++) {
        InstDesc &I = inst[i];
        I.vbase = N;
        I.rbase = (int32_t)M;
        I.G = gtab[tune_bucket(I.n)];
        I.W = JOIN_WMAX / I.G;
        I.nw = I.n > 0 ? (int32_t)((I.n + I.W - 1) / I.W) : 0;
        I.packed = I.n < (1 << 24) ? 1 : 0;
        I.qwbase = nqw;
        I.wbase = nwptr;
        I.pbase = npw;
        npw += 4 * (((int64_t)I.n + 31) / 32);  // 32 codes per 16 bytes, each instance aligned
        nqw += (int64_t)I.n * I.nw;
        if (I.nw > 1) nwptr += (int64_t)I.m * (I.nw + 1);
        N += I.n;
        M += I.m;
        maxm = std::max(maxm, I.m);
        maxn = std::max(maxn, I.n);
        maxnw = std::max(maxnw, I.nw);
    }
    if (M >= (1ll << 31) || N >= (1ll << 31)) {
        set_error("too many vectors or dimensions (limit 2^31 - 1)");
        return APS_EINVAL;
    }
    ix->N = N;
    ix->M = M;
    ix->nqw = nqw;
    ix->nwptr = nwptr;
    ix->npw = npw;
    ix->maxm = maxm;
    ix->inst_h = inst;
    IndexArrays &d = ix->d;

    int64_t nnz = 0;
    APS_CUDA(cudaMemcpyAsync(&nnz, indptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    int64_t first = 0;
    APS_CUDA(cudaMemcpyAsync(&first, indptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (first != 0 || nnz < 0 || nnz >= (1ll << 31)) {
        set_error("indptr[0] must be 0 and nnz in [0, 2^31); got indptr[0]=%lld nnz=%lld",
                  (long long)first, (long long)nnz);
        return APS_EINVAL;
    }
    ix->nnz = nnz;
    for (int i = 0; i < k; i++) inst[i].ebase = 0;

    APS_TRY(d.inst.alloc((size_t)k, s));
    APS_CUDA(cudaMemcpyAsync(d.inst.p, inst.data(), sizeof(InstDesc) * k, cudaMemcpyHostToDevice, s));
    APS_TRY(d.vinst.alloc((size_t)N, s));
    APS_TRY(d.cptr.alloc((size_t)N + 1, s));
    APS_CUDA(cudaMemcpyAsync(d.cptr.p, indptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToDevice, s));
    APS_TRY(d.len.alloc((size_t)N, s));
    APS_TRY(d.mw.alloc((size_t)N, s));
    APS_TRY(d.split.alloc((size_t)N, s));
    APS_TRY(d.qsplit.alloc((size_t)N, s));
    APS_TRY(d.mwpre.alloc((size_t)N, s));
    APS_TRY(d.crank.alloc((size_t)nnz, s));
    APS_TRY(d.cval.alloc((size_t)nnz, s));
    APS_TRY(d.nnz_d.alloc((size_t)M, s));
    APS_TRY(d.mw_d.alloc((size_t)M, s));
    APS_TRY(d.mwr.alloc((size_t)M, s));
    APS_TRY(d.rank_of_dim.alloc((size_t)M, s));
    APS_TRY(d.dim_of_rank.alloc((size_t)M, s));
    APS_TRY(d.lptr.alloc((size_t)M + 1, s));

    DBuf<int32_t> erow;
    DBuf<float> vout;
    DBuf<unsigned long long> err;
    APS_TRY(erow.alloc((size_t)nnz, s));
    APS_TRY(vout.alloc((size_t)nnz, s));
    APS_TRY(err.alloc(JOIN_NCLS, s));
    APS_CUDA(cudaMemsetAsync(err.p, 0xff, sizeof(unsigned long long), s));
    APS_CUDA(cudaMemsetAsync(err.p + 1, 0, 3 * sizeof(unsigned long long), s));

    const unsigned gN = grid_for(N, T256), gE = grid_for(nnz, T256), gM = grid_for(M, T256);
    // ---- a1: validation, |x|, maxweight(x), per-dimension statistics
    k_vinst<<<gN, T256, 0, s>>>(d.inst.p, k, N, d.vinst.p);
    APS_LAUNCH_CHECK();
    k_validate<<<grid_for(N * 32, T256), T256, 0, s>>>(indptr, idx, val, d.vinst.p, d.inst.p, N, nnz, ix->flags,
                                                       erow.p, vout.p, d.len.p, d.mw.p, err.p, err.p + 2);
    APS_LAUNCH_CHECK();
    unsigned long long e3[3] = {~0ull, 0ull, 0ull};  // first error, (unused here), longest row
    APS_CUDA(cudaMemcpyAsync(e3, err.p, sizeof(e3), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    const unsigned long long e_h = e3[0], longest_row = e3[2];
    if (e_h != ~0ull) {
        long long row = (long long)(e_h >> 8);
        int code = (int)(e_h & 0xff);
        int inst_id = 0;
        for (int i = 0; i < k; i++)
            if (inst[i].vbase <= row) inst_id = i;
        if (k > 1)
            set_error("invalid input in instance %d, row %lld: %s", inst_id, row - (long long)inst[inst_id].vbase,
                      code_name(code));
        else
            set_error("invalid input at row %lld: %s", row, code_name(code));
        return APS_EINVAL;
    }
    APS_CUDA(cudaMemsetAsync(d.nnz_d.p, 0, sizeof(int32_t) * M, s));
    APS_CUDA(cudaMemsetAsync(d.mw_d.p, 0, sizeof(float) * M, s));
    if (nnz > 0 && k > 1 && maxm <= DIMSTATS_DIMS) {  // a batch of small instances: one CTA each
        const int sm = (int)(sizeof(uint32_t) * (size_t)maxm);
        APS_CUDA(cudaFuncSetAttribute(k_dimstats_inst, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        k_dimstats_inst<<<k, 1024, sm, s>>>(d.cptr.p, idx, vout.p, d.inst.p, d.nnz_d.p, d.mw_d.p);
        APS_LAUNCH_CHECK();
    } else if (nnz > 0) {
        k_dimstats<<<gE, T256, 0, s>>>(idx, vout.p, erow.p, d.vinst.p, d.inst.p, nnz, d.nnz_d.p, d.mw_d.p);
        APS_LAUNCH_CHECK();
    }
    // ---- a2: dimension ranks and rank-ordered rows
    {
        DBuf<uint64_t> keys;
        DBuf<uint32_t> vals;
        APS_TRY(keys.alloc((size_t)M, s));
        APS_TRY(vals.alloc((size_t)M, s));
        int nb = bits_for((uint64_t)maxn);
        k_rank_keys<<<gM, T256, 0, s>>>(d.nnz_d.p, d.inst.p, k, M, nb, (uint64_t)maxn, keys.p, vals.p);
        APS_LAUNCH_CHECK();
        APS_TRY(sort_pairs(keys.p, vals.p, M, nb + bits_for((uint64_t)(k - 1)), s));
        k_rank_scatter<<<gM, T256, 0, s>>>(vals.p, d.inst.p, k, M, d.mw_d.p, d.rank_of_dim.p, d.dim_of_rank.p,
                                           d.mwr.p);
        APS_LAUNCH_CHECK();
    }
    if (nnz > 0 && longest_row <= 64) {  // every row sorted inside one warp
        k_canon_rows64<<<grid_for(N * 32, T256), T256, 0, s>>>(d.cptr.p, idx, vout.p, d.vinst.p, d.inst.p,
                                                               d.rank_of_dim.p, N, d.crank.p, d.cval.p);
        APS_LAUNCH_CHECK();
    } else if (nnz > 0) {  // a global sort by (row, rank)
        DBuf<uint64_t> keys;
        DBuf<uint32_t> vals;
        APS_TRY(keys.alloc((size_t)nnz, s));
        APS_TRY(vals.alloc((size_t)nnz, s));
        int rb = bits_for((uint64_t)(maxm - 1));
        if (rb == 0) rb = 1;
        k_canon_keys<<<gE, T256, 0, s>>>(idx, erow.p, d.vinst.p, d.inst.p, d.rank_of_dim.p, nnz, rb, keys.p, vals.p);
        APS_LAUNCH_CHECK();
        APS_TRY(sort_pairs(keys.p, vals.p, nnz, rb + bits_for((uint64_t)(N - 1)), s));
        k_canon_gather<<<gE, T256, 0, s>>>(keys.p, vals.p, vout.p, nnz, (1ull << rb) - 1, d.crank.p, d.cval.p);
        APS_LAUNCH_CHECK();
    }
    // ---- a3: partial-indexing split
    APS_TRY(d.pnorm.alloc((size_t)std::max<int64_t>(N, 1), s));
    // the split also writes each row's posting keys for a4 (and counts the indexed components)
    DBuf<uint64_t> pkeys;
    DBuf<uint32_t> pvals;
    APS_TRY(pkeys.alloc((size_t)std::max<int64_t>(nnz, 1), s));
    APS_TRY(pvals.alloc((size_t)std::max<int64_t>(nnz, 1), s));
    unsigned long long *nsuf_d = err.p + 1;
    k_split<<<grid_for(N * 32, T256), T256, 0, s>>>(d.cptr.p, d.crank.p, d.cval.p, d.mwr.p, d.vinst.p, d.inst.p, N,
                                                    ix->flags, d.split.p, d.qsplit.p, d.mwpre.p, d.pnorm.p, M,
                                                    pkeys.p, pvals.p, nsuf_d);
    APS_LAUNCH_CHECK();
    // ---- a4: suffix inverted index
    {
        DBuf<uint64_t> &keys = pkeys;
        DBuf<uint32_t> &vals = pvals;
        unsigned long long nsuf_h = 0;
        APS_CUDA(cudaMemcpyAsync(&nsuf_h, nsuf_d, sizeof(nsuf_h), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        ix->nsuf = (int64_t)nsuf_h;
        if (nnz > 0) APS_TRY(sort_pairs(keys.p, vals.p, nnz, bits_for((uint64_t)M), s));
        APS_TRY(d.post.alloc((size_t)std::max<int64_t>(ix->nsuf, 1), s));
        APS_TRY(d.wptr.alloc((size_t)std::max<int64_t>(nwptr, 1), s));
        if (nwptr) APS_CUDA(cudaMemsetAsync(d.wptr.p, 0, sizeof(int32_t) * nwptr, s));
        if (ix->nsuf > 0) {
            k_post_fill<<<grid_for(ix->nsuf, T256), T256, 0, s>>>(vals.p, erow.p, d.cval.p, d.len.p, d.vinst.p,
                                                                  d.inst.p, ix->nsuf, d.post.p);
            APS_LAUNCH_CHECK();
        }
        k_lptr<<<grid_for(M + 1, T256), T256, 0, s>>>(keys.p, ix->nsuf, M, d.lptr.p);
        APS_LAUNCH_CHECK();
        if (nwptr) {
            k_wptr<<<gM, T256, 0, s>>>(d.inst.p, k, M, d.lptr.p, d.post.p, d.wptr.p);
            APS_LAUNCH_CHECK();
        }
        APS_TRY(d.crow.alloc((size_t)std::max<int64_t>(nnz, 1), s));
        APS_TRY(d.vmeta.alloc((size_t)std::max<int64_t>(N, 1), s));
        APS_TRY(d.vcand.alloc((size_t)std::max<int64_t>(N, 1), s));
        APS_TRY(d.pn4.alloc((size_t)std::max<int64_t>(ix->npw, 4), s));
        APS_CUDA(cudaMemsetAsync(d.pn4.p, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(ix->npw, 4), s));
        k_pack<<<grid_for(std::max(nnz, N), T256), T256, 0, s>>>(d.cptr.p, d.crank.p, d.cval.p, d.len.p, d.split.p,
                                                                 d.mwpre.p, d.pnorm.p, d.vinst.p, d.inst.p, N, nnz,
                                                                 d.crow.p, d.vmeta.p, d.vcand.p, d.pn4.p);
        APS_LAUNCH_CHECK();
    }
    // ---- join work list
    {
        DBuf<uint64_t> keys;
        DBuf<uint32_t> vals;
        APS_TRY(keys.alloc((size_t)std::max<int64_t>(N, 1), s));
        APS_TRY(vals.alloc((size_t)std::max<int64_t>(N, 1), s));
        unsigned long long *cc = err.p;  // reused: one counter per class
        APS_CUDA(cudaMemsetAsync(cc, 0, JOIN_NCLS * sizeof(unsigned long long), s));
        if (N > 0) {
            k_item_keys<<<grid_for(N * 32, T256), T256, 0, s>>>(d.cptr.p, d.crank.p, d.lptr.p, d.vinst.p, d.inst.p,
                                                               N, keys.p, vals.p,
                                            cc);
            APS_LAUNCH_CHECK();
            APS_TRY(sort_pairs(keys.p, vals.p, N, 27, s));  // 3 class bits + 24 cost bits
        }
        unsigned long long cnt_h[JOIN_NCLS] = {};
        APS_CUDA(cudaMemcpyAsync(cnt_h, cc, sizeof(cnt_h), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        int64_t acc = 0;
        for (int c = 0; c < JOIN_NCLS; c++) {
            ix->class_begin[c] = acc;
            acc += (int64_t)cnt_h[c];
        }
        ix->class_begin[JOIN_NCLS] = acc;
        APS_TRY(ix->items.alloc((size_t)std::max<int64_t>(acc, 1), s));
        if (acc > 0) {
            k_take_vals<<<grid_for(acc, T256), T256, 0, s>>>(vals.p, acc, ix->items.p);
            APS_LAUNCH_CHECK();
        }
    }
    APS_CUDA(cudaStreamSynchronize(s));
    return APS_OK;
}

// ------------------------------------------------------------------ external queries
namespace {

__global__ void k_q_keys(const int32_t *__restrict__ qidx, const int32_t *__restrict__ erow,
                         const int32_t *__restrict__ rank_of_dim, int64_t nnz, int rb, uint64_t *keys, uint32_t *vals) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        keys[p] = ((uint64_t)erow[p] << rb) | (uint64_t)rank_of_dim[qidx[p]];
        vals[p] = (uint32_t)p;
    }
}

__global__ void k_q_gather(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                           const float *__restrict__ vout, int64_t nnz, uint64_t rmask, int2 *crow) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        crow[q] = make_int2((int32_t)(keys[q] & rmask), __float_as_int(vout[vals[q]]));
}

// Remscore boundary of a query: the first rank-ordered component where
// sum x[i] * maxweight_i(V) reaches t (float64, as for indexed vectors).
__global__ void k_q_split(const int64_t *__restrict__ qptr, const int2 *__restrict__ crow,
                          const float *__restrict__ mwr, int64_t nq, float t, int32_t *qsplit, int4 *vmeta) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nq; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = qptr[x], b = qptr[x + 1];
        const int32_t L = (int32_t)(b - a);
        int32_t qs = L;
        double bmw = 0.0;
        for (int64_t p = a; p < b; p++) {
            bmw += (double)__int_as_float(crow[p].y) * (double)mwr[crow[p].x];
            if (bmw >= (double)t) {
                qs = (int32_t)(p - a);
                break;
            }
        }
        qsplit[x] = qs;
        vmeta[x] = make_int4((int32_t)a, L, 0, 0);
    }
}

}  // namespace

aps_status prepare_queries(const aps_index *ix, const int64_t *qptr, const int32_t *qidx, const float *qval,
                           int32_t nq, float t, uint32_t flags, cudaStream_t s, QueryArrays &qa, int64_t nnz_known) {
    const IndexArrays &d = ix->d;
    int64_t nnz = nnz_known, first = 0;
    if (nnz_known < 0) {  // the row pointers live on the device only: read their ends back
        APS_CUDA(cudaMemcpyAsync(&nnz, qptr + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaMemcpyAsync(&first, qptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
    }
    if (first != 0 || nnz < 0 || nnz >= (1ll << 31)) {
        set_error("query indptr[0] must be 0 and nnz in [0, 2^31)");
        return APS_EINVAL;
    }
    qa.nq = nq;
    qa.nnz = nnz;
    // the index's single instance describes the dimension space
    InstDesc qd = ix->inst_h[0];
    qd.vbase = 0;
    qd.n = nq;
    DBuf<InstDesc> dinst;
    DBuf<int32_t> vinst, erow, len;
    DBuf<float> vout;
    DBuf<unsigned long long> err;
    APS_TRY(dinst.alloc(1, s));
    APS_CUDA(cudaMemcpyAsync(dinst.p, &qd, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
    APS_TRY(vinst.alloc((size_t)std::max<int64_t>(nq, 1), s));
    APS_CUDA(cudaMemsetAsync(vinst.p, 0, sizeof(int32_t) * std::max<int64_t>(nq, 1), s));
    APS_TRY(erow.alloc((size_t)std::max<int64_t>(nnz, 1), s));
    APS_TRY(vout.alloc((size_t)std::max<int64_t>(nnz, 1), s));
    APS_TRY(len.alloc((size_t)std::max<int64_t>(nq, 1), s));
    APS_TRY(qa.mw.alloc((size_t)std::max<int64_t>(nq, 1), s));
    APS_TRY(err.alloc(1, s));
    APS_CUDA(cudaMemsetAsync(err.p, 0xff, sizeof(unsigned long long), s));
    if (nq > 0) {
        k_validate<<<grid_for((int64_t)nq * 32, T256), T256, 0, s>>>(qptr, qidx, qval, vinst.p, dinst.p, nq, nnz,
                                                                     flags, erow.p, vout.p, len.p, qa.mw.p, err.p,
                                                                     nullptr);
        APS_LAUNCH_CHECK();
    }
    unsigned long long e_h = ~0ull;
    APS_CUDA(cudaMemcpyAsync(&e_h, err.p, sizeof(e_h), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (e_h != ~0ull) {
        set_error("invalid query row %lld: %s", (long long)(e_h >> 8), code_name((int)(e_h & 0xff)));
        return APS_EINVAL;
    }
    APS_TRY(qa.crow.alloc((size_t)std::max<int64_t>(nnz, 1), s));
    if (nnz > 0) {
        DBuf<uint64_t> keys;
        DBuf<uint32_t> vals;
        APS_TRY(keys.alloc((size_t)nnz, s));
        APS_TRY(vals.alloc((size_t)nnz, s));
        const int rb = std::max(1, bits_for((uint64_t)(ix->maxm - 1)));
        k_q_keys<<<grid_for(nnz, T256), T256, 0, s>>>(qidx, erow.p, d.rank_of_dim.p, nnz, rb, keys.p, vals.p);
        APS_LAUNCH_CHECK();
        APS_TRY(sort_pairs(keys.p, vals.p, nnz, rb + bits_for((uint64_t)std::max(nq - 1, 0)), s));
        k_q_gather<<<grid_for(nnz, T256), T256, 0, s>>>(keys.p, vals.p, vout.p, nnz, (1ull << rb) - 1, qa.crow.p);
        APS_LAUNCH_CHECK();
    }
    APS_TRY(qa.qsplit.alloc((size_t)std::max<int64_t>(nq, 1), s));
    APS_TRY(qa.vmeta.alloc((size_t)std::max<int64_t>(nq, 1), s));
    if (nq > 0) {
        k_q_split<<<grid_for(nq, T256), T256, 0, s>>>(qptr, qa.crow.p, d.mwr.p, nq, t, qa.qsplit.p, qa.vmeta.p);
        APS_LAUNCH_CHECK();
    }
    return APS_OK;
}

}  // namespace aps
