// The inverted-index join (Alg. 2, Find-Matches, with the all-pairs-2 bounds) and the
// output stage.
//
// One persistent kernel per size class. A CTA of 1024 threads runs G query groups
// (G = 1, 2, 4, 8); each group owns a dense score array A over a window of W candidate
// ids in shared memory (the paper's all-pairs-0-array accumulator, cut into windows
// because n floats do not fit on chip). For a query x (a whole vector of the set, taken
// from a cost-ordered work list) and each window of candidates y > x:
//   1. accumulate: A[y] += x[i] * y[i] over the posting lists of x's components,
//      first over the components with remscore >= t (these may create candidates),
//      then over the rest, which only update candidates that exist (remscore);
//      entries with |y| below minsize are cut off (lists are ordered by |y| inside a
//      window, so this is a tail cut found by binary search);
//   2. verify: for every A[y] != 0, the upperbound test
//      A[y] + min(|y'|, |x|) * maxweight(x) * maxweight(y') >= t, then
//      s = A[y] + dot(x, y') with y' the unindexed prefix of y;
//      scores within a band of t are recomputed in float64 and decided there;
//   3. compact: warp ballots give each emitted pair its slot; one global reservation
//      per (x, window); pairs land in a staging buffer as (y, score) in increasing y.
// The output stage scans the per-(x, window) counts and gathers the staged runs into
// (i, j, score) arrays, which are then in (i, j) order without a sort.
#include <algorithm>
#include <cmath>

#include "index.cuh"

namespace aps {
namespace {

struct JoinParams {
    const InstDesc *inst;
    const int32_t *vinst;
    const int32_t *items;
    int64_t item_begin, item_end;
    int G;
    const int64_t *cptr;
    const int32_t *crank;
    const float *cval;
    const int32_t *len;
    const int32_t *split;
    const int32_t *qsplit;
    const float *mw;
    const float *mwpre;
    const int64_t *lptr;
    const int32_t *wptr;
    const int2 *post;
    uint32_t flags;
    int2 *stage;
    int64_t stage_cap;
    unsigned long long *stage_count;
    Segment *segs;
    int64_t seg_cap;
    unsigned long long *seg_count;
    int32_t *cntq;
    unsigned long long *counters;  // visits, candidates, verified, pairs, band
    unsigned long long *work;
};

__host__ __device__ constexpr int group_bytes(int G) {
    return 4 * (JOIN_WMAX / G)                       // A
           + 8 * (JOIN_THREADS / G + 2)              // c_pref
           + 8 * (JOIN_THREADS / G)                  // c_start
           + 4 * (JOIN_THREADS / G)                  // c_xv
           + 4 * (JOIN_RMAX / G)                     // xtab
           + 8 * 32                                  // wsum
           + 4 * 32                                  // wcnt
           + 8 * 4;                                  // broadcast
}

__device__ __forceinline__ void gsync(int G, int g, int GT) {
    if (G == 1)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// x's value at rank r: dense table for small ranks, binary search of x's rank-sorted row
// otherwise.
__device__ __forceinline__ float x_at(int r, const float *xtab, int RG, const int32_t *__restrict__ crank,
                                      const float *__restrict__ cval, int64_t xa, int xl) {
    if (r < RG) return xtab[r];
    int lo = 0, hi = xl;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (crank[xa + mid] < r) lo = mid + 1; else hi = mid;
    }
    return (lo < xl && crank[xa + lo] == r) ? cval[xa + lo] : 0.f;
}

// float64 dot product of two rank-sorted rows (used inside the decision band).
__device__ double dot64(const int32_t *__restrict__ crank, const float *__restrict__ cval, int64_t xa, int xl,
                        int64_t ya, int yl) {
    double s = 0.0;
    int p = 0, q = 0;
    while (p < xl && q < yl) {
        int a = crank[xa + p], b = crank[ya + q];
        if (a == b) {
            s += (double)cval[xa + p] * (double)cval[ya + q];
            p++;
            q++;
        } else if (a < b) {
            p++;
        } else {
            q++;
        }
    }
    return s;
}

__global__ void __launch_bounds__(JOIN_THREADS, 1) join_kernel(JoinParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int G = P.G;
    const int GT = JOIN_THREADS / G;
    const int g = threadIdx.x / GT, gt = threadIdx.x % GT;
    const int lane = gt & 31, gw = gt >> 5, NW = GT >> 5;
    const int WG = JOIN_WMAX / G, RG = JOIN_RMAX / G;
    unsigned char *base = smem + (size_t)g * group_bytes(G);
    float *A = reinterpret_cast<float *>(base);
    int64_t *c_pref = reinterpret_cast<int64_t *>(A + WG);
    int64_t *c_start = c_pref + GT + 2;
    float *c_xv = reinterpret_cast<float *>(c_start + GT);
    float *xtab = c_xv + GT;
    int64_t *wsum = reinterpret_cast<int64_t *>(xtab + RG);
    int32_t *wcnt = reinterpret_cast<int32_t *>(wsum + 32);
    int64_t *bc = reinterpret_cast<int64_t *>(wcnt + 32);
    const unsigned lt_mask = (1u << lane) - 1u;
    const bool f_minsize = !(P.flags & APS_NO_MINSIZE);
    const bool f_remscore = !(P.flags & APS_NO_REMSCORE);
    const bool f_upper = !(P.flags & APS_NO_UPPERBOUND);

    for (int i = gt; i < WG; i += GT) A[i] = 0.f;
    unsigned long long n_visits = 0, n_cand = 0, n_verified = 0, n_band = 0, n_pairs = 0;
    gsync(G, g, GT);

    for (;;) {
        gsync(G, g, GT);  // every thread is done with the previous item's broadcast slots
        if (gt == 0) bc[0] = (int64_t)atomicAdd(P.work, 1ull) + P.item_begin;
        gsync(G, g, GT);
        const int64_t it = bc[0];
        if (it >= P.item_end) break;
        const int64_t x = P.items[it];
        const InstDesc I = P.inst[P.vinst[x]];
        const int32_t lx = (int32_t)(x - I.vbase);
        const int64_t xa = P.cptr[x];
        const int32_t xl = (int32_t)(P.cptr[x + 1] - xa);
        const int32_t qs = f_remscore ? P.qsplit[x] : 0;
        const float mwx = P.mw[x];
        const float t = I.t;
        const float beta = fmaxf(1e-5f, (float)(xl + 2) * 1.1920929e-7f);  // (|x|+2) * 2^-23
        // no component reaches remscore >= t: x can create no candidate at all
        if (f_remscore ? qs >= xl : xl == 0) continue;
        int smin = 0;
        if (f_minsize && mwx > 0.f) smin = (int)ceil(((double)t - (double)beta) / ((double)mwx * 1.002));
        // dense table of x over small ranks for dot(x, y')
        for (int i = gt; i < RG; i += GT) xtab[i] = 0.f;
        gsync(G, g, GT);
        for (int c = gt; c < xl; c += GT) {
            int r = P.crank[xa + c];
            if (r < RG) xtab[r] = P.cval[xa + c];
        }
        gsync(G, g, GT);

        for (int w = (lx + 1) / I.W; w < I.nw; w++) {
            const int w0 = w * I.W;
            const int wn = min(I.W, I.n - w0);
            const int lo = max(0, lx + 1 - w0);
            // ---------------- accumulate: phase 0 creates candidates, phase 1 updates
            for (int phase = 0; phase < 2; phase++) {
                const int cb = phase == 0 ? qs : 0;
                const int ce = phase == 0 ? xl : qs;
                for (int c0 = cb; c0 < ce; c0 += GT) {
                    const int c = c0 + gt;
                    int64_t cnt = 0, st = 0;
                    float xv = 0.f;
                    if (c < ce) {
                        const int r = P.crank[xa + c];
                        const int64_t R = (int64_t)I.rbase + r;
                        xv = P.cval[xa + c];
                        int64_t ls = P.lptr[R], le = P.lptr[R + 1];
                        if (I.nw > 1) {
                            const int32_t *wp = P.wptr + I.wbase + (int64_t)r * (I.nw + 1);
                            le = ls + wp[w + 1];
                            ls = ls + wp[w];
                        }
                        if (smin > 1 && le > ls) {  // minsize: drop the tail with |y| < smin
                            int64_t a = ls, b = le;
                            while (a < b) {
                                int64_t mid = (a + b) >> 1;
                                if (P.len[I.vbase + P.post[mid].x] >= smin) a = mid + 1; else b = mid;
                            }
                            le = a;
                        }
                        cnt = le - ls;
                        st = ls;
                    }
                    // compact the non-empty components and prefix-sum their entry counts
                    const int64_t packed = (cnt << 11) | (cnt > 0 ? 1 : 0);
                    const int64_t inc = warp_incl_scan(packed, lane);
                    if (lane == 31) wsum[gw] = inc;
                    gsync(G, g, GT);
                    int64_t before = 0, total = 0;
                    for (int k = 0; k < NW; k++) {
                        int64_t s = wsum[k];
                        if (k < gw) before += s;
                        total += s;
                    }
                    const int64_t ex = before + inc - packed;
                    if (cnt > 0) {
                        const int pos = (int)(ex & 2047);
                        c_pref[pos] = ex >> 11;
                        c_start[pos] = st;
                        c_xv[pos] = xv;
                    }
                    const int ncomp = (int)(total & 2047);
                    const int64_t T = total >> 11;
                    if (gt == 0) c_pref[ncomp] = T;
                    gsync(G, g, GT);
                    n_visits += (gt == 0) ? (unsigned long long)T : 0ull;
                    // flat loop over all entries of this component batch, 128 per warp step
                    int cc = 0;
                    for (int64_t f = (int64_t)gw * 128; f < T; f += (int64_t)NW * 128) {
                        if (c_pref[cc + 1] <= f) {  // advance to the component holding f
                            int a = cc + 1, b = ncomp - 1;
                            while (a < b) {
                                int mid = (a + b) >> 1;
                                if (c_pref[mid + 1] <= f) a = mid + 1; else b = mid;
                            }
                            cc = a;
                        }
                        const bool single = c_pref[cc + 1] >= f + 128;
                        int2 ent[4];
                        float xvu[4];
                        bool ok[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int64_t e = f + u * 32 + lane;
                            ok[u] = e < T;
                            int cu = cc;
                            if (!single) {  // each compacted component has >= 1 entry
                                int a = cc, b = min(cc + 127, ncomp - 1);
                                while (a < b) {
                                    int mid = (a + b + 1) >> 1;
                                    if (c_pref[mid] <= e) a = mid; else b = mid - 1;
                                }
                                cu = a;
                            }
                            if (ok[u]) {
                                ent[u] = __ldg(&P.post[c_start[cu] + (e - c_pref[cu])]);
                                xvu[u] = c_xv[cu];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            if (!ok[u]) continue;
                            const int slot = ent[u].x - w0;
                            if (slot < lo) continue;
                            const float prod = xvu[u] * __int_as_float(ent[u].y);
                            if (phase == 0) {
                                atomicAdd(&A[slot], prod);
                            } else if (A[slot] != 0.f) {
                                atomicAdd(&A[slot], prod);
                            }
                        }
                    }
                    gsync(G, g, GT);
                }
                if (!f_remscore) break;  // single phase: every component creates
            }
            // ---------------- verify
            const int span = wn - lo;
            const int chunk = span > 0 ? (((span + NW - 1) / NW + 31) & ~31) : 0;
            const int sb0 = lo + gw * chunk;
            const int se = min(lo + (gw + 1) * chunk, wn);
            int my = 0;
            for (int sb = sb0; sb < se; sb += 32) {
                const int s = sb + lane;
                const bool valid = s < se;
                const float v = valid ? A[s] : 0.f;
                bool emit = false;
                float sc = 0.f;
                if (v != 0.f) {
                    n_cand++;
                    const int64_t gy = I.vbase + w0 + s;
                    const int32_t ys = P.split[gy];
                    bool ok = true;
                    if (ys > 0) {
                        if (f_upper) {
                            const float bound = v + (float)min(ys, xl) * mwx * P.mwpre[gy];
                            ok = bound >= t - beta;
                        }
                    } else {
                        ok = v > t - beta;
                    }
                    if (ok) {
                        sc = v;
                        const int64_t ya = P.cptr[gy];
                        if (ys > 0) {
                            n_verified++;
                            float acc = 0.f;
                            for (int k = 0; k < ys; k++) {
                                const float xv = x_at(P.crank[ya + k], xtab, RG, P.crank, P.cval, xa, xl);
                                acc = fmaf(xv, P.cval[ya + k], acc);
                            }
                            sc = v + acc;
                        }
                        if (sc >= t + beta) {
                            emit = true;
                        } else if (sc > t - beta) {
                            n_band++;
                            const double s64 = dot64(P.crank, P.cval, xa, xl, ya, P.len[gy]);
                            emit = s64 >= (double)t;
                            sc = (float)s64;
                        }
                    }
                    A[s] = emit ? sc : 0.f;
                }
                my += __popc(__ballot_sync(0xffffffffu, emit));
            }
            if (lane == 0) wcnt[gw] = my;
            gsync(G, g, GT);
            if (gt == 0) {
                int64_t tot = 0;
                for (int k = 0; k < NW; k++) {
                    int c = wcnt[k];
                    wcnt[k] = (int32_t)tot;
                    tot += c;
                }
                const int64_t qw = I.qwbase + (int64_t)lx * I.nw + w;
                P.cntq[qw] = (int32_t)tot;
                int64_t b = 0, wr = 0;
                if (tot > 0) {
                    b = (int64_t)atomicAdd(P.stage_count, (unsigned long long)tot);
                    const int64_t sid = (int64_t)atomicAdd(P.seg_count, 1ull);
                    if (b + tot <= P.stage_cap && sid < P.seg_cap) {
                        Segment S;
                        S.src = b;
                        S.qw = qw;
                        S.cnt = (int32_t)tot;
                        S.i = lx;
                        P.segs[sid] = S;
                        wr = 1;
                    }
                }
                n_pairs += (unsigned long long)tot;
                bc[1] = b;
                bc[2] = wr;
            }
            gsync(G, g, GT);
            // ---------------- compact: write emitted pairs in increasing y, clear A
            {
                const int64_t b = bc[1];
                const bool wr = bc[2] != 0;
                int64_t off = b + wcnt[gw];
                for (int sb = sb0; sb < se; sb += 32) {
                    const int s = sb + lane;
                    const bool valid = s < se;
                    const float v = valid ? A[s] : 0.f;
                    const bool emit = v != 0.f;
                    const unsigned bal = __ballot_sync(0xffffffffu, emit);
                    if (emit) {
                        if (wr) P.stage[off + __popc(bal & lt_mask)] = make_int2(w0 + s, __float_as_int(v));
                        A[s] = 0.f;
                    }
                    off += __popc(bal);
                }
            }
            gsync(G, g, GT);
        }
    }
    // flush counters (warp-reduce, one atomic per warp)
    unsigned long long v5[5] = {n_visits, n_cand, n_verified, n_pairs, n_band};
#pragma unroll
    for (int k = 0; k < 5; k++) {
        unsigned long long v = v5[k];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(&P.counters[k], v);
    }
}

__global__ void k_gather(const Segment *__restrict__ segs, int64_t nseg, const int2 *__restrict__ stage,
                         const int64_t *__restrict__ qwoff, int32_t *__restrict__ oi, int32_t *__restrict__ oj,
                         float *__restrict__ os) {
    for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const Segment S = segs[sg];
        const int64_t dst = qwoff[S.qw];
        for (int e = threadIdx.x; e < S.cnt; e += blockDim.x) {
            const int2 v = stage[S.src + e];
            oi[dst + e] = S.i;
            oj[dst + e] = v.x;
            os[dst + e] = __int_as_float(v.y);
        }
    }
}

__global__ void k_inst_offsets(const InstDesc *__restrict__ inst, int k, const int64_t *__restrict__ qwoff,
                               int64_t nqw, int64_t *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= k; i += gridDim.x * blockDim.x)
        out[i] = i < k ? qwoff[inst[i].qwbase] : qwoff[nqw];
}

}  // namespace

aps_status join_all_pairs(aps_index *ix, uint32_t flags, aps_pairs *out, std::vector<int64_t> *pair_offsets_h) {
    cudaStream_t s = ix->stream;
    IndexArrays &d = ix->d;
    const int sms = num_sms();
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; i++) APS_CUDA(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 4; i++) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    const int Gs[4] = {1, 2, 4, 8};
    // the largest requirement of the four group shapes covers every launch
    int need = 0;
    for (int c = 0; c < 4; c++) need = std::max(need, group_bytes(Gs[c]) * Gs[c]);
    APS_CUDA(cudaFuncSetAttribute(join_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, need));

    DBuf<int32_t> cntq;
    DBuf<unsigned long long> ctr;  // 0..4 counters, 5 stage count, 6 seg count, 8..11 work
    APS_TRY(cntq.alloc((size_t)std::max<int64_t>(ix->nqw, 1), s));
    APS_TRY(ctr.alloc(16, s));
    int64_t stage_cap = std::max<int64_t>({ix->hint_pairs, (int64_t)1 << 20, ix->nnz});
    int64_t seg_cap = std::max<int64_t>({ix->hint_segs, (int64_t)1 << 16, ix->nqw / 4});
    if (seg_cap > ix->nqw) seg_cap = std::max<int64_t>(ix->nqw, 1);
    DBuf<int2> stage;
    DBuf<Segment> segs;
    int64_t total_pairs = 0, total_segs = 0;
    unsigned long long ch[16];
    int reruns = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        APS_TRY(stage.alloc((size_t)stage_cap, s));
        APS_TRY(segs.alloc((size_t)seg_cap, s));
        APS_CUDA(cudaMemsetAsync(ctr.p, 0, 16 * sizeof(unsigned long long), s));
        if (ix->nqw) APS_CUDA(cudaMemsetAsync(cntq.p, 0, sizeof(int32_t) * ix->nqw, s));
        APS_CUDA(cudaEventRecord(ev[0], s));
        for (int c = 0; c < 4; c++) {
            const int64_t b = ix->class_begin[c], e = ix->class_begin[c + 1];
            if (e <= b) continue;
            JoinParams P;
            P.inst = d.inst.p;
            P.vinst = d.vinst.p;
            P.items = ix->items.p;
            P.item_begin = b;
            P.item_end = e;
            P.G = Gs[c];
            P.cptr = d.cptr.p;
            P.crank = d.crank.p;
            P.cval = d.cval.p;
            P.len = d.len.p;
            P.split = d.split.p;
            P.qsplit = d.qsplit.p;
            P.mw = d.mw.p;
            P.mwpre = d.mwpre.p;
            P.lptr = d.lptr.p;
            P.wptr = d.wptr.p;
            P.post = d.post.p;
            P.flags = flags | (ix->flags & (APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND));
            P.stage = stage.p;
            P.stage_cap = stage_cap;
            P.stage_count = ctr.p + 5;
            P.segs = segs.p;
            P.seg_cap = seg_cap;
            P.seg_count = ctr.p + 6;
            P.cntq = cntq.p;
            P.counters = ctr.p;
            P.work = ctr.p + 8 + c;
            const int64_t nitems = e - b;
            const int64_t groups_needed = (nitems + Gs[c] - 1) / Gs[c];
            const int grid = (int)std::min<int64_t>(sms, std::max<int64_t>(groups_needed, 1));
            join_kernel<<<grid, JOIN_THREADS, group_bytes(Gs[c]) * Gs[c], s>>>(P);
            APS_LAUNCH_CHECK();
        }
        APS_CUDA(cudaEventRecord(ev[1], s));
        APS_CUDA(cudaMemcpyAsync(ch, ctr.p, sizeof(ch), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        total_pairs = (int64_t)ch[5];
        total_segs = (int64_t)ch[6];
        if (total_pairs <= stage_cap && total_segs <= seg_cap) break;
        // the staging buffers were too small: grow to the exact need and run again
        reruns++;
        stage_cap = std::max<int64_t>(total_pairs, 1);
        seg_cap = std::max<int64_t>(total_segs, 1);
        if (attempt == 2) {
            set_error("pair staging overflow persisted");
            return APS_EOVERFLOW;
        }
    }
    ix->hint_pairs = total_pairs + total_pairs / 16 + 1024;
    ix->hint_segs = total_segs + total_segs / 16 + 1024;
    APS_CUDA(cudaEventRecord(ev[3], s));

    // ---------------- output: scan counts, gather runs into (i, j, score)
    DBuf<int64_t> qwoff;
    APS_TRY(qwoff.alloc((size_t)ix->nqw + 1, s));
    APS_TRY(scan_exclusive(cntq.p, qwoff.p, ix->nqw, s));
    const int64_t npairs = total_pairs;
    PairsAlloc *pa = new PairsAlloc();
    pa->stream = s;
    const size_t bytes = (size_t)std::max<int64_t>(npairs, 1) * 12 + 256;
    aps_status st = dalloc(&pa->block, bytes, s);
    if (st != APS_OK) {
        delete pa;
        return st;
    }
    char *blk = static_cast<char *>(pa->block);
    int32_t *oi = reinterpret_cast<int32_t *>(blk);
    int32_t *oj = reinterpret_cast<int32_t *>(blk + (((size_t)npairs * 4 + 127) & ~(size_t)127));
    float *os = reinterpret_cast<float *>(blk + 2 * (((size_t)npairs * 4 + 127) & ~(size_t)127));
    if (total_segs > 0) {
        const unsigned grid = (unsigned)std::min<int64_t>(total_segs, (int64_t)sms * 32);
        k_gather<<<grid, 256, 0, s>>>(segs.p, total_segs, stage.p, qwoff.p, oi, oj, os);
        APS_LAUNCH_CHECK();
    }
    if (pair_offsets_h) {
        DBuf<int64_t> offs;
        APS_TRY(offs.alloc((size_t)ix->k + 1, s));
        k_inst_offsets<<<grid_for(ix->k + 1, 256), 256, 0, s>>>(d.inst.p, ix->k, qwoff.p, ix->nqw, offs.p);
        APS_LAUNCH_CHECK();
        pair_offsets_h->assign((size_t)ix->k + 1, 0);
        APS_CUDA(cudaMemcpyAsync(pair_offsets_h->data(), offs.p, sizeof(int64_t) * (ix->k + 1),
                                 cudaMemcpyDeviceToHost, s));
    }
    APS_CUDA(cudaEventRecord(ev[2], s));
    APS_CUDA(cudaEventSynchronize(ev[2]));
    float ms_join = 0, ms_sort = 0;
    cudaEventElapsedTime(&ms_join, ev[0], ev[1]);
    cudaEventElapsedTime(&ms_sort, ev[3], ev[2]);
    aps_stats &S = ix->stats;
    S.visits = (int64_t)ch[0];
    S.candidates = (int64_t)ch[1];
    S.verified = (int64_t)ch[2];
    S.pairs = (int64_t)ch[3];
    S.band = (int64_t)ch[4];
    S.reruns = reruns;
    S.ms_join = ms_join;
    S.ms_sort = ms_sort;
    S.evaluations = 0;
    for (const InstDesc &I : ix->inst_h) S.evaluations += (int64_t)I.n * (I.n - 1) / 2;
    out->count = npairs;
    out->i = oi;
    out->j = oj;
    out->score = os;
    out->on_device = 1;
    out->_reserved = 0;
    out->_priv = pa;
    return APS_OK;
}

void pairs_release(aps_pairs *p) {
    if (!p || !p->_priv) return;
    PairsAlloc *pa = static_cast<PairsAlloc *>(p->_priv);
    if (--pa->refs <= 0) {
        if (pa->on_device)
            dfree(pa->block, pa->stream);
        else
            cudaFreeHost(pa->block);
        delete pa;
    }
    p->_priv = nullptr;
    p->i = p->j = nullptr;
    p->score = nullptr;
    p->count = 0;
}

// Copy device pairs into one pinned host allocation (replacing the device one).
aps_status pairs_to_host(aps_pairs *p, cudaStream_t s) {
    if (!p->on_device) return APS_OK;
    PairsAlloc *pa = new PairsAlloc();
    pa->on_device = 0;
    pa->stream = s;
    const size_t n = (size_t)p->count;
    cudaError_t e = cudaMallocHost(&pa->block, std::max<size_t>(n, 1) * 12);
    if (e != cudaSuccess) {
        delete pa;
        return cuda_status(e, "cudaMallocHost", __FILE__, __LINE__);
    }
    char *blk = static_cast<char *>(pa->block);
    int32_t *hi = reinterpret_cast<int32_t *>(blk);
    int32_t *hj = reinterpret_cast<int32_t *>(blk + n * 4);
    float *hs = reinterpret_cast<float *>(blk + n * 8);
    if (n) {
        APS_CUDA(cudaMemcpyAsync(hi, p->i, n * 4, cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaMemcpyAsync(hj, p->j, n * 4, cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaMemcpyAsync(hs, p->score, n * 4, cudaMemcpyDeviceToHost, s));
    }
    APS_CUDA(cudaStreamSynchronize(s));
    pairs_release(p);
    p->count = (int64_t)n;
    p->i = hi;
    p->j = hj;
    p->score = hs;
    p->on_device = 0;
    p->_priv = pa;
    return APS_OK;
}

}  // namespace aps
