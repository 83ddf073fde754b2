// The inverted-index join (Alg. 2, Find-Matches, with the all-pairs-2 bounds) and the
// output stage.
//
// One persistent launch takes every size class in turn. A CTA of 1024 threads runs G
// query groups (G = 1, 2, 4, 8); each group owns a dense score array A over a window of W
// candidate ids in shared memory (the paper's all-pairs-0-array accumulator, cut into
// windows because n floats do not fit on chip). For a query x (a whole vector of the set, taken
// from a cost-ordered work list) and each window of candidates y > x:
//   1. accumulate: A[y] += x[i] * y[i] over the posting lists of x's components,
//      first over the components with remscore >= t (these may create candidates), then
//      over the rest, which only update candidates that exist (remscore); entries with |y|
//      below minsize are skipped using the size class stored in the entry. A holds 32-bit
//      fixed-point sums (products rounded up to multiples of 2^-30, so a creating product
//      is at least one unit), so its updates are native integer shared-memory atomics. A
//      creating update that finds its slot still zero (a plain read before the add) also
//      sets the slot's bit in a bitmap of candidates: the first update of a slot always
//      does, so every candidate is marked, at one bitmap update per candidate rather than
//      per entry. Lists are in id order, so a warp's 32 lanes add into 32 increasing slots;
//   2. verify: each warp walks its share of the bitmap and takes the marked slots in slot
//      order, one candidate per lane: A[y] + ||y'||_2 < t rejects cheaply, then the
//      upperbound test A[y] + min(|y'|, |x|) * maxweight(x) * maxweight(y') >= t, then
//      s = A[y] + dot(x, y') with y' the unindexed prefix of y; scores within a band of
//      t are recomputed in float64 and decided there;
//   3. compact: warp ballots give each emitted pair its slot; the window's run comes from
//      a staging slab the group reserves in bulk; pairs land as (y, score) in increasing
//      y and the run is recorded at its (x, window) slot.
// The output stage scans the per-(x, window) counts and gathers the staged runs into
// (i, j, score) arrays, which are then in (i, j) order without a sort.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "index.cuh"

namespace aps {
namespace {

std::atomic<int64_t> g_stage_hint{0};
std::atomic<int64_t> g_stage_cap_once{0};  // test hook: staging room of the next self-join

struct JoinParams {
    const InstDesc *inst;
    const int32_t *vinst;
    const int32_t *items;
    // classes, taken in order by one persistent launch: class c is the work-list range
    // [cls_begin[c], cls_begin[c + 1]) run with cls_G[c] query groups per CTA, or, when
    // cls_G[c] is 0, one warp per vector with one or two components
    int ncls;
    int cls_G[JOIN_NCLS];
    int64_t cls_begin[JOIN_NCLS + 1];
    const int2 *crow;    // rank-ordered rows {rank, value}
    const int4 *vmeta;   // {row offset, |x|, |x'|, maxweight(x')}
    const int4 *vcand;   // {row offset, |y'|, maxweight(y'), ||y'||_2 bound}
    const uint32_t *pn4; // 4-bit ||y'||_2 codes, eight per word (instance I from word I.pbase)
    // dimension-block items (the vertical split with local pruning, Sec. 5.1): iblk[it] >= 0
    // makes work item it one of nblk blocks of the vector items[it]; null: none
    const int8_t *iblk;
    int nblk;
    unsigned long long *sp_key;    // pairs found by block items: local x * n + local y
    uint32_t *sp_score;            // their float32 scores (bits)
    unsigned long long *sp_count;  // pairs reserved in sp_key / sp_score
    int64_t sp_cap;
    const int32_t *qsplit;
    const float *mw;
    const int64_t *lptr;
    const int32_t *wptr;
    const int2 *post;
    uint32_t flags;
    int2 *stage;
    int64_t stage_cap;
    unsigned long long *stage_count;  // staging slots handed out (in slabs of stage_slab)
    int64_t stage_slab;
    Segment *segs;                    // [slots]: the run of slot qw
    int32_t *cntq;
    unsigned long long *counters;  // visits, candidates, verified, pairs, band; [6] entries read
    unsigned long long *work;       // [ncls] work-list cursors
    int2 *scratch;                  // per-warp lists of emitted pairs, JOIN_ECAP each
    // query mode: items are external query rows matched against every indexed vector
    int qmode;
    const int2 *qcrow;    // query rows over the index's ranks
    const int4 *qvmeta;   // {row offset, |q|, 0, 0}
    const int32_t *qqsplit;
    const float *qmw;
    float qt;
    int qnw;              // windows of the index: query-mode items are (query, window) pairs
};

constexpr int NWARPS = JOIN_THREADS / 32;

__host__ __device__ constexpr int group_bytes(int G) {
    return 4 * (JOIN_WMAX / G)                       // A
           + 4 * (JOIN_WMAX / G / 8)                 // the window's 4-bit ||y'||_2 codes
           + 8 * (JOIN_THREADS / G)                  // c_start
           + 4 * (JOIN_THREADS / G)                  // c_cnt
           + 4 * (JOIN_THREADS / G + 4)              // c_ch0
           + 4 * (JOIN_THREADS / G)                  // c_xv
           + 4 * (JOIN_RMAX / G)                     // xtab
           + 8 * (JOIN_XCAP / G)                     // x's row
           + 4 * (JOIN_WMAX / G / 32)                // bitmap of the window's candidates
           + 8 * 32                                  // wsum
           + 4 * 32                                  // wcnt
           + 8 * 8;                                  // broadcast and the staging slab
}

// every class layout of a CTA plus the kernel's per-warp counters (static shared memory)
// within the 227 KB a CTA can opt into on this part
constexpr int JOIN_SMEM_LIMIT = 232448;
static_assert(group_bytes(1) * 1 + NWARPS * 6 * 8 <= JOIN_SMEM_LIMIT, "G = 1 layout too large");
static_assert(group_bytes(2) * 2 + NWARPS * 6 * 8 <= JOIN_SMEM_LIMIT, "G = 2 layout too large");
static_assert(group_bytes(4) * 4 + NWARPS * 6 * 8 <= JOIN_SMEM_LIMIT, "G = 4 layout too large");
static_assert(group_bytes(8) * 8 + NWARPS * 6 * 8 <= JOIN_SMEM_LIMIT, "G = 8 layout too large");

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

__device__ __forceinline__ int warp_excl_scan_int(int v, int lane, int *total) {
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// x's value at rank r: dense table for small ranks, binary search of x's rank-ordered row
// otherwise.
__device__ __noinline__ float x_at_search(int r, const int2 *__restrict__ xrow, int xl) {
    int lo = 0, hi = xl;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (xrow[mid].x < r) lo = mid + 1; else hi = mid;
    }
    if (lo < xl) {
        const int2 e = xrow[lo];
        if (e.x == r) return __int_as_float(e.y);
    }
    return 0.f;
}

// x's value at rank r: dense table for small ranks, then a binary search of x's row held
// in shared memory (xr, xs entries; xs = 0 when the row did not fit), else in global memory.
__device__ __forceinline__ float x_at(int r, const float *xtab, int RG, const int2 *xr, int xs,
                                      const int2 *__restrict__ xrow, int xl) {
    if (r < RG) return xtab[r];
    if (xs == 0) return x_at_search(r, xrow, xl);
    int lo = 0, hi = xs;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (xr[mid].x < r) lo = mid + 1; else hi = mid;
    }
    return (lo < xs && xr[lo].x == r) ? __int_as_float(xr[lo].y) : 0.f;
}

// The accumulation of one warp over chunks [ch, che) of the current component batch
// (Alg. 2's A[y] += x[i] * y[i]). Chunk ch of component cc covers entries
// (ch - c_ch0[cc]) * 128 .. + 127 of that component's segment, and no further than its end.
// Each product is rounded up to a multiple of 2^-30 (so a creating product is at least one
// unit and its slot becomes non-zero); CREATE: the component may create candidates, and an
// add that found its slot zero marks the slot in bm (the first add to a slot always finds
// it zero, so every candidate is marked; a few concurrent first adds mark it again, which
// is harmless); otherwise it only adds where A is already non-zero (remscore). FIRST: the
// window holds ids at or below x's (slots below lo are skipped).
// Asynchronous 16-byte global -> shared copy (cp.async, completes out of band) and waits.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A thread's work counters, 32-bit: folded (warp-reduced) into its warp's 64-bit totals in
// shared memory after every item, so no 64-bit register pair stays live across the loops.
struct Ctr {
    uint32_t visits = 0, cand = 0, verified = 0, pairs = 0, band = 0, read = 0;
};
__device__ __forceinline__ void ctr_flush(Ctr &c, unsigned long long *wtot, const int lane) {
    uint32_t v[6] = {c.visits, c.cand, c.verified, c.pairs, c.band, c.read};
#pragma unroll
    for (int k = 0; k < 6; k++) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) wtot[k] += v[k];
    }
    c = Ctr();
}

// One 128-entry chunk of a segment: entries off .. off + 127 of seg[0, cnt), lane l taking
// off + l, off + l + 32, ... (see walk_chunks).
template <bool CREATE, bool FIRST>
__device__ __forceinline__ void walk_chunk(const int2 *__restrict__ seg, const int cnt, const int off, const float cxv,
                                           uint32_t *A, uint32_t *bm, const uint32_t smin_tag, const int32_t idmask,
                                           const int w0, const int lo, const int lane, uint32_t &nv) {
    const int rem = cnt - off - lane;  // entries from this lane's first one to the segment's end
    const int2 *pp = seg + off + lane;
    int2 ent[4];
#pragma unroll
    for (int u = 0; u < 4; u++) ent[u] = u * 32 < rem ? __ldg(pp + u * 32) : make_int2(0, 0);
#pragma unroll
    for (int u = 0; u < 4; u++) {
        if (u * 32 >= rem || (uint32_t)ent[u].x < smin_tag) continue;  // past the end; minsize
        const int slot = (ent[u].x & idmask) - w0;
        if (FIRST && slot < lo) continue;
        nv++;  // an entry Alg. 2 visits: y after x, |y| >= minsize
        const uint32_t q = __float2uint_ru(cxv * __int_as_float(ent[u].y));
        const uint32_t old = A[slot];
        if (CREATE) {
            atomicAdd(&A[slot], q);
            if (old == 0u) atomicOr(&bm[slot >> 5], 1u << (slot & 31));
        } else if (old != 0u) {
            atomicAdd(&A[slot], q);
        }
    }
}

// The accumulation of one warp over chunks [ch, che) of the current component batch
// (Alg. 2's A[y] += x[i] * y[i]), the components' segments in shared memory. Chunk ch of
// component cc covers entries (ch - c_ch0[cc]) * 128 .. + 127 of that component's segment,
// and no further than its end. Each product is rounded up to a multiple of 2^-30 (so a
// creating product is at least one unit and its slot becomes non-zero); CREATE: the
// component may create candidates, and an add that found its slot zero marks the slot in bm
// (the first add to a slot always finds it zero, so every candidate is marked; a few
// concurrent first adds mark it again, which is harmless); otherwise it only adds where A
// is already non-zero (remscore). FIRST: the window holds ids at or below x's (slots below
// lo are skipped).
template <bool CREATE, bool FIRST>
__device__ __forceinline__ void walk_chunks(int ch, const int che, int cc, const int64_t *c_start,
                                            const int32_t *c_cnt, const int32_t *c_ch0, const float *c_xv,
                                            const int2 *__restrict__ post, uint32_t *A, uint32_t *bm,
                                            const uint32_t smin_tag, const int32_t idmask, const int w0, const int lo,
                                            const int lane, uint32_t &n_visits) {
    uint32_t nv = 0;
    const int2 *seg = post + c_start[cc];
    int cnt = c_cnt[cc], cch0 = c_ch0[cc], cnext = c_ch0[cc + 1];
    float cxv = c_xv[cc] * 1073741824.f;  // x's value scaled by 2^30 (exact)
    for (; ch < che; ch++) {
        if (ch >= cnext) {
            cc++;
            seg = post + c_start[cc];
            cnt = c_cnt[cc];
            cch0 = cnext;
            cnext = c_ch0[cc + 1];
            cxv = c_xv[cc] * 1073741824.f;
        }
        walk_chunk<CREATE, FIRST>(seg, cnt, (ch - cch0) << 7, cxv, A, bm, smin_tag, idmask, w0, lo, lane, nv);
    }
    n_visits += nv;
}

// The same with the (at most 32) components of a short x held in registers, lane c holding
// component c: its segment start st, length cnt, first chunk ch0 and x's value xv.
template <bool CREATE, bool FIRST>
__device__ __forceinline__ void walk_chunks_r(int ch, const int che, int cc, const int64_t st, const int cnt_l,
                                              const int ch0_l, const float xv_l, const int2 *__restrict__ post,
                                              uint32_t *A, uint32_t *bm, const uint32_t smin_tag, const int32_t idmask,
                                              const int w0, const int lo, const int lane, uint32_t &n_visits) {
    uint32_t nv = 0;
    const int2 *seg = post + __shfl_sync(0xffffffffu, st, cc);
    int cnt = __shfl_sync(0xffffffffu, cnt_l, cc), cch0 = __shfl_sync(0xffffffffu, ch0_l, cc);
    float cxv = __shfl_sync(0xffffffffu, xv_l, cc) * 1073741824.f;
    for (; ch < che; ch++) {
        while (ch >= cch0 + ((cnt + 127) >> 7)) {  // the next component with entries
            cc++;
            seg = post + __shfl_sync(0xffffffffu, st, cc);
            cnt = __shfl_sync(0xffffffffu, cnt_l, cc);
            cch0 = __shfl_sync(0xffffffffu, ch0_l, cc);
            cxv = __shfl_sync(0xffffffffu, xv_l, cc) * 1073741824.f;
        }
        walk_chunk<CREATE, FIRST>(seg, cnt, (ch - cch0) << 7, cxv, A, bm, smin_tag, idmask, w0, lo, lane, nv);
    }
    n_visits += nv;
}

// dot(x, y') over the |y'| leading (unindexed) entries of y's rank-ordered row, by one
// lane (short prefixes): two entries per step.
__device__ __forceinline__ float dot_prefix(const int2 *__restrict__ yr, int ys, const float *xtab, int RG,
                                           const int2 *xr, int xs, const int2 *__restrict__ xrow, int xl) {
    float acc = 0.f;
    int k = 0;
    for (; k + 2 <= ys; k += 2) {
        const int2 e0 = __ldg(yr + k), e1 = __ldg(yr + k + 1);
        acc = fmaf(x_at(e0.x, xtab, RG, xr, xs, xrow, xl), __int_as_float(e0.y), acc);
        acc = fmaf(x_at(e1.x, xtab, RG, xr, xs, xrow, xl), __int_as_float(e1.y), acc);
    }
    if (k < ys) {
        const int2 e0 = __ldg(yr + k);
        acc = fmaf(x_at(e0.x, xtab, RG, xr, xs, xrow, xl), __int_as_float(e0.y), acc);
    }
    return acc;
}

// First position in [a, b) of a posting list (ids increasing) whose id exceeds lx, or b
// when none does: a 32-way search by the whole warp (each step probes 32 evenly spaced
// entries and keeps the one gap that holds the answer).
__device__ __forceinline__ int64_t first_after(const int2 *__restrict__ post, int64_t a, int64_t b, const int32_t lx,
                                               const int32_t idmask, const int lane) {
    while (b - a > 32) {
        const int64_t step = (b - a + 31) >> 5;
        const int64_t pos = a + (int64_t)lane * step;
        const bool past = pos >= b || (__ldg(&post[pos].x) & idmask) > lx;
        const unsigned m = __ballot_sync(0xffffffffu, past);
        if (m & 1u) return a;  // the range's first entry is already after x
        if (m == 0u) {
            a += 31 * step + 1;  // every probe at or before x: the answer lies after the last one
        } else {
            const int f = __ffs(m) - 1;  // probe f is past x, probe f - 1 is not
            b = min(b, a + (int64_t)f * step);
            a += (int64_t)(f - 1) * step + 1;
        }
    }
    const int64_t pos = a + lane;
    const unsigned m = __ballot_sync(0xffffffffu, pos < b && (__ldg(&post[pos].x) & idmask) > lx);
    return m ? a + (__ffs(m) - 1) : b;
}

// The part of a posting list after x: [first, end) of list rank r of instance I (the
// search starts in the window of x's successor, whose part of the list holds the answer
// or ends right before it).
__device__ __forceinline__ void list_after(const JoinParams &P, const InstDesc &I, const int r, const int32_t lx,
                                           const int wf, const int32_t idmask, const int lane, int64_t &first,
                                           int64_t &end) {
    const int64_t R = (int64_t)I.rbase + r;
    const int64_t ls = P.lptr[R];
    end = P.lptr[R + 1];
    int64_t a = ls, b = end;
    if (I.nw > 1) {
        const int32_t *wp = P.wptr + I.wbase + (int64_t)r * (I.nw + 1);
        a = ls + wp[wf];
        b = ls + wp[wf + 1];
    }
    first = first_after(P.post, a, b, lx, idmask, lane);
}

// Number of the 32 values v held by the lanes (increasing with the lane, padded with
// INT_MAX) that are below key (LE: at or below key), by halving over the lanes.
template <bool LE>
__device__ __forceinline__ int count_below(const int v, const int key) {
    int c = 0;
#pragma unroll
    for (int h = 16; h; h >>= 1) {
        const int w = __shfl_sync(0xffffffffu, v, c + h - 1);
        if (LE ? w <= key : w < key) c += h;
    }
    const int w = __shfl_sync(0xffffffffu, v, 31);
    if (c == 31 && (LE ? w <= key : w < key)) c = 32;
    return c;
}

// The vectors with one or two components (Alg. 2 for |x| <= 2), one warp per vector, no
// accumulator and no windows.
//   |x| = 1 (rank r, value x0): every entry (y, w) of r's list with y after x and
//   |y| >= minsize is a candidate whose accumulated score x0 * w is its whole score (x has
//   no other component, and dot(x, y') = 0 since r lies in y's indexed part).
//   |x| = 2 (ranks r0 < r1, values x0, x1): the two lists after x are merged by id, 32
//   entries at a time. An id on both lists scores x0 * w0 + x1 * w1 (both ranks in y's
//   indexed part, so y's prefix holds neither); an id on r0's list alone scores x0 * w0
//   (y has no r1: it is not in the indexed part, and the prefix ranks lie below r0), and is
//   a candidate only if r0 may create (remscore); an id on r1's list alone scores
//   x1 * w1 + x0 * y[r0], where y[r0] can only sit in y's unindexed prefix (looked up there
//   unless the ||y'||_2 bound already rules the pair out).
// Each candidate is decided like the windowed path (float32 outside a band of beta around
// t, the exact float64 sum of the products inside it). The matches, in increasing y, go to
// the warp's scratch list and are then copied as x's run in its first window's slot, from
// a staging slab the warp reserves in bulk; a vector with more matches than the scratch
// list holds is streamed a second time, writing them there directly.
__device__ __forceinline__ void stream_short(const JoinParams &P, unsigned long long *work, const int64_t item_begin,
                                          const int64_t item_end, const bool f_minsize, const bool f_remscore,
                                          unsigned long long *wtot) {
    const int lane = threadIdx.x & 31;
    Ctr ct;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t wslab = max((int64_t)32, P.stage_slab / 8);
    int2 *const elist = P.scratch + ((size_t)blockIdx.x * NWARPS + (threadIdx.x >> 5)) * JOIN_ECAP;
    int64_t sb = 0, su = 0, ss = 0;  // this warp's staging slab: base, used, size
    for (;;) {
        ctr_flush(ct, wtot, lane);
        unsigned long long iw = 0;
        if (lane == 0) iw = atomicAdd(work, 1ull);
        const int64_t it = (int64_t)__shfl_sync(0xffffffffu, iw, 0) + item_begin;
        if (it >= item_end) break;
        const int64_t x = P.items[it];
        const InstDesc I = P.inst[P.vinst[x]];
        const int32_t lx = (int32_t)(x - I.vbase);
        const int4 xm = P.vmeta[x];
        const int xl = xm.y;  // 1 or 2
        const int qs = f_remscore ? P.qsplit[x] : 0;
        if (qs >= xl) continue;  // remscore < t from the first component on: no candidate
        const int2 xe0 = P.crow[xm.x];
        const int2 xe1 = xl == 2 ? P.crow[xm.x + 1] : make_int2(0, 0);
        const float x0 = __int_as_float(xe0.y), x1 = __int_as_float(xe1.y);
        const float t = I.t;
        const float beta = fmaxf(1e-5f, (float)(xl + 2) * 1.1920929e-7f);  // (|x| + 2) * 2^-23
        const float mwx = P.mw[x];
        int smin = 0;  // minsize, bounded as in the windowed path
        if (f_minsize && I.packed && mwx > 0.f)
            smin = (int)ceilf(fminf(__fdiv_rd(__fsub_rd(t, beta), __fmul_ru(mwx, 1.0020001f)), 255.f));
        const uint32_t smin_tag = (uint32_t)max(smin, 0) << 24;
        const int32_t idmask = I.packed ? 0x00ffffff : 0x7fffffff;
        const int wf = (lx + 1) / I.W;  // the window of x's successor
        int64_t f0, e0, f1 = 0, e1 = 0;
        list_after(P, I, xe0.x, lx, wf, idmask, lane, f0, e0);
        if (xl == 2) list_after(P, I, xe1.x, lx, wf, idmask, lane, f1, e1);
        if (lane == 0) ct.read += (uint32_t)((e0 - f0) + (e1 - f1));
        // pass 0: count the matches, the first JOIN_ECAP into the scratch list; pass 1 (only
        // when there were more): write them all into the reserved run
        int cnt = 0;
        int64_t dst = 0;
        bool wr = false;
        for (int pass = 0; pass < 2; pass++) {
            int k = 0;  // matches so far
            if (xl == 1) {
                for (int64_t p0 = f0; p0 < e0; p0 += 128) {
                    int2 e[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int64_t p = p0 + u * 32 + lane;
                        e[u] = p < e0 ? __ldg(&P.post[p]) : make_int2(0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int64_t p = p0 + u * 32 + lane;
                        bool m = false;
                        float sc = 0.f;
                        if (p < e0 && (uint32_t)e[u].x >= smin_tag) {
                            if (pass == 0) { ct.visits++; ct.cand++; }
                            sc = x0 * __int_as_float(e[u].y);
                            if (sc >= t + beta) {
                                m = true;
                            } else if (sc > t - beta) {  // inside the band: the exact product decides
                                const double ex = (double)x0 * (double)__int_as_float(e[u].y);
                                if (pass == 0) ct.band++;
                                m = ex >= (double)t;
                                sc = (float)ex;
                            }
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, m);
                        if (m) {
                            const int at = k + __popc(bal & lt_mask);
                            const int2 v2 = make_int2(e[u].x & idmask, __float_as_int(sc));
                            if (pass == 1) P.stage[dst + at] = v2;
                            else if (at < JOIN_ECAP) elist[at] = v2;
                        }
                        k += __popc(bal);
                    }
                }
            } else {
                // merge of the two lists after x, 32 merged entries per step: lane l holds
                // entry i + l of r0's list (a) and entry j + l of r1's list (b); an entry's
                // place in the merged order is its lane plus the other list's entries below
                // it (ties: a first, so an id on both lists gives a then b, adjacent)
                const int64_t n0 = e0 - f0, n1 = e1 - f1;
                int64_t i = 0, j = 0;
                const bool create0 = qs == 0;  // r0 may create candidates (remscore >= t)
                while (i < n0 || j < n1) {
                    const bool va = i + lane < n0, vb = j + lane < n1;
                    const int2 ea = va ? __ldg(&P.post[f0 + i + lane]) : make_int2(0x7fffffff, 0);
                    const int2 eb = vb ? __ldg(&P.post[f1 + j + lane]) : make_int2(0x7fffffff, 0);
                    const int ida = va ? (ea.x & idmask) : 0x7fffffff;
                    const int idb = vb ? (eb.x & idmask) : 0x7fffffff;
                    const int nb = count_below<false>(idb, ida);  // b entries below a
                    const int na = count_below<true>(ida, idb);   // a entries at or below b
                    const int ra = lane + nb, rb = lane + na;       // places in the merged order
                    const bool ina = va && ra < 32, inb = vb && rb < 32;
                    const float wbd = __int_as_float(__shfl_sync(0xffffffffu, eb.y, nb & 31));
                    // (every lane takes part in the shuffles; their results are used where valid)
                    const int idb_nb = __shfl_sync(0xffffffffu, idb, nb & 31);
                    const int ida_na = __shfl_sync(0xffffffffu, ida, (na - 1) & 31);
                    const bool dupa = va && nb < 32 && idb_nb == ida;
                    const bool dupb = vb && na > 0 && ida_na == idb;
                    const int ca = __popc(__ballot_sync(0xffffffffu, ina));
                    int cb = __popc(__ballot_sync(0xffffffffu, inb));
                    // an id on both lists whose a entry closes the step: its b entry goes too
                    {
                        const bool nd = __shfl_sync(0xffffffffu, dupb, cb & 31), nv2 = __shfl_sync(0xffffffffu, vb, cb & 31);
                        const int nna = __shfl_sync(0xffffffffu, na, cb & 31);
                        if (cb < 32 && nv2 && nd && nna <= ca) cb++;
                    }
                    // candidates: a entries (on both lists, or r0 may create), b entries alone
                    bool ma = false, mb = false;
                    float sa = 0.f, sbs = 0.f;
                    if (ina && (uint32_t)ea.x >= smin_tag) {
                        if (pass == 0) ct.visits += dupa ? 2u : 1u;  // the b entry of a shared id visits too
                        if (dupa || create0) {
                            if (pass == 0) ct.cand++;
                            const float wa = __int_as_float(ea.y), wb = dupa ? wbd : 0.f;
                            sa = fmaf(x1, wb, x0 * wa);
                            if (sa >= t + beta) {
                                ma = true;
                            } else if (sa > t - beta) {
                                const double ex = (double)x0 * (double)wa + (double)x1 * (double)wb;
                                if (pass == 0) ct.band++;
                                ma = ex >= (double)t;
                                sa = (float)ex;
                            }
                        }
                    }
                    if (inb && !dupb && (uint32_t)eb.x >= smin_tag) {
                        if (pass == 0) { ct.visits++; ct.cand++; }
                        const float wb = __int_as_float(eb.y);
                        const float s1 = x1 * wb;
                        float y0 = 0.f;
                        // y[r0] <= 1 + 1e-3 (the norm tolerance): most pairs stop here, unloaded
                        bool look = s1 + x0 * 1.0011f > t - beta;
                        int4 yc = make_int4(0, 0, 0, 0);  // {row offset, |y'|, ., ||y'||_2 bound}
                        if (look) {
                            yc = __ldg(&P.vcand[I.vbase + idb]);
                            look = yc.y > 0 && s1 + x0 * __int_as_float(yc.w) > t - beta;
                        }
                        if (look) {  // r0 in y's unindexed prefix (ranks increasing)?
                            if (pass == 0) ct.verified++;
                            for (int q = 0; q < yc.y; q++) {
                                const int2 ye = __ldg(&P.crow[yc.x + q]);
                                if (ye.x >= xe0.x) {
                                    if (ye.x == xe0.x) y0 = __int_as_float(ye.y);
                                    break;
                                }
                            }
                        }
                        sbs = fmaf(x0, y0, s1);
                        if (sbs >= t + beta) {
                            mb = true;
                        } else if (sbs > t - beta) {
                            const double ex = (double)x0 * (double)y0 + (double)x1 * (double)wb;
                            if (pass == 0) ct.band++;
                            mb = ex >= (double)t;
                            sbs = (float)ex;
                        }
                    }
                    // matches in merged order: a bit per place
                    const unsigned mm = __reduce_or_sync(0xffffffffu, (ma ? 1u << ra : 0u) | (mb ? 1u << rb : 0u));
                    if (ma) {  // (a lane may hold a match in both lists)
                        const int at = k + __popc(mm & ((1u << ra) - 1u));
                        const int2 v2 = make_int2(ida, __float_as_int(sa));
                        if (pass == 1) P.stage[dst + at] = v2;
                        else if (at < JOIN_ECAP) elist[at] = v2;
                    }
                    if (mb) {
                        const int at = k + __popc(mm & ((1u << rb) - 1u));
                        const int2 v2 = make_int2(idb, __float_as_int(sbs));
                        if (pass == 1) P.stage[dst + at] = v2;
                        else if (at < JOIN_ECAP) elist[at] = v2;
                    }
                    k += __popc(mm);
                    i += ca;
                    j += cb;
                }
            }
            if (pass == 0) {
                cnt = k;
                if (cnt == 0) break;
                if (su + cnt > ss) {  // a new slab: one global atomic per slab
                    const int64_t want = max(wslab, (int64_t)cnt);
                    unsigned long long bw = 0;
                    if (lane == 0) bw = atomicAdd(P.stage_count, (unsigned long long)want);
                    sb = (int64_t)__shfl_sync(0xffffffffu, bw, 0);
                    su = 0;
                    ss = want;
                }
                dst = sb + su;
                su += cnt;
                wr = dst + cnt <= P.stage_cap;
                if (lane == 0) {
                    const int64_t qw = I.qwbase + (int64_t)lx * I.nw + wf;
                    P.cntq[qw] = cnt;
                    if (wr) {
                        Segment S;
                        S.src = dst;
                        S.cnt = cnt;
                        S.i = lx;
                        P.segs[qw] = S;
                    }
                    ct.pairs += (uint32_t)cnt;
                }
                if (!wr) break;  // no room: the host grows the staging buffer and runs again
                if (cnt <= JOIN_ECAP) {  // every match is in the scratch list
                    __syncwarp();
                    for (int q = lane; q < cnt; q += 32) P.stage[dst + q] = elist[q];
                    break;
                }
            }
        }
    }
}

// One class of windowed items (G query groups per CTA, G known at compile time so that the
// group's shared-memory layout is constant offsets): every group takes items from the
// class's work list until it is empty, with its own work counters (folded into wtot).
template <bool QMODE, bool SPLIT, int G>
__device__ __forceinline__ void join_class(const JoinParams &P, const int64_t item_begin, const int64_t item_end,
                                        unsigned long long *const work, unsigned long long *const wtot,
                                        const bool f_minsize, const bool f_remscore, const bool f_upper) {
    extern __shared__ __align__(16) unsigned char smem[];
    Ctr ct;
    constexpr int GT = JOIN_THREADS / G;
    const int g = threadIdx.x / GT, gt = threadIdx.x % GT;
    const int lane = gt & 31, gw = gt >> 5;
    constexpr int NW = GT >> 5;
    constexpr int WG = JOIN_WMAX / G, RG = JOIN_RMAX / G;
    unsigned char *base = smem + (size_t)g * group_bytes(G);
    uint32_t *A = reinterpret_cast<uint32_t *>(base);  // fixed point, units of 2^-30
    uint32_t *pn4s = A + WG;                                        // [WG / 8], 16-byte aligned
    int64_t *c_start = reinterpret_cast<int64_t *>(pn4s + WG / 8);  // [GT]
    int32_t *c_cnt = reinterpret_cast<int32_t *>(c_start + GT);    // [GT]
    int32_t *c_ch0 = c_cnt + GT;                                    // [GT + 4] chunk prefix
    float *c_xv = reinterpret_cast<float *>(c_ch0 + GT + 4);        // [GT]
    float *xtab = c_xv + GT;                                        // [RG]
    int2 *xr = reinterpret_cast<int2 *>(xtab + RG);
    constexpr int XG = JOIN_XCAP / G;
    uint32_t *bm = reinterpret_cast<uint32_t *>(xr + XG);            // [WG / 32]
    int64_t *wsum = reinterpret_cast<int64_t *>(bm + WG / 32);
    int32_t *wcnt = reinterpret_cast<int32_t *>(wsum + 32);
    int64_t *bc = reinterpret_cast<int64_t *>(wcnt + 32);
    int2 *elist = P.scratch + ((size_t)blockIdx.x * NWARPS + (threadIdx.x >> 5)) * JOIN_ECAP;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int i = gt; i < WG; i += GT) A[i] = 0u;
    for (int i = gt; i < WG / 32; i += GT) bm[i] = 0u;
    if (gt == 0) bc[3] = bc[4] = bc[5] = 0;  // this group's staging slab: base, used, size

    for (;;) {
        ctr_flush(ct, wtot, lane);
        gsync(G, g, GT);  // every thread is done with the previous item's broadcast slots
        if (gt == 0) bc[0] = (int64_t)atomicAdd(work, 1ull) + item_begin;
        gsync(G, g, GT);
        const int64_t it = bc[0];
        if (it >= item_end) break;
        // x: a vector of the set (self-join: candidates are the later ids of its instance)
        // or an external query (all indexed vectors are candidates)
        // query mode: item = (query, window), so the windows of a long query run on several
        // CTAs at once instead of one after another
        const int64_t x = QMODE ? it / P.qnw : (int64_t)P.items[it];
        const int blk = (SPLIT && P.iblk) ? (int)P.iblk[it] : -1;  // group-uniform
        const int wq_item = QMODE ? (int)(it % P.qnw) : 0;
        const InstDesc I = P.inst[QMODE ? 0 : P.vinst[x]];
        const int32_t lx = QMODE ? -1 : (int32_t)(x - I.vbase);
        const int4 xm = QMODE ? P.qvmeta[x] : P.vmeta[x];
        const int2 *xrow = (QMODE ? P.qcrow : P.crow) + xm.x;
        const int32_t xl = xm.y;
        const int32_t qs = f_remscore ? (QMODE ? P.qqsplit[x] : P.qsplit[x]) : 0;
        const float mwx = QMODE ? P.qmw[x] : P.mw[x];
        const float t = QMODE ? P.qt : I.t;
        const float beta = fmaxf(1e-5f, (float)(xl + 2) * 1.1920929e-7f);  // (|x|+2) * 2^-23
        if (gt == 0) {  // what the emit step needs of x, kept in shared memory (not in registers)
            bc[6] = QMODE ? x * I.nw : I.qwbase + (int64_t)lx * I.nw;  // x's first (x, window) slot
            bc[7] = QMODE ? x : (int64_t)lx;                           // x's id in the output
        }
        // no component reaches remscore >= t: x can create no candidate at all
        if (f_remscore ? qs >= xl : xl == 0) continue;
        // A block item walks its share of x's creating components (every nblk-th, from its
        // block index on) and all of x's updating ones, which only add to candidates its
        // own creating components made.
        const int cstr = blk < 0 ? 1 : P.nblk, coff = blk < 0 ? 0 : blk;
        const int ncreate = blk < 0 ? xl - qs : (xl - qs > blk ? (xl - qs - blk + P.nblk - 1) / P.nblk : 0);
        const int nwalk = ncreate + qs;  // components this item walks
        if (ncreate == 0) continue;
        // minsize: a match y needs |y| >= t / maxweight(x) (margin for rounding and the
        // 1e-3 norm tolerance); the size class byte of each entry is compared with it
        // (float, directed rounding: numerator down, denominator up, quotient down, so the
        // bound can only come out below its exact value and never prunes a match)
        int smin = 0;
        if (f_minsize && I.packed && mwx > 0.f)
            smin = (int)ceilf(fminf(__fdiv_rd(__fsub_rd(t, beta), __fmul_ru(mwx, 1.0020001f)), 255.f));
        const uint32_t smin_tag = (uint32_t)max(smin, 0) << 24;
        const int32_t idmask = I.packed ? 0x00ffffff : 0x7fffffff;
        // dense table of x over small ranks for dot(x, y')
        for (int i = gt; i < RG; i += GT) xtab[i] = 0.f;
        gsync(G, g, GT);
        const int xs = xl <= XG ? xl : 0;  // x's row in shared memory when it fits
        for (int c = gt; c < xl; c += GT) {
            const int2 e = xrow[c];
            if (e.x < RG) xtab[e.x] = __int_as_float(e.y);
            if (c < xs) xr[c] = e;
        }
        gsync(G, g, GT);

        const int wfirst = QMODE ? wq_item : (lx + 1) / I.W;
        const int wend = QMODE ? wq_item + 1 : I.nw;
        for (int w = wfirst; w < wend; w++) {
            const int w0 = w * I.W;
            const int wn = min(I.W, I.n - w0);
            const int lo = max(0, lx + 1 - w0);
            bool created = false;  // any entry of a creating component in this window
            if (f_upper || blk >= 0) {  // the window's 4-bit ||y'||_2 codes into shared memory, behind the accumulation
                const uint32_t *src = P.pn4 + I.pbase + (w0 >> 3);
                for (int q = gt; q < (wn + 31) >> 5; q += GT) cp_async16(pn4s + 4 * q, src + 4 * q);
                cp_async_commit();
            }
            // ---------------- accumulate. Components are walked creating-first (those with
            // remscore >= t), so every batch holds its creating part before its updating part.
            if (nwalk <= 32) {
                // a short x: every warp builds the window's segment table itself, lane c
                // holding component c (no shared table, no barrier)
                int64_t st = 0;
                int cnt = 0;
                float xv = 0.f;
                if (lane < nwalk) {
                    const int c = lane < ncreate ? qs + coff + lane * cstr : lane - ncreate;
                    const int2 e = c < xs ? xr[c] : xrow[c];
                    const int64_t R = (int64_t)I.rbase + e.x;
                    xv = __int_as_float(e.y);
                    int64_t ls = P.lptr[R], le = P.lptr[R + 1];
                    if (I.nw > 1) {
                        const int32_t *wp = P.wptr + I.wbase + (int64_t)e.x * (I.nw + 1);
                        le = ls + wp[w + 1];
                        ls = ls + wp[w];
                    }
                    cnt = (int32_t)(le - ls);
                    st = ls;
                    if (gw == 0) ct.read += (uint32_t)cnt;
                }
                const int nch = (cnt + 127) >> 7;
                int nchk;
                const int ch0 = warp_excl_scan_int(nch, lane, &nchk);
                const int P0 = ncreate > 0 ? __shfl_sync(0xffffffffu, ch0 + nch, ncreate - 1) : 0;
                created = P0 > 0;
                for (int phase = 0; phase < 2; phase++) {
                    const int pb = phase == 0 ? 0 : P0, pe = phase == 0 ? P0 : nchk;
                    if (pe <= pb) continue;
                    if (phase == 1 && P0 > 0) gsync(G, g, GT);  // creations land before updates
                    const int K = (pe - pb + NW - 1) / NW;
                    const int ch = pb + gw * K;
                    const int che = min(ch + K, pe);
                    if (ch >= che) continue;
                    // the last component with entries whose first chunk is at or before ch
                    const int cc = 31 - __clz(__ballot_sync(0xffffffffu, nch > 0 && ch0 <= ch));
                    if (phase == 0) {
                        if (lo > 0) walk_chunks_r<true, true>(ch, che, cc, st, cnt, ch0, xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                        else walk_chunks_r<true, false>(ch, che, cc, st, cnt, ch0, xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                    } else {
                        if (lo > 0) walk_chunks_r<false, true>(ch, che, cc, st, cnt, ch0, xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                        else walk_chunks_r<false, false>(ch, che, cc, st, cnt, ch0, xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                    }
                }
                cp_async_wait_all();  // the window's codes have landed (visible after the barrier)
                gsync(G, g, GT);
            } else
            for (int c0 = 0; c0 < nwalk; c0 += GT) {
                const int cp = c0 + gt;
                int64_t st = 0;
                int32_t cnt = 0;
                float xv = 0.f;
                const bool ph0 = cp < ncreate;
                if (cp < nwalk) {
                    const int c = ph0 ? qs + coff + cp * cstr : cp - ncreate;
                    const int2 e = c < xs ? xr[c] : xrow[c];  // x's row from shared memory when held there
                    const int64_t R = (int64_t)I.rbase + e.x;
                    xv = __int_as_float(e.y);
                    int64_t ls = P.lptr[R], le = P.lptr[R + 1];
                    if (I.nw > 1) {
                        const int32_t *wp = P.wptr + I.wbase + (int64_t)e.x * (I.nw + 1);
                        le = ls + wp[w + 1];
                        ls = ls + wp[w];
                    }
                    cnt = (int32_t)(le - ls);
                    st = ls;
                    ct.read += (uint32_t)cnt;  // every entry of the window's list is loaded
                }
                // scan of (chunks, non-empty, non-empty creating) packed in one int64
                const int64_t nch = (cnt + 127) >> 7;
                const int64_t packed = (nch << 22) | ((cnt > 0 && ph0) ? (1 << 11) : 0) | (cnt > 0 ? 1 : 0);
                const int64_t inc = warp_incl_scan(packed, lane);
                if (lane == 31) wsum[gw] = inc;
                gsync(G, g, GT);
                const int64_t wv = lane < NW ? wsum[lane] : 0;
                const int64_t winc = warp_incl_scan(wv, lane);
                const int64_t before = __shfl_sync(0xffffffffu, winc - wv, gw);
                const int64_t total = __shfl_sync(0xffffffffu, winc, NW - 1);
                const int64_t ex = before + inc - packed;
                if (cnt > 0) {
                    const int pos = (int)(ex & 2047);
                    c_start[pos] = st;
                    c_cnt[pos] = cnt;
                    c_ch0[pos] = (int32_t)(ex >> 22);
                    c_xv[pos] = xv;
                }
                const int ncomp = (int)(total & 2047);
                const int ncomp0 = (int)((total >> 11) & 2047);
                const int nchk = (int)(total >> 22);
                if (gt == 0) c_ch0[ncomp] = nchk;
                gsync(G, g, GT);
                const int P0 = c_ch0[ncomp0];
                created = created || P0 > 0;
                // phase 0 chunks [0, P0) create candidates; phase 1 chunks [P0, nchk) update
                for (int phase = 0; phase < 2; phase++) {
                    const int pb = phase == 0 ? 0 : P0, pe = phase == 0 ? P0 : nchk;
                    if (pe <= pb) continue;
                    if (phase == 1 && P0 > 0) gsync(G, g, GT);  // creations land before updates
                    const int K = (pe - pb + NW - 1) / NW;
                    int ch = pb + gw * K;
                    const int che = min(ch + K, pe);
                    if (ch >= che) continue;
                    int cc = 0;
                    {  // component holding the warp's first chunk
                        int a = 0, b = ncomp - 1;
                        while (a < b) {
                            const int mid = (a + b + 1) >> 1;
                            if (c_ch0[mid] <= ch) a = mid; else b = mid - 1;
                        }
                        cc = a;
                    }
                    // four specialisations: creating or updating, first window (ids at or
                    // below x present) or not
                    if (phase == 0) {
                        if (lo > 0) walk_chunks<true, true>(ch, che, cc, c_start, c_cnt, c_ch0, c_xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                        else walk_chunks<true, false>(ch, che, cc, c_start, c_cnt, c_ch0, c_xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                    } else {
                        if (lo > 0) walk_chunks<false, true>(ch, che, cc, c_start, c_cnt, c_ch0, c_xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                        else walk_chunks<false, false>(ch, che, cc, c_start, c_cnt, c_ch0, c_xv, P.post, A, bm, smin_tag, idmask, w0, lo, lane, ct.visits);
                    }
                }
                cp_async_wait_all();  // the window's codes have landed (visible after the barrier)
                gsync(G, g, GT);
            }
            if (!created) continue;  // no candidate can exist in this window
            // ---------------- verify. The creating pass marked every candidate in bm. Each
            // warp walks its share of bm 32 words (1024 slots) at a time, a word per lane.
            // First each lane tests its word's candidates against the window's ||y'||_2
            // codes: since dot(x, y') <= ||y'||_2, a candidate with A[y] + ||y'||_2 <=
            // t - beta cannot match (most stop here, with no global load; their A is
            // cleared). Then the remaining bits are taken in slot order, 32 candidates per
            // batch: lane j of a batch takes the candidate at position b + j, located from
            // the lanes' popcount prefix. Taken slots are cleared in A (bm words as they are
            // read), and the emitted (y, score) go to the warp's scratch list in increasing y.
            const int wlo = lo >> 5, whi = (wn + 31) >> 5;
            const int wper = (whi - wlo + NW - 1) / NW;
            const int wb = wlo + gw * wper, we = min(wb + wper, whi);
            // A[y] + ||y'||_2 <= t - beta in units of 2^-30: threshold rounded down, codes
            // rounded up, so the test keeps at least every candidate the exact one keeps
            const uint32_t thq = __float2uint_rd(fmaxf(t - beta, 0.f) * 1073741824.f);
            int ne = 0;
            for (int wq = wb; wq < we; wq += 32) {
                uint32_t word = 0u;
                if (wq + lane < we) {
                    word = bm[wq + lane];
                    bm[wq + lane] = 0u;
                }
                ct.cand += (uint32_t)__popc(word);
                if (f_upper || blk >= 0) {
                    // a block item keeps y by Lemma 1 (local pruning): a match scores
                    // A + dot(x, y') >= t, the blocks that created y hold all of A between
                    // them, so one of them has A_b >= (t - ||y'||_2) / nblk
                    const uint32_t mul = blk < 0 ? 1u : (uint32_t)P.nblk;
                    const int sb = (wq + lane) << 5;
                    uint32_t keep = 0u;
                    for (uint32_t wv = word; wv; wv &= wv - 1u) {
                        const int b = __ffs(wv) - 1;
                        const int sl = sb + b;
                        const uint32_t a = A[sl];
                        const uint32_t code = (pn4s[sl >> 3] >> ((sl & 7) << 2)) & 15u;
                        const bool kp = SPLIT ? (uint64_t)a * mul + code * PN4_UNIT > (uint64_t)thq
                                              : a + code * PN4_UNIT > thq;
                        if (kp) keep |= 1u << b; else A[sl] = 0u;
                    }
                    word = keep;
                }
                const int c = __popc(word);
                int T;
                const int excl = warp_excl_scan_int(c, lane, &T);
                const int incl = excl + c;
                for (int b0 = 0; b0 < T; b0 += 32) {
                    const int p = b0 + lane;
                    // owner: the first lane whose inclusive count exceeds p (31 when p >= T)
                    int own = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1)
                        if (__shfl_sync(0xffffffffu, incl, own + step - 1) <= p) own += step;
                    uint32_t ow = __shfl_sync(0xffffffffu, word, own);
                    const int oex = __shfl_sync(0xffffffffu, excl, own);
                    const bool have = p < T;
                    bool emit = false;
                    float sc = 0.f, v = 0.f;
                    int s = 0;
                    int4 yc = make_int4(0, 0, 0, 0);  // {row offset, |y'|, maxweight(y'), ||y'||_2 bound}
                    // 0: rejected or emitted, 1: score known, 2: short dot(x, y') left, 3: long one
                    int stage = 0;
                    if (have) {
                        for (int k = p - oex; k > 0; k--) ow &= ow - 1u;
                        s = ((wq + own) << 5) + (__ffs(ow) - 1);
                        v = __uint2float_rn(A[s]) * 9.31322574615478515625e-10f;  // 2^-30
                        A[s] = 0u;
                        yc = __ldg(&P.vcand[I.vbase + w0 + s]);
                        const int ys = blk < 0 ? yc.y : 0;  // a block item scores y whole, below
                        bool ok = true;
                        // (a block item's A is a partial sum: these bounds apply to whole sums
                        // only, and the block's candidates passed the local test instead)
                        if (f_upper && blk < 0) {
                            // dot(x, y') <= ||y'||_2 (Cauchy-Schwarz; most candidates stop here),
                            // then the paper's upperbound; both off with NO_UPPERBOUND
                            ok = v + __int_as_float(yc.w) > t - beta;
                            if (ok && ys > 0) ok = v + (float)min(ys, xl) * mwx * __int_as_float(yc.z) >= t - beta;
                        }
                        if (ok) {
                            sc = v;
                            stage = ys == 0 ? 1 : (ys <= 16 ? 2 : 3);
                        }
                        if (blk >= 0) stage = 4;  // kept by the local test: score decided in float64
                    }
                    if (stage == 2) {  // short prefixes: each lane its own candidate
                        ct.verified++;
                        sc = v + dot_prefix(P.crow + yc.x, yc.y, xtab, RG, xr, xs, xrow, xl);
                        stage = 1;
                    }
                    // long prefixes: the whole warp takes one candidate at a time, its lanes
                    // reading y's prefix entries side by side
                    for (unsigned lm = __ballot_sync(0xffffffffu, stage == 3); lm; lm &= lm - 1u) {
                        const int src = __ffs(lm) - 1;
                        const int yo = __shfl_sync(0xffffffffu, yc.x, src);
                        const int yl = __shfl_sync(0xffffffffu, yc.y, src);
                        float acc = 0.f;
                        for (int k = lane; k < yl; k += 32) {
                            const int2 e = __ldg(&P.crow[yo + k]);
                            acc = fmaf(x_at(e.x, xtab, RG, xr, xs, xrow, xl), __int_as_float(e.y), acc);
                        }
#pragma unroll
                        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (lane == src) {
                            ct.verified++;
                            sc = v + acc;
                            stage = 1;
                        }
                    }
                    if (stage == 1) {
                        if (sc >= t + beta) {
                            emit = true;
                            stage = 0;
                        } else if (sc <= t - beta) {
                            stage = 0;
                        }
                    }
                    if (stage == 4) stage = 1;
                    // inside the band: float64 dot(x, y) over all of y, one candidate at a
                    // time across the warp (x's values from shared memory, exact products)
                    int yfull = 0;
                    if (stage == 1) yfull = __ldg(&P.vmeta[I.vbase + w0 + s]).y;
                    for (unsigned lm = __ballot_sync(0xffffffffu, stage == 1); lm; lm &= lm - 1u) {
                        const int src = __ffs(lm) - 1;
                        const int yo = __shfl_sync(0xffffffffu, yc.x, src);
                        const int yl = __shfl_sync(0xffffffffu, yfull, src);
                        double acc = 0.0;
                        for (int k = lane; k < yl; k += 32) {
                            const int2 e = P.crow[yo + k];
                            acc += (double)x_at(e.x, xtab, RG, xr, xs, xrow, xl) * (double)__int_as_float(e.y);
                        }
#pragma unroll
                        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                        if (lane == src) {
                            ct.band++;
                            emit = acc >= (double)t;
                            sc = (float)acc;
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, emit);
                    if (blk >= 0) {  // block items: pairs to the global list, merged after the join
                        unsigned long long b = 0;
                        if (lane == 0 && bal) b = atomicAdd(P.sp_count, (unsigned long long)__popc(bal));
                        b = __shfl_sync(0xffffffffu, b, 0) + (unsigned long long)__popc(bal & lt_mask);
                        if (emit && b < (unsigned long long)P.sp_cap) {
                            P.sp_key[b] = (unsigned long long)lx * (unsigned long long)I.n + (unsigned long long)(w0 + s);
                            P.sp_score[b] = __float_as_uint(sc);
                        }
                    } else {
                        if (emit) elist[ne + __popc(bal & lt_mask)] = make_int2(w0 + s, __float_as_int(sc));
                        ne += __popc(bal);
                    }
                }
            }
            if (blk >= 0) {  // (group-uniform) no run for this (x, window) slot; the barrier
                gsync(G, g, GT);  // keeps the next window's copies and adds off this window's data
                continue;
            }
            if (lane == 0) wcnt[gw] = ne;
            gsync(G, g, GT);
            if (gw == 0) {  // offsets of the warps' runs; the window's run in the group's slab
                const int cw = lane < NW ? wcnt[lane] : 0;
                int tot;
                const int exw = warp_excl_scan_int(cw, lane, &tot);
                if (lane < NW) wcnt[lane] = exw;
                if (lane == 0) {
                    const int64_t qw = bc[6] + w;
                    P.cntq[qw] = tot;
                    int64_t b = 0, wr = 0;
                    if (tot > 0) {
                        if (bc[4] + tot > bc[5]) {  // a new slab: one global atomic per slab
                            const int64_t want = max(P.stage_slab, (int64_t)tot);
                            bc[3] = (int64_t)atomicAdd(P.stage_count, (unsigned long long)want);
                            bc[4] = 0;
                            bc[5] = want;
                        }
                        b = bc[3] + bc[4];
                        bc[4] += tot;
                        if (b + tot <= P.stage_cap) {
                            Segment S;
                            S.src = b;
                            S.cnt = tot;
                            S.i = (int32_t)bc[7];
                            P.segs[qw] = S;
                            wr = 1;
                        }
                    }
                    ct.pairs += (uint32_t)tot;
                    bc[1] = b;
                    bc[2] = wr;
                }
            }
            gsync(G, g, GT);
            // ---------------- copy the warp's emitted pairs to the reserved run
            if (bc[2] != 0) {
                int2 *dst = P.stage + bc[1] + wcnt[gw];
                for (int k = lane; k < ne; k += 32) dst[k] = elist[k];
            }
            __syncwarp();
        }
    }
    ctr_flush(ct, wtot, lane);
}

// QMODE: external queries against the index (P.qmode = 1); SPLIT: a self-join whose work
// list may hold dimension-block items (P.iblk). Each is compiled separately, so that the
// plain self-join carries none of the other paths' state.
template <bool QMODE, bool SPLIT = false>
__global__ void __launch_bounds__(JOIN_THREADS, 1) join_kernel(const __grid_constant__ JoinParams P) {
    const bool f_minsize = !(P.flags & APS_NO_MINSIZE);
    const bool f_remscore = !(P.flags & APS_NO_REMSCORE);
    const bool f_upper = !(P.flags & APS_NO_UPPERBOUND);
    // per-warp 64-bit work totals (visits, candidates, verified, pairs, band, entries read)
    __shared__ unsigned long long wtot_s[NWARPS][6];
    for (int i = threadIdx.x; i < NWARPS * 6; i += blockDim.x) (&wtot_s[0][0])[i] = 0ull;
    __syncthreads();
    unsigned long long *const wtot = wtot_s[threadIdx.x >> 5];
    // A CTA that finds a class's work list empty moves on to the next class and re-carves
    // its shared memory for that class's G, so the classes share one launch and one tail.
    for (int cls = 0; cls < P.ncls; cls++) {
    const int64_t item_begin = P.cls_begin[cls], item_end = P.cls_begin[cls + 1];
    if (item_end <= item_begin) continue;
    const int G = P.cls_G[cls];
    unsigned long long *const work = P.work + cls;
    if (!QMODE && G == 0) {  // vectors with one or two components: one warp each, no shared memory
        stream_short(P, work, item_begin, item_end, f_minsize, f_remscore, wtot);
        continue;
    }
    switch (G) {
        case 1: join_class<QMODE, SPLIT, 1>(P, item_begin, item_end, work, wtot, f_minsize, f_remscore, f_upper); break;
        case 2: join_class<QMODE, SPLIT, 2>(P, item_begin, item_end, work, wtot, f_minsize, f_remscore, f_upper); break;
        case 4: join_class<QMODE, SPLIT, 4>(P, item_begin, item_end, work, wtot, f_minsize, f_remscore, f_upper); break;
        default: join_class<QMODE, SPLIT, 8>(P, item_begin, item_end, work, wtot, f_minsize, f_remscore, f_upper); break;
    }
    __syncthreads();  // every group is done with this class's layout of shared memory
    }
    // flush counters: the warps' totals, one global atomic per counter and warp
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 6; k++)
            if (wtot[k]) atomicAdd(&P.counters[k < 5 ? k : 6], wtot[k]);
    }
}

// One warp per (x, window) slot: copy its staged run to the output at scan(counts)[qw].
__global__ void k_gather(const Segment *__restrict__ segs, const int32_t *__restrict__ cntq, int64_t nqw,
                         const int2 *__restrict__ stage, const int64_t *__restrict__ qwoff, int32_t *__restrict__ oi,
                         int32_t *__restrict__ oj, float *__restrict__ os) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < nqw; q += nwarps) {
        const int cnt = cntq[q];
        if (cnt == 0) continue;
        const Segment S = segs[q];
        const int64_t dst = qwoff[q];
        for (int e = lane; e < cnt; e += 32) {
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

// The index's work-list classes as one launch's class list. Returns the CTA count (enough
// for every class's groups, or warps for the class of one- and two-component vectors, at most max_ctas) and
// sets *smem to the largest class layout used.
int set_classes(JoinParams &P, const aps_index *ix, int max_ctas, int *smem) {
    static const int Gs[JOIN_NCLS] = {1, 2, 4, 8, 0};
    P.ncls = JOIN_NCLS;
    int64_t ctas = 0;
    *smem = 0;
    for (int c = 0; c < JOIN_NCLS; c++) {
        P.cls_G[c] = Gs[c];
        P.cls_begin[c] = ix->class_begin[c];
        const int64_t ni = ix->class_begin[c + 1] - ix->class_begin[c];
        if (ni <= 0) continue;
        const int per_cta = Gs[c] > 0 ? Gs[c] : NWARPS;
        ctas = std::max(ctas, (ni + per_cta - 1) / per_cta);
        if (Gs[c] > 0) *smem = std::max(*smem, group_bytes(Gs[c]) * Gs[c]);
    }
    P.cls_begin[JOIN_NCLS] = ix->class_begin[JOIN_NCLS];
    return (int)std::min<int64_t>(max_ctas, std::max<int64_t>(ctas, 1));
}

// The join phase (reset the counters and the per-slot pair counts, then the persistent
// join) as a CUDA graph: captured on the index's first join (on a private stream, so any
// caller stream works, including the legacy default one), then replayed with the memset
// targets and the kernel's parameters and grid updated in place for each later join.
aps_status run_join_graph(aps_index *ix, JoinParams &P, int grid, int smem, unsigned long long *ctr, int32_t *cntq,
                          cudaStream_t s) {
    JoinGraph &G = ix->jgraph;
    const size_t ctr_bytes = 16 * sizeof(unsigned long long), cnt_bytes = sizeof(int32_t) * (size_t)ix->nqw;
    if (!G.exec) {
        cudaStream_t cs = nullptr;
        APS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(ctr, 0, ctr_bytes, cs);
            cudaMemsetAsync(cntq, 0, cnt_bytes, cs);
            join_kernel<false><<<grid, JOIN_THREADS, smem, cs>>>(P);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cs, &g);
            G.graph = g;
        }
        cudaStreamDestroy(cs);
        APS_CUDA(e);
        size_t nn = 0;
        APS_CUDA(cudaGraphGetNodes(G.graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        APS_CUDA(cudaGraphGetNodes(G.graph, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            APS_CUDA(cudaGraphNodeGetType(nd, &ty));
            if (ty == cudaGraphNodeTypeKernel) {
                G.join = nd;
            } else if (ty == cudaGraphNodeTypeMemset) {
                cudaMemsetParams mp;
                APS_CUDA(cudaGraphMemsetNodeGetParams(nd, &mp));
                if (mp.dst == ctr) G.reset_ctr = nd;
                if (mp.dst == cntq) G.reset_cnt = nd;
            }
        }
        if (nn != 3 || !G.join || !G.reset_ctr || !G.reset_cnt) {
            set_error("join graph: expected two memset nodes and one kernel node, captured %zu nodes", nn);
            return APS_ECUDA;
        }
        APS_CUDA(cudaGraphInstantiate(&G.exec, G.graph, 0));
    } else {
        cudaMemsetParams mp;
        APS_CUDA(cudaGraphMemsetNodeGetParams(G.reset_ctr, &mp));
        mp.dst = ctr;
        APS_CUDA(cudaGraphExecMemsetNodeSetParams(G.exec, G.reset_ctr, &mp));
        APS_CUDA(cudaGraphMemsetNodeGetParams(G.reset_cnt, &mp));
        mp.dst = cntq;
        APS_CUDA(cudaGraphExecMemsetNodeSetParams(G.exec, G.reset_cnt, &mp));
        void *args[1] = {&P};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = reinterpret_cast<void *>(join_kernel<false>);
        kp.gridDim = dim3((unsigned)grid);
        kp.blockDim = dim3(JOIN_THREADS);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = args;
        APS_CUDA(cudaGraphExecKernelNodeSetParams(G.exec, G.join, &kp));
    }
    APS_CUDA(cudaGraphLaunch(G.exec, s));
    count_launch();
    G.launches++;
    return APS_OK;
}

}  // namespace

namespace {

// The work list of a split join: the first `heavy` items of the list (the costliest
// vectors) become nblk block items each, the rest stay whole.
__global__ void k_split_items(const int32_t *__restrict__ items, int64_t nitems, int64_t heavy, int nblk,
                              int32_t *out, int8_t *blk) {
    const int64_t total = nitems + heavy * (nblk - 1);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        if (k < heavy * nblk) {
            out[k] = items[k / nblk];
            blk[k] = (int8_t)(k % nblk);
        } else {
            out[k] = items[k - heavy * (nblk - 1)];
            blk[k] = -1;
        }
    }
}

// First occurrence of each key in a sorted list (the block items of one vector may find a
// pair twice, with the same score).
__global__ void k_first_of_key(const unsigned long long *__restrict__ key, int64_t n, int32_t *flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = (k == 0 || key[k] != key[k - 1]) ? 1 : 0;
}

// The split vectors' pairs (key = local x * n + local y, sorted, first occurrences at
// off[k]) into the staging buffer from `base` on, as the runs of their (x, window) slots.
__global__ void k_split_place(const unsigned long long *__restrict__ key, const uint32_t *__restrict__ score,
                              const int32_t *__restrict__ flag, const int64_t *__restrict__ off, int64_t n,
                              const InstDesc *__restrict__ inst, int64_t base, int2 *stage, Segment *segs,
                              int32_t *cntq) {
    const InstDesc I = inst[0];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        const unsigned long long kk = key[k];
        const int32_t lx = (int32_t)(kk / (unsigned long long)I.n), y = (int32_t)(kk % (unsigned long long)I.n);
        const int w = y / I.W;
        const int64_t qw = I.qwbase + (int64_t)lx * I.nw + w;
        const int64_t pos = base + off[k];
        stage[pos] = make_int2(y, (int)score[k]);
        atomicAdd(&cntq[qw], 1);
        bool first = k == 0;
        if (!first) {
            const unsigned long long pk = key[k - 1];
            first = (int32_t)(pk / (unsigned long long)I.n) != lx || (int32_t)(pk % (unsigned long long)I.n) / I.W != w;
        }
        if (first) {
            Segment S;
            S.src = pos;
            S.cnt = 0;
            S.i = lx;
            segs[qw] = S;
        }
    }
}

}  // namespace

// Staging slots one CTA can reserve and leave unused: a slab per group of every windowed
// class (1 + 2 + 4 + 8 groups) and a slab per warp of the streamed class.
int64_t join_slab_slack() { return 15 * (int64_t)JOIN_STAGE_SLAB + (int64_t)NWARPS * (JOIN_STAGE_SLAB / 8); }

void debug_stage_cap(int64_t pairs) { g_stage_cap_once.store(pairs > 0 ? pairs : 0); }

aps_status join_all_pairs(aps_index *ix, uint32_t flags, aps_pairs *out, std::vector<int64_t> *pair_offsets_h,
                          int nblk, int64_t heavy) {
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
    APS_CUDA(cudaFuncSetAttribute(join_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, need));

    // the vertical split: the costliest `heavy` vectors as nblk dimension blocks each
    const bool split = nblk >= 2 && heavy > 0 && ix->k == 1;
    int split_cls = -1;
    int64_t nsplit = 0, sp_cap = 0;
    DBuf<int32_t> items2;
    DBuf<int8_t> iblk;
    DBuf<unsigned long long> sp_key;
    DBuf<uint32_t> sp_score;
    if (split) {
        // block items come from the windowed classes (G = 1 ... 8), never from the
        // streamed class (one- and two-component vectors) that follows them
        for (int c = 0; c < 4; c++)
            if (ix->class_begin[c + 1] > ix->class_begin[c]) split_cls = c;
        const int64_t nitems = ix->class_begin[JOIN_NCLS] - ix->class_begin[0];
        nsplit = std::min<int64_t>(heavy, ix->class_begin[4] - ix->class_begin[0]);
        if (nsplit > 0) {
            APS_CUDA(cudaFuncSetAttribute(join_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, need));
            const int64_t total = nitems + nsplit * (nblk - 1);
            APS_TRY(items2.alloc((size_t)total, s));
            APS_TRY(iblk.alloc((size_t)total, s));
            k_split_items<<<grid_for(total, 256), 256, 0, s>>>(ix->items.p, nitems, nsplit, nblk, items2.p, iblk.p);
            APS_LAUNCH_CHECK();
            sp_cap = std::max<int64_t>((int64_t)1 << 20, nsplit * 4096);
        }
    }

    DBuf<int32_t> cntq;
    DBuf<unsigned long long> ctr;  // 0..4 counters, 5 stage count, 6 entries read, 8..12 work, 13 split pairs
    APS_TRY(cntq.alloc((size_t)std::max<int64_t>(ix->nqw, 1), s));
    APS_TRY(ctr.alloc(16, s));
    // Staging capacity: the index's own hint, else the last join of this process; a join
    // that still overflows is re-run with room for what it reserved plus one slab per
    // group. Segments are stored per (vector, window) slot, so their table never overflows.
    int64_t stage_cap = std::max<int64_t>({ix->hint_pairs, g_stage_hint.load(), (int64_t)1 << 20, ix->nnz});
    if (ix->hint_pairs == 0 && g_stage_hint.load() == 0) {
        // no join of this process has sized the staging yet: take room for every possible
        // pair plus one slab per group, but at most an eighth of the free device memory
        // and 2^28 pairs, so that a first join rarely has to run twice
        int64_t most = (int64_t)sms * join_slab_slack();
        for (const InstDesc &I : ix->inst_h) most += (int64_t)I.n * (I.n - 1) / 2;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const int64_t room = std::min<int64_t>({most, (int64_t)(fr / 8 / sizeof(int2)), (int64_t)1 << 28});
            stage_cap = std::max(stage_cap, room);
        } else {
            cudaGetLastError();
        }
    }
    if (const int64_t once = g_stage_cap_once.exchange(0); once > 0) stage_cap = once;
    DBuf<int2> stage;
    DBuf<Segment> segs;
    DBuf<int2> scratch;
    APS_TRY(scratch.alloc((size_t)sms * NWARPS * JOIN_ECAP, s));
    APS_TRY(segs.alloc((size_t)std::max<int64_t>(ix->nqw, 1), s));
    int64_t total_pairs = 0, reserved = 0;
    unsigned long long ch[16];
    int reruns = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        APS_TRY(stage.alloc((size_t)stage_cap, s));
        if (nsplit > 0) {
            APS_TRY(sp_key.alloc((size_t)sp_cap, s));
            APS_TRY(sp_score.alloc((size_t)sp_cap, s));
        }
        if (ix->class_begin[JOIN_NCLS] <= ix->class_begin[0]) {  // nothing to join: just the resets
            APS_CUDA(cudaMemsetAsync(ctr.p, 0, 16 * sizeof(unsigned long long), s));
            if (ix->nqw) APS_CUDA(cudaMemsetAsync(cntq.p, 0, sizeof(int32_t) * ix->nqw, s));
            APS_CUDA(cudaEventRecord(ev[0], s));
        } else {
            JoinParams P;
            P.inst = d.inst.p;
            P.vinst = d.vinst.p;
            P.items = ix->items.p;
            int smem = 0;
            const int grid = set_classes(P, ix, sms, &smem);
            P.crow = d.crow.p;
            P.vmeta = d.vmeta.p;
            P.vcand = d.vcand.p;
            P.pn4 = d.pn4.p;
            P.qsplit = d.qsplit.p;
            P.mw = d.mw.p;
            P.lptr = d.lptr.p;
            P.wptr = d.wptr.p;
            P.post = d.post.p;
            P.flags = flags | (ix->flags & (APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND));
            P.stage = stage.p;
            P.stage_cap = stage_cap;
            P.stage_count = ctr.p + 5;
            P.stage_slab = JOIN_STAGE_SLAB;
            P.segs = segs.p;
            P.cntq = cntq.p;
            P.counters = ctr.p;
            P.work = ctr.p + 8;
            P.scratch = scratch.p;
            P.qmode = 0;
            P.qnw = 1;
            P.iblk = nullptr;
            P.nblk = 1;
            P.sp_key = nullptr;
            P.sp_score = nullptr;
            P.sp_count = ctr.p + 13;
            P.sp_cap = 0;
            APS_CUDA(cudaEventRecord(ev[0], s));
            if (nsplit > 0) {  // the split work list, one direct launch
                P.items = items2.p;
                P.iblk = iblk.p;
                P.nblk = nblk;
                P.sp_key = sp_key.p;
                P.sp_score = sp_score.p;
                P.sp_cap = sp_cap;
                for (int c = split_cls + 1; c <= JOIN_NCLS; c++) P.cls_begin[c] += nsplit * (nblk - 1);
                APS_CUDA(cudaMemsetAsync(ctr.p, 0, 16 * sizeof(unsigned long long), s));
                APS_CUDA(cudaMemsetAsync(cntq.p, 0, sizeof(int32_t) * std::max<int64_t>(ix->nqw, 1), s));
                join_kernel<false, true><<<grid, JOIN_THREADS, smem, s>>>(P);
                APS_LAUNCH_CHECK();
            } else {
                APS_TRY(run_join_graph(ix, P, grid, smem, ctr.p, cntq.p, s));
            }
        }
        APS_CUDA(cudaEventRecord(ev[1], s));
        APS_CUDA(cudaMemcpyAsync(ch, ctr.p, sizeof(ch), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        total_pairs = (int64_t)ch[3];
        reserved = (int64_t)ch[5];
        const int64_t sp_found = nsplit > 0 ? (int64_t)ch[13] : 0;
        if (reserved <= stage_cap && sp_found <= sp_cap) {
            if (sp_found > 0) {
                // the split vectors' pairs: sorted by (x, y), first occurrences kept, placed
                // after the join's staged runs as the runs of their (x, window) slots
                const InstDesc &I0 = ix->inst_h[0];
                APS_TRY(sort_pairs(reinterpret_cast<uint64_t *>(sp_key.p), sp_score.p, sp_found,
                                   bits_for((uint64_t)I0.n * (uint64_t)I0.n), s));
                DBuf<int32_t> flag;
                DBuf<int64_t> off;
                APS_TRY(flag.alloc((size_t)sp_found, s));
                APS_TRY(off.alloc((size_t)sp_found + 1, s));
                k_first_of_key<<<grid_for(sp_found, 256), 256, 0, s>>>(sp_key.p, sp_found, flag.p);
                APS_LAUNCH_CHECK();
                APS_TRY(scan_exclusive(flag.p, off.p, sp_found, s));
                int64_t nuniq = 0;
                APS_CUDA(cudaMemcpyAsync(&nuniq, off.p + sp_found, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                APS_CUDA(cudaStreamSynchronize(s));
                if (reserved + nuniq > stage_cap) {  // room after the join's runs
                    DBuf<int2> grown;
                    APS_TRY(grown.alloc((size_t)(reserved + nuniq), s));
                    if (reserved > 0)
                        APS_CUDA(cudaMemcpyAsync(grown.p, stage.p, sizeof(int2) * reserved, cudaMemcpyDeviceToDevice, s));
                    std::swap(grown.p, stage.p);
                    std::swap(grown.n, stage.n);
                    stage_cap = reserved + nuniq;
                }
                k_split_place<<<grid_for(sp_found, 256), 256, 0, s>>>(sp_key.p, sp_score.p, flag.p, off.p, sp_found,
                                                                     d.inst.p, reserved, stage.p, segs.p, cntq.p);
                APS_LAUNCH_CHECK();
                total_pairs += nuniq;
            }
            break;
        }
        if (sp_found > sp_cap) sp_cap = sp_found + sp_found / 8 + 1024;
        if (reserved <= stage_cap) {
            reruns++;
            if (attempt == 2) {
                set_error("split pair list overflow persisted");
                return APS_EOVERFLOW;
            }
            continue;
        }
        // the staging buffer was too small: grow it and run again
        reruns++;
        stage_cap = reserved + (int64_t)sms * join_slab_slack();  // plus every slab a CTA can leave unfilled
        if (attempt == 2) {
            set_error("pair staging overflow persisted");
            return APS_EOVERFLOW;
        }
    }
    ix->hint_pairs = reserved + reserved / 16 + 1024;
    g_stage_hint.store(ix->hint_pairs);
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
    if (npairs > 0) {
        k_gather<<<grid_for(ix->nqw * 32, 256, (int64_t)sms * 32), 256, 0, s>>>(segs.p, cntq.p, ix->nqw, stage.p,
                                                                               qwoff.p, oi, oj, os);
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
    std::lock_guard<std::mutex> lk(ix->stats_mu);  // queries may report meanwhile
    aps_stats &S = ix->stats;
    S.visits = (int64_t)ch[0];
    S.candidates = (int64_t)ch[1];
    S.verified = (int64_t)ch[2];
    S.pairs = total_pairs;
    S.band = (int64_t)ch[4];
    S.entries_read = (int64_t)ch[6];
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
            hfree(pa->block, pa->bytes);
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
    pa->bytes = std::max<size_t>(n, 1) * 12;
    aps_status hst = halloc(&pa->block, pa->bytes);
    if (hst != APS_OK) {
        delete pa;
        return hst;
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

// ------------------------------------------------------------------ arena variant
// The same join and output kernels with every buffer carved out of a caller-provided
// device arena instead of allocated: counters, per-(x, window) counts and offsets, the
// segment table, the per-warp emit lists (for at most max_ctas CTAs) and, in what is left,
// the pair staging buffer. Pairs are gathered into the caller's (i, j, score) arrays.
namespace {

constexpr int SCAN1_THREADS = 1024;

// Exclusive prefix sum by a single CTA, tile by tile with a running carry (no scratch).
__global__ void __launch_bounds__(SCAN1_THREADS) k_scan_single(const int32_t *__restrict__ in, int64_t n,
                                                               int64_t *__restrict__ out) {
    __shared__ int64_t wt[SCAN1_THREADS / 32];
    __shared__ int64_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += (int64_t)SCAN1_THREADS * 4) {
        const int64_t i0 = base + (int64_t)threadIdx.x * 4;
        int64_t v[4], local = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[k] = (i0 + k < n) ? (int64_t)in[i0 + k] : 0;
            local += v[k];
        }
        int64_t inc = warp_incl_scan(local, lane);
        if (lane == 31) wt[warp] = inc;
        __syncthreads();
        const int64_t wv = lane < SCAN1_THREADS / 32 ? wt[lane] : 0;
        const int64_t winc = warp_incl_scan(wv, lane);
        const int64_t before = __shfl_sync(0xffffffffu, winc - wv, warp);
        const int64_t tile = __shfl_sync(0xffffffffu, winc, 31);
        int64_t run = carry_s + before + inc - local;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (i0 + k < n) out[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tile;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry_s;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

aps_status join_noalloc(aps_index *ix, unsigned char *arena, size_t arena_bytes, int max_ctas, int32_t *oi,
                        int32_t *oj, float *os, int64_t cap, int64_t *count, cudaStream_t s) {
    IndexArrays &d = ix->d;
    const int grid_max = std::max(1, std::min(num_sms(), max_ctas));
    const int64_t nqw = std::max<int64_t>(ix->nqw, 1);
    size_t off = 0;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(arena + off);
    off = align256(off + 16 * sizeof(unsigned long long));
    int32_t *cntq = reinterpret_cast<int32_t *>(arena + off);
    off = align256(off + sizeof(int32_t) * nqw);
    int64_t *qwoff = reinterpret_cast<int64_t *>(arena + off);
    off = align256(off + sizeof(int64_t) * (nqw + 1));
    Segment *segs = reinterpret_cast<Segment *>(arena + off);
    off = align256(off + sizeof(Segment) * nqw);
    int2 *elists = reinterpret_cast<int2 *>(arena + off);
    off = align256(off + sizeof(int2) * (size_t)grid_max * NWARPS * JOIN_ECAP);
    if (off >= arena_bytes) {
        set_error("index too large for the %zu-byte arena: its %lld (vector, window) slots need %zu bytes "
                  "before any pair is staged",
                  arena_bytes, (long long)ix->nqw, off);
        return APS_EINVAL;
    }
    int2 *stage = reinterpret_cast<int2 *>(arena + off);
    const int64_t stage_cap = (int64_t)((arena_bytes - off) / sizeof(int2));

    const int Gs[4] = {1, 2, 4, 8};
    int need = 0;
    for (int c = 0; c < 4; c++) need = std::max(need, group_bytes(Gs[c]) * Gs[c]);
    APS_CUDA(cudaFuncSetAttribute(join_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, need));
    APS_CUDA(cudaMemsetAsync(ctr, 0, 16 * sizeof(unsigned long long), s));
    APS_CUDA(cudaMemsetAsync(cntq, 0, sizeof(int32_t) * nqw, s));
    if (ix->class_begin[JOIN_NCLS] > ix->class_begin[0]) {
        JoinParams P;
        P.inst = d.inst.p;
        P.vinst = d.vinst.p;
        P.items = ix->items.p;
        int smem = 0;
        const int grid = set_classes(P, ix, grid_max, &smem);
        P.crow = d.crow.p;
        P.vmeta = d.vmeta.p;
        P.vcand = d.vcand.p;
        P.pn4 = d.pn4.p;
        P.qsplit = d.qsplit.p;
        P.mw = d.mw.p;
        P.lptr = d.lptr.p;
        P.wptr = d.wptr.p;
        P.post = d.post.p;
        P.flags = ix->flags & (APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND);
        P.stage = stage;
        P.stage_cap = stage_cap;
        P.stage_count = ctr + 5;
        P.stage_slab = 256;  // small slabs: the arena's staging room is modest
        P.segs = segs;
        P.cntq = cntq;
        P.counters = ctr;
        P.work = ctr + 8;
        P.scratch = elists;
        P.qmode = 0;
        P.qnw = 1;
        join_kernel<false><<<grid, JOIN_THREADS, smem, s>>>(P);
        APS_LAUNCH_CHECK();
    }
    unsigned long long ch[16];
    APS_CUDA(cudaMemcpyAsync(ch, ctr, sizeof(ch), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    const int64_t total = (int64_t)ch[3];
    *count = total;
    if ((int64_t)ch[5] > stage_cap) {
        set_error("%lld staged pairs (%lld emitted) exceed the arena's staging room of %lld pairs",
                  (long long)ch[5], (long long)total, (long long)stage_cap);
        return APS_EOVERFLOW;
    }
    if (total > cap) {
        set_error("%lld pairs do not fit the caller's capacity of %lld", (long long)total, (long long)cap);
        return APS_EOVERFLOW;
    }
    k_scan_single<<<1, SCAN1_THREADS, 0, s>>>(cntq, ix->nqw, qwoff);
    APS_LAUNCH_CHECK();
    if (total > 0) {
        k_gather<<<grid_for(ix->nqw * 32, 256, (int64_t)num_sms() * 32), 256, 0, s>>>(segs, cntq, ix->nqw, stage,
                                                                                     qwoff, oi, oj, os);
        APS_LAUNCH_CHECK();
    }
    APS_CUDA(cudaStreamSynchronize(s));
    // the index's stats report the last join, whichever entry point ran it (no timings:
    // this path records no events)
    std::lock_guard<std::mutex> lk(ix->stats_mu);
    aps_stats &S = ix->stats;
    S.visits = (int64_t)ch[0];
    S.candidates = (int64_t)ch[1];
    S.verified = (int64_t)ch[2];
    S.pairs = (int64_t)ch[3];
    S.band = (int64_t)ch[4];
    S.entries_read = (int64_t)ch[6];
    S.reruns = 0;
    S.ms_join = S.ms_sort = S.ms_total = 0.f;
    S.evaluations = 0;
    for (const InstDesc &I : ix->inst_h) S.evaluations += (int64_t)I.n * (I.n - 1) / 2;
    return APS_OK;
}

// ------------------------------------------------------------------ external queries
aps_status join_queries(const aps_index *ix, const QueryArrays &qa, float t, uint32_t flags, cudaStream_t s,
                        aps_pairs *out, aps_stats *stats) {
    const IndexArrays &d = ix->d;
    const InstDesc &I = ix->inst_h[0];
    const int sms = num_sms();
    const int64_t nq = qa.nq;
    const int64_t nqw = std::max<int64_t>(nq * (int64_t)std::max(I.nw, 1), 1);
    const int G = I.G;
    const int Gs[4] = {1, 2, 4, 8};
    int need = 0;
    for (int c = 0; c < 4; c++) need = std::max(need, group_bytes(Gs[c]) * Gs[c]);
    APS_CUDA(cudaFuncSetAttribute(join_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, need));
    cudaEvent_t ev[3];
    for (int i = 0; i < 3; i++) APS_CUDA(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 3; i++) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    const int64_t nitems = nq * (int64_t)I.nw;  // (query, window) items
    const int grid = (int)std::min<int64_t>(sms, std::max<int64_t>((nitems + G - 1) / G, 1));
    DBuf<int32_t> cntq;
    DBuf<unsigned long long> ctr;
    DBuf<int2> scratch, stage;
    DBuf<Segment> segs;
    APS_TRY(cntq.alloc((size_t)nqw, s));
    APS_TRY(ctr.alloc(16, s));
    APS_TRY(scratch.alloc((size_t)grid * NWARPS * JOIN_ECAP, s));
    APS_TRY(segs.alloc((size_t)nqw, s));
    // staging: the pairs per query this index's batches have needed so far (at least 64),
    // plus one slab per group
    const int64_t ppq16 = ix->q_ppq16.load(std::memory_order_relaxed);
    int64_t stage_cap = std::max<int64_t>(nq * ppq16 / 16 + (int64_t)grid * G * 256, (int64_t)1 << 16);
    unsigned long long ch[16];
    for (int attempt = 0; attempt < 2; attempt++) {
        APS_TRY(stage.alloc((size_t)stage_cap, s));
        APS_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(ch), s));
        APS_CUDA(cudaMemsetAsync(cntq.p, 0, sizeof(int32_t) * nqw, s));
        APS_CUDA(cudaEventRecord(ev[0], s));
        if (nq > 0) {
            JoinParams P;
            memset(&P, 0, sizeof(P));
            P.inst = d.inst.p;
            P.vinst = d.vinst.p;
            P.items = nullptr;
            P.ncls = 1;
            P.cls_G[0] = G;
            P.cls_begin[0] = 0;
            P.cls_begin[1] = nitems;
            P.crow = d.crow.p;
            P.vmeta = d.vmeta.p;
            P.vcand = d.vcand.p;
            P.pn4 = d.pn4.p;
            P.qsplit = d.qsplit.p;
            P.mw = d.mw.p;
            P.lptr = d.lptr.p;
            P.wptr = d.wptr.p;
            P.post = d.post.p;
            P.flags = flags & (APS_NO_MINSIZE | APS_NO_REMSCORE | APS_NO_UPPERBOUND);
            P.stage = stage.p;
            P.stage_cap = stage_cap;
            P.stage_count = ctr.p + 5;
            P.stage_slab = 256;  // query batches are small: keep the slab tails short
            P.segs = segs.p;
            P.cntq = cntq.p;
            P.counters = ctr.p;
            P.work = ctr.p + 8;
            P.scratch = scratch.p;
            P.qmode = 1;
            P.qcrow = qa.crow.p;
            P.qvmeta = qa.vmeta.p;
            P.qqsplit = qa.qsplit.p;
            P.qmw = qa.mw.p;
            P.qt = t;
            P.qnw = std::max(I.nw, 1);
            join_kernel<true><<<grid, JOIN_THREADS, group_bytes(G) * G, s>>>(P);
            APS_LAUNCH_CHECK();
        }
        APS_CUDA(cudaEventRecord(ev[1], s));
        APS_CUDA(cudaMemcpyAsync(ch, ctr.p, sizeof(ch), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        if ((int64_t)ch[5] <= stage_cap) break;
        stage_cap = (int64_t)ch[5] + (int64_t)grid * G * 256;  // what was reserved, plus one slab per group
    }
    if (nq > 0) {  // remember what this batch needed (with a quarter more), for the next ones
        const int64_t need16 = (int64_t)ch[5] * 20 / nq;
        int64_t cur = ix->q_ppq16.load(std::memory_order_relaxed);
        while (need16 > cur && !ix->q_ppq16.compare_exchange_weak(cur, need16, std::memory_order_relaxed)) {
        }
    }
    if ((int64_t)ch[5] > stage_cap) {
        set_error("pair staging overflow persisted");
        return APS_EOVERFLOW;
    }
    const int64_t npairs = (int64_t)ch[3];
    DBuf<int64_t> qwoff;
    APS_TRY(qwoff.alloc((size_t)nqw + 1, s));
    APS_TRY(scan_exclusive(cntq.p, qwoff.p, nqw, s));
    PairsAlloc *pa = new PairsAlloc();
    pa->stream = s;
    const size_t seg4 = ((size_t)npairs * 4 + 127) & ~(size_t)127;
    aps_status st = dalloc(&pa->block, std::max<size_t>(3 * seg4, 256), s);
    if (st != APS_OK) {
        delete pa;
        return st;
    }
    char *blk = static_cast<char *>(pa->block);
    int32_t *oi = reinterpret_cast<int32_t *>(blk);
    int32_t *oj = reinterpret_cast<int32_t *>(blk + seg4);
    float *os = reinterpret_cast<float *>(blk + 2 * seg4);
    if (npairs > 0) {
        k_gather<<<grid_for(nqw * 32, 256, (int64_t)sms * 32), 256, 0, s>>>(segs.p, cntq.p, nqw, stage.p, qwoff.p, oi,
                                                                           oj, os);
        APS_LAUNCH_CHECK();
    }
    APS_CUDA(cudaEventRecord(ev[2], s));
    APS_CUDA(cudaEventSynchronize(ev[2]));
    if (stats) {
        float mj = 0, mo = 0;
        cudaEventElapsedTime(&mj, ev[0], ev[1]);
        cudaEventElapsedTime(&mo, ev[1], ev[2]);
        memset(stats, 0, sizeof(*stats));
        stats->visits = (int64_t)ch[0];
        stats->candidates = (int64_t)ch[1];
        stats->verified = (int64_t)ch[2];
        stats->pairs = (int64_t)ch[3];
        stats->band = (int64_t)ch[4];
        stats->entries_read = (int64_t)ch[6];
        stats->evaluations = nq * (int64_t)I.n;
        stats->ms_join = mj;
        stats->ms_sort = mo;
    }
    out->count = npairs;
    out->i = oi;
    out->j = oj;
    out->score = os;
    out->on_device = 1;
    out->_reserved = 0;
    out->_priv = pa;
    return APS_OK;
}

}  // namespace aps
