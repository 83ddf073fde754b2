// Dense-embedding all-pairs: the matrix view S = D.D^T of the problem definition (Sec. 2.1)
// on the 5th-generation tensor cores, then exact decisions.
//
//   1. X (float32) -> Xb (bfloat16, rows padded with zeros to a multiple of 256).
//   2. dense_gemm_kernel: persistent clusters of two CTAs, one CTA per SM. A pair owns a
//      256-row block of Xb (the "A" operand; each CTA keeps its 128 rows resident in
//      shared memory) and streams 256-row blocks of Xb (the "B" operand; each CTA loads its
//      128-row half) through a TMA ring. One thread of the even CTA issues
//      tcgen05.mma.cta_group::2 (M = N = 256, K = 16, BF16 in, float32 accumulators in the
//      tensor memory of both SMs, double-buffered); sixteen epilogue warps per CTA read the
//      accumulators with tcgen05.ld and keep (i < j) with S_ij >= t - delta, where delta
//      bounds |x.y - bf16(x).bf16(y)| plus the float32 accumulation error, so no pair with
//      x.y >= t is lost. Sharing B across the pair halves each SM's shared-memory operand
//      reads per MMA compared with a single-SM 128-row tile.
//   3. Candidates are sorted by (i, j), rescored in float32 from X (float64 when within
//      the band of t) and compacted into the result.
// Every wait on an mbarrier is bounded in time; on expiry the kernel records an error code,
// lets its MMAs and every TMA copy either CTA issued settle (again bounded), frees its
// tensor memory and leaves, and the host reports APS_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "index.cuh"

namespace aps {
namespace {

constexpr int EPI_WARPS = 16;                     // four per TMEM lane quadrant
constexpr int DN_THREADS = 64 + 32 * EPI_WARPS;   // warp 0: TMA, warp 1: MMA + TMEM owner, then epilogue
constexpr int EPI_COLS = 256 / (EPI_WARPS / 4);   // accumulator columns one epilogue warp reads
constexpr int PAIR_ROWS = 256;                    // rows of an output block (both CTAs)
constexpr int TILE_ROWS = 128;                    // rows of one CTA's operand tile
constexpr int KBLK = 64;                          // bf16 elements per 128-byte swizzle row
constexpr int TILE_BYTES = TILE_ROWS * KBLK * 2;  // 16 KB
constexpr int SMEM_BUDGET = 224 * 1024;
constexpr int MAX_STAGES = 12;
constexpr int UNIT_BLOCKS = 32;  // B blocks per work unit
constexpr uint32_t TMEM_COLS = 512;  // two 256-column accumulators
constexpr unsigned long long WAIT_NS_DEFAULT = 2000000000ull;  // 2 s for one wait
constexpr unsigned long long WAIT_SPIN_CAP = 1ull << 28;       // iteration backstop of a wait

struct DenseParams {
    int n, KB, S;
    int nunits;
    const int4 *units;  // {A block, first B block, end B block, 0}, blocks of 256 rows
    float thr;
    unsigned long long *cand;
    unsigned long long cap;
    unsigned long long *count;   // candidate slots handed out (reserved in slabs)
    unsigned long long *padded;  // slots of those left holding CAND_PAD
    int *err;
    unsigned long long wait_ns;  // time limit of one mbarrier wait
    uint32_t stall;              // test hook: 1 = the MMA issuer waits for an accumulator release
                                 // that never comes, so the waits run out
    float *raw;                  // measurement: when set, every computed product S_ij (row-major n x n)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false, with an error code in *err, when the phase has not completed within
// limit_ns (or WAIT_SPIN_CAP probes); with heed_err, also false as soon as another role has
// given up. The first probe is inline; the spin is out of line.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity, int *err, int code,
                                            unsigned long long limit_ns, bool heed_err) {
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned long long i = 0; i < WAIT_SPIN_CAP; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 4095) == 4095) {
            if (heed_err && *(volatile int *)err) return false;
            if (globaltimer_ns() - t0 > limit_ns) break;
            __nanosleep(256);
        }
    }
    atomicCAS(err, 0, code);
    return false;
}

// a pipeline wait: gives up early once any role has failed
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code,
                                          unsigned long long limit_ns) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity, err, code, limit_ns, true);
}

// a wait for asynchronous work this kernel issued (MMAs, TMA copies) to settle before the
// CTA leaves: bounded in time only, whatever the other roles did
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity, int *err, int code,
                                           unsigned long long limit_ns) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity, err, code, limit_ns, false);
}

__device__ __forceinline__ void mbar_complete_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128 rows x 128 bytes written by TMA with
// 128-byte swizzle; 8-row core-matrix groups are 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint32_t a = smem_u32(p);
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFF) >> 4);   // start address (16-byte units)
    d |= (uint64_t)1 << 16;                // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;                // descriptor version
    d |= (uint64_t)2 << 61;                // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive columns of float32 from tensor memory (no wait).
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Largest of 64 values, as a balanced tree (no long dependency chain).
__device__ __forceinline__ float max64(const uint32_t *r) {
    float m[32];
#pragma unroll
    for (int k = 0; k < 32; k++) m[k] = fmaxf(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
#pragma unroll
    for (int w = 16; w; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; k++) m[k] = fmaxf(m[k], m[k + w]);
    return m[0];
}

__device__ __forceinline__ unsigned long long mask64(const uint32_t *r, float thr) {
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int k = 0; k < 32; k++) {
        lo |= (__uint_as_float(r[k]) >= thr ? 1u : 0u) << k;
        hi |= (__uint_as_float(r[k + 32]) >= thr ? 1u : 0u) << k;
    }
    return ((unsigned long long)hi << 32) | lo;
}

constexpr uint32_t EMIT_CHUNK = 256;            // candidate slots a warp reserves at a time
constexpr unsigned long long CAND_PAD = ~0ull;  // fills reserved slots that stay unused

// A warp's current slice of the candidate list: slots [base + used, base + lim) are its own.
// Reserving whole slices keeps the shared counter off the per-candidate path.
struct Slab {
    unsigned long long base;
    uint32_t used, lim;
    unsigned long long padded;  // slots of earlier slices filled with CAND_PAD
};

// Bits k of a 64-column slice starting at column j0 with i < j0 + k < n.
__device__ __forceinline__ unsigned long long tri_mask(int i, int j0, int n) {
    const int lo = max(i - j0 + 1, 0), hi = min(n - j0, 64);
    if (lo >= hi) return 0ull;
    const unsigned long long m = hi == 64 ? ~0ull : (1ull << hi) - 1ull;
    return m & (~0ull << lo);
}

// Warp-collective: the rest of the current slice becomes padding.
__device__ __forceinline__ void slab_close(Slab &w, unsigned long long *cand, unsigned long long cap) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = w.used + lane; k < w.lim; k += 32)
        if (w.base + k < cap) cand[w.base + k] = CAND_PAD;
    w.padded += w.lim - w.used;
    w.used = w.lim;
}

// Warp-collective append of the keys i * n + j0 + k, one per set bit k of each lane's mask;
// lanes are laid out in lane order inside the warp's slice.
__device__ __forceinline__ void slab_append(Slab &w, unsigned long long mask, int i, int j0, int n,
                                            unsigned long long *cand, unsigned long long cap,
                                            unsigned long long *count) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t c = (uint32_t)__popcll(mask);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (w.used + total > w.lim) {
        slab_close(w, cand, cap);
        const uint32_t want = max(EMIT_CHUNK, total);
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(count, (unsigned long long)want);
        w.base = __shfl_sync(0xffffffffu, b, 0);
        w.used = 0;
        w.lim = want;
    }
    unsigned long long pos = w.base + w.used + (incl - c);
    while (mask) {
        const int k = __ffsll((long long)mask) - 1;
        mask &= mask - 1ull;
        if (pos < cap) cand[pos] = (unsigned long long)i * (unsigned long long)n + (unsigned long long)(j0 + k);
        pos++;
    }
    w.used += total;
}

// Warp-collective, after a warp's last tile: close its slice and count its padding.
__device__ __forceinline__ void slab_finish(Slab &w, unsigned long long *cand, unsigned long long cap,
                                            unsigned long long *padded) {
    slab_close(w, cand, cap);
    if ((threadIdx.x & 31) == 0 && w.padded) atomicAdd(padded, w.padded);
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_to_rank(const void *p, uint32_t rank) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
    return out;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive, without release semantics, on a barrier of either CTA of the pair: used where the
// arrival only says that tensor-memory loads have completed (tcgen05.wait::ld), so no memory
// writes need to be made visible to the waiter.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar_cluster, int x,
                                                 int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on the barrier at this offset in both CTAs of the pair once prior MMAs complete
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// Instruction descriptor, kind::f16: BF16 A and B, float32 D, both K-major, M = N = 256
// (the pair's shape under cta_group::2).
__host__ __device__ constexpr uint32_t idesc_bf16_256x256() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

__global__ void __launch_bounds__(DN_THREADS, 1)
    dense_gemm_kernel(const __grid_constant__ CUtensorMap tmap, DenseParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int KB = P.KB, S = P.S;
    unsigned char *sA = smem;                                  // this CTA's 128 rows of A
    unsigned char *sB = smem + (size_t)KB * TILE_BYTES;        // this CTA's halves of the B stages
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)S * TILE_BYTES);
    uint64_t *a_full = bars, *a_empty = bars + 1, *done = bars + 2;
    uint64_t *b_full = bars + 3, *b_empty = b_full + S;
    uint64_t *d_full = b_empty + S, *d_empty = d_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d_empty + 2);
    uint32_t *loads = tmem_slot + 1;  // (A tiles, B stage fills) each CTA issued; the leader's copy
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        mbar_init(done, 1);
        for (int s = 0; s < S; s++) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&d_full[b], 1);
            mbar_init(&d_empty[b], 2 * EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            const uint32_t a_full_l = map_to_rank(a_full, 0);
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            uint32_t na = 0, nf = 0;
            bool ok = true;
            for (int u = cluster; u < P.nunits && ok; u += nclusters, it++) {
                const int4 U = P.units[u];
                if (it > 0 && !(ok = mbar_wait(a_empty, (uint32_t)(it - 1) & 1u, P.err, 1, P.wait_ns))) break;
                if (leader) mbar_expect_tx(a_full, (uint32_t)(2 * KB * TILE_BYTES));
                for (int kb = 0; kb < KB; kb++)
                    tma_load_2d_pair(sA + (size_t)kb * TILE_BYTES, &tmap, a_full_l, kb * KBLK,
                                     U.x * PAIR_ROWS + (int)rank * TILE_ROWS);
                na++;
                for (int bc = U.y; bc < U.z && ok; bc++) {
                    for (int kb = 0; kb < KB; kb++) {
                        if (!(ok = mbar_wait(&b_empty[stage], phase ^ 1u, P.err, 2, P.wait_ns))) break;
                        if (leader) mbar_expect_tx(&b_full[stage], (uint32_t)(2 * TILE_BYTES));
                        tma_load_2d_pair(sB + (size_t)stage * TILE_BYTES, &tmap, map_to_rank(&b_full[stage], 0),
                                         kb * KBLK, bc * PAIR_ROWS + (int)rank * TILE_ROWS);
                        nf++;
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // the leader settles every copy either CTA issued before the pair leaves
            st_cluster_u32(map_to_rank(&loads[2 * rank], 0), na);
            st_cluster_u32(map_to_rank(&loads[2 * rank + 1], 0), nf);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer (even CTA)
        if (lane == 0 && leader) {
            const uint32_t idesc = idesc_bf16_256x256();
            const uint64_t adesc0 = smem_desc(sA), bdesc0 = smem_desc(sB);
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t uses[2] = {0, 0};
            int it = 0;
            bool ok = true;
            for (int u = cluster; u < P.nunits && ok; u += nclusters, it++) {
                const int4 U = P.units[u];
                if (!(ok = mbar_wait(a_full, (uint32_t)it & 1u, P.err, 3, P.wait_ns))) break;
                for (int bc = U.y; bc < U.z && ok; bc++) {
                    if (!(ok = mbar_wait(&d_empty[buf], (uses[buf] & 1u) ^ 1u ^ P.stall, P.err, 4, P.wait_ns))) break;
                    tc_fence_after();
                    const uint32_t td = tmem + (uint32_t)(buf * 256);
                    for (int kb = 0; kb < KB; kb++) {
                        if (!(ok = mbar_wait(&b_full[stage], phase, P.err, 5, P.wait_ns))) break;
                        const uint64_t bdesc = bdesc0 + (uint64_t)(stage * (TILE_BYTES >> 4));
                        const uint64_t adesc = adesc0 + (uint64_t)(kb * (TILE_BYTES >> 4));
#pragma unroll
                        for (int k16 = 0; k16 < KBLK / 16; k16++)
                            umma_bf16_pair(td, adesc + 2u * k16, bdesc + 2u * k16, idesc, (kb | k16) != 0);
                        umma_commit_pair(&b_empty[stage]);  // frees the stage in both CTAs
                        if (++stage == S) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    umma_commit_pair(&d_full[buf]);
                    uses[buf]++;
                    buf ^= 1;
                }
                umma_commit_pair(a_empty);
            }
            umma_commit_pair(done);
            mbar_drain(done, 0, P.err, 6, P.wait_ns);  // every MMA has finished with TMEM and shared memory
        }
    } else {
        // ------------------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;  // which EPI_COLS-column slice of the 256 columns
        int buf = 0;
        uint32_t uses[2] = {0, 0};
        bool ok = true;
        Slab w = {0ull, 0u, 0u, 0ull};
        for (int u = cluster; u < P.nunits && ok; u += nclusters) {
            const int4 U = P.units[u];
            const int i = U.x * PAIR_ROWS + (int)rank * TILE_ROWS + q * 32 + lane;
            for (int bc = U.y; bc < U.z; bc++) {
                if (!(ok = __all_sync(0xffffffffu, mbar_wait(&d_full[buf], uses[buf] & 1u, P.err, 7, P.wait_ns)))) break;
                tc_fence_after();
                uint32_t r[EPI_COLS];
                const uint32_t col = (uint32_t)(buf * 256 + h * EPI_COLS);
#pragma unroll
                for (int cc = 0; cc < EPI_COLS / 32; cc++)
                    tmem_ld32_issue(tmem + ((uint32_t)(q * 32) << 16) + col + 32 * cc, r + 32 * cc);
                tmem_ld_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(map_to_rank(&d_empty[buf], 0));
                if (P.raw && i < P.n) {  // (measurement only) this thread's row slice of the products
                    const int jb = bc * PAIR_ROWS + h * EPI_COLS;
                    for (int kk = 0; kk < EPI_COLS; kk++)
                        if (jb + kk < P.n) P.raw[(int64_t)i * P.n + jb + kk] = __uint_as_float(r[kk]);
                }
                for (int cc = 0; cc < EPI_COLS / 64; cc++) {
                    const int j0 = bc * PAIR_ROWS + h * EPI_COLS + cc * 64;
                    unsigned long long m = 0ull;
                    if (max64(r + 64 * cc) >= P.thr && i < P.n) m = mask64(r + 64 * cc, P.thr) & tri_mask(i, j0, P.n);
                    if (__any_sync(0xffffffffu, m != 0ull)) slab_append(w, m, i, j0, P.n, P.cand, P.cap, P.count);
                }
                uses[buf]++;
                buf ^= 1;
            }
        }
        slab_finish(w, P.cand, P.cap, P.padded);
    }
    __syncthreads();
    cluster_sync_all();  // every role of both CTAs is done; both load counts are published
    if (leader && warp == 0 && lane == 0) {
        // A phase of a_full / b_full[s] is left open when one CTA issued its half of a copy
        // and the other did not (a wait ran out between the two): the missing half is
        // accounted for, then the last phase is awaited, so no copy lands after exit. Within
        // one barrier the CTAs' counts differ by at most one fill, and every earlier phase
        // has completed (the MMA waited on it before the refill was allowed).
        const uint32_t naL = loads[0], nfL = loads[1], naO = loads[2], nfO = loads[3];
        for (int b = -1; b < S; b++) {
            uint64_t *bar = b < 0 ? a_full : &b_full[b];
            const uint32_t half = b < 0 ? (uint32_t)(KB * TILE_BYTES) : (uint32_t)TILE_BYTES;
            const uint32_t cL = b < 0 ? naL : nfL / S + ((uint32_t)b < nfL % S ? 1u : 0u);
            const uint32_t cO = b < 0 ? naO : nfO / S + ((uint32_t)b < nfO % S ? 1u : 0u);
            const uint32_t c = max(cL, cO);
            if (c == 0) continue;
            if (cL > cO) mbar_complete_tx(bar, half);  // armed for both halves; the peer's never left
            if (cO > cL) mbar_expect_tx(bar, half);    // the peer's half was never armed for
            mbar_drain(bar, (c - 1) & 1u, P.err, 8, P.wait_ns);
        }
    }
    __syncwarp();
    cluster_sync_all();  // the peer no longer touches this CTA's barriers, copies or tensor memory
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// One warp per row: float64 norm; with normalise, rows are scaled into Y; otherwise a row
// whose norm is off by more than 1e-3 (or holds a non-finite value) is reported in *bad.
__global__ void k_dense_rows(const float *__restrict__ X, int64_t n, int d, int normalise, float *Y,
                             unsigned long long *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += nw) {
        double ss = 0.0;
        bool finite = true;
        for (int e = lane; e < d; e += 32) {
            const float v = X[r * d + e];
            finite = finite && isfinite(v);
            ss += (double)v * (double)v;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        finite = __all_sync(0xffffffffu, finite);
        const double nrm = sqrt(ss);
        if (normalise) {
            const double sc = nrm > 0.0 ? 1.0 / nrm : 0.0;
            for (int e = lane; e < d; e += 32) Y[r * d + e] = (float)((double)X[r * d + e] * sc);
            if (lane == 0 && (!finite || nrm == 0.0)) atomicMin(bad, (unsigned long long)r);
        } else if (lane == 0 && (!finite || fabs(nrm - 1.0) > 1e-3)) {
            atomicMin(bad, (unsigned long long)r);
        }
    }
}

__global__ void k_to_bf16(const float *__restrict__ X, int64_t n, int d, int64_t n_pad, __nv_bfloat16 *Xb) {
    const int64_t total = n_pad * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        Xb[e] = (e < n * d) ? __float2bfloat16_rn(X[e]) : __float2bfloat16_rn(0.f);
}

// Exact rescoring of the candidates (sorted keys i*n + j). Each warp takes a contiguous run
// of candidates and scores four at a time, issuing all their row loads (float4) before any
// arithmetic, so that four pairs' reads are in flight per warp; consecutive candidates share
// row i, which then comes from L1. float32 dot with a tree reduction; float64 when the
// float32 score lies within the band of t. X is 16-byte aligned and d % 64 == 0, d <= 512.
constexpr int RS_BATCH = 4;

__global__ void k_rescore(const unsigned long long *__restrict__ keys, int64_t nc, const float *__restrict__ X, int n,
                          int d, float t, float beta, int32_t *keep, float *score, unsigned long long *nband) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t per = (nc + nw - 1) / nw;
    const int64_t c0 = wid * per, c1 = min(nc, c0 + per);
    const int d4 = d >> 2;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    for (int64_t c = c0; c < c1; c += RS_BATCH) {
        int64_t ii[RS_BATCH], jj[RS_BATCH];
        float acc[RS_BATCH];
#pragma unroll
        for (int u = 0; u < RS_BATCH; u++) {
            const unsigned long long k = keys[min(c + u, c1 - 1)];
            ii[u] = (int64_t)(k / (unsigned long long)n);
            jj[u] = (int64_t)(k % (unsigned long long)n);
            acc[u] = 0.f;
        }
#pragma unroll
        for (int v = 0; v < 4; v++) {
            if (lane + 32 * v < d4) {
                float4 a[RS_BATCH], b[RS_BATCH];
#pragma unroll
                for (int u = 0; u < RS_BATCH; u++) {
                    a[u] = X4[ii[u] * d4 + lane + 32 * v];
                    b[u] = X4[jj[u] * d4 + lane + 32 * v];
                }
#pragma unroll
                for (int u = 0; u < RS_BATCH; u++) {
                    acc[u] = fmaf(a[u].x, b[u].x, acc[u]);
                    acc[u] = fmaf(a[u].y, b[u].y, acc[u]);
                    acc[u] = fmaf(a[u].z, b[u].z, acc[u]);
                    acc[u] = fmaf(a[u].w, b[u].w, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < RS_BATCH; u++) {
#pragma unroll
            for (int o = 16; o; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
        }
        for (int u = 0; u < RS_BATCH && c + u < c1; u++) {
            float s = acc[u];
            bool in = s >= t;
            if (fabsf(s - t) <= beta) {
                const float *xi = X + ii[u] * d, *xj = X + jj[u] * d;
                double a64 = 0.0;
                for (int e = lane; e < d; e += 32) a64 += (double)xi[e] * (double)xj[e];
#pragma unroll
                for (int o = 16; o; o >>= 1) a64 += __shfl_xor_sync(0xffffffffu, a64, o);
                in = a64 >= (double)t;
                s = (float)a64;
                if (lane == 0) atomicAdd(nband, 1ull);
            }
            if (lane == 0) {
                keep[c + u] = in ? 1 : 0;
                score[c + u] = s;
            }
        }
    }
}

__global__ void k_compact(const unsigned long long *__restrict__ keys, const int32_t *__restrict__ keep,
                          const float *__restrict__ score, const int64_t *__restrict__ pos, int64_t nc, int n,
                          int32_t *oi, int32_t *oj, float *os) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[c]) continue;
        const int64_t p = pos[c];
        oi[p] = (int32_t)(keys[c] / (unsigned long long)n);
        oj[p] = (int32_t)(keys[c] % (unsigned long long)n);
        os[p] = score[c];
    }
}

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);

aps_status encode_map(CUtensorMap *map, void *base, int64_t rows, int d) {
    static PFN_encodeTiled_t fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return APS_EUNSUPPORTED;
        }
        fn = reinterpret_cast<PFN_encodeTiled_t>(p);
    }
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d * 2};
    cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)TILE_ROWS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return APS_ECUDA;
    }
    return APS_OK;
}

std::atomic<int64_t> g_dense_hint{0};
std::atomic<int64_t> g_dense_stall{0};                // launches left to stall (test hook)
std::atomic<unsigned long long> g_dense_stall_ns{0};  // their wait limit; 0 = the default

}  // namespace

void dense_debug_stall(int64_t launches, uint64_t wait_ns) {
    g_dense_stall_ns.store(wait_ns);
    g_dense_stall.store(launches > 0 ? launches : 0);
}

// Margin of the BF16 candidate test for unit vectors of dimension d: rounding both operands
// to BF16 (unit roundoff 2^-8) changes x.y by at most (2u + u^2) ||x|| ||y||, the float32
// accumulation adds at most 2 d 2^-23, and the 1e-3 norm tolerance scales by 1.002.
double dense_margin(int d) {
    const double u = std::ldexp(1.0, -8);
    return (2.0 * u + u * u) * 1.002 + 2.0 * d * std::ldexp(1.0, -23);
}

aps_status dense_all_pairs_device(const float *X, int32_t n, int32_t d, float t, cudaStream_t s, aps_pairs *out,
                                  aps_stats *stats, float *raw) {
    int dev = 0, major = 0, minor = 0;
    APS_CUDA(cudaGetDevice(&dev));
    APS_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    APS_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (major != 10 || minor != 3) {
        set_error("the dense path needs an sm_103 device (found sm_%d%d)", major, minor);
        return APS_EUNSUPPORTED;
    }
    const int KB = d / KBLK;
    const int64_t n_pad = std::max<int64_t>(PAIR_ROWS, ((int64_t)n + PAIR_ROWS - 1) / PAIR_ROWS * PAIR_ROWS);
    const int S = std::min(MAX_STAGES, (SMEM_BUDGET - KB * TILE_BYTES) / TILE_BYTES);
    const int smem = (KB + S) * TILE_BYTES + 1024 + 512;  // operands, alignment slack, barriers
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; i++) APS_CUDA(cudaEventCreate(&ev[i]));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 5; i++) cudaEventDestroy(e[i]);
        }
    } evg{ev};
    APS_CUDA(cudaEventRecord(ev[0], s));
    DBuf<__nv_bfloat16> Xb;
    APS_TRY(Xb.alloc((size_t)(n_pad * d), s));
    k_to_bf16<<<grid_for(n_pad * d, 256, 65536), 256, 0, s>>>(X, n, d, n_pad, Xb.p);
    APS_LAUNCH_CHECK();
    CUtensorMap map;
    APS_TRY(encode_map(&map, Xb.p, n_pad, d));
    // work units: (A block, run of B blocks), B blocks from the diagonal onward
    const int64_t nb = n_pad / PAIR_ROWS;
    std::vector<int4> units;
    for (int64_t a = 0; a < nb; a++)
        for (int64_t b = a; b < nb; b += UNIT_BLOCKS)
            units.push_back(make_int4((int)a, (int)b, (int)std::min<int64_t>(b + UNIT_BLOCKS, nb), 0));
    // longest units first: the clusters take them round-robin, so the short tail units
    // even out the finish
    std::stable_sort(units.begin(), units.end(), [](const int4 &p, const int4 &q) { return p.z - p.y > q.z - q.y; });
    DBuf<int4> dunits;
    APS_TRY(dunits.alloc(units.size(), s));
    APS_CUDA(cudaMemcpyAsync(dunits.p, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice, s));
    DBuf<unsigned long long> ctr;
    DBuf<int> err;
    APS_TRY(ctr.alloc(4, s));
    APS_TRY(err.alloc(1, s));
    constexpr int SMEM_MAX = SMEM_BUDGET + 1024 + 512;
    APS_CUDA(cudaFuncSetAttribute(dense_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAX));
    const double delta = dense_margin(d);
    // one cluster per SM pair that can be resident at once
    static int max_clusters = 0;
    if (!max_clusters) {
        cudaLaunchConfig_t q;
        memset(&q, 0, sizeof(q));
        q.gridDim = dim3((unsigned)(num_sms() & ~1));
        q.blockDim = dim3(DN_THREADS);
        q.dynamicSmemBytes = (size_t)SMEM_MAX;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = 2;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int c = 0;
        APS_CUDA(cudaOccupancyMaxActiveClusters(&c, dense_gemm_kernel, &q));
        max_clusters = std::max(1, c);
    }
    const int npairs_sm = std::max(1, std::min<int>(max_clusters, (int)units.size()));
    int64_t cap = std::max<int64_t>({g_dense_hint.load(), (int64_t)1 << 22, (int64_t)n * 4});
    DBuf<unsigned long long> cand;
    int64_t nslots = 0, npad = 0;
    float ms_gemm = 0.f;
    for (int attempt = 0; attempt < 2; attempt++) {
        APS_TRY(cand.alloc((size_t)cap, s));
        APS_CUDA(cudaMemsetAsync(ctr.p, 0, 4 * sizeof(unsigned long long), s));
        APS_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
        DenseParams P;
        P.n = n;
        P.KB = KB;
        P.S = S;
        P.nunits = (int)units.size();
        P.units = dunits.p;
        P.thr = raw ? INFINITY : (float)((double)t - delta);
        P.cand = cand.p;
        P.cap = (unsigned long long)cap;
        P.count = ctr.p;
        P.padded = ctr.p + 2;
        P.err = err.p;
        P.wait_ns = WAIT_NS_DEFAULT;
        P.stall = 0;
        P.raw = raw;
        for (int64_t k = g_dense_stall.load(); k > 0;)
            if (g_dense_stall.compare_exchange_weak(k, k - 1)) {
                P.stall = 1;
                if (g_dense_stall_ns.load()) P.wait_ns = g_dense_stall_ns.load();
                break;
            }
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(2 * npairs_sm));
        cfg.blockDim = dim3(DN_THREADS);
        cfg.dynamicSmemBytes = (size_t)smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        APS_CUDA(cudaEventRecord(ev[1], s));
        APS_CUDA(cudaLaunchKernelEx(&cfg, dense_gemm_kernel, map, P));
        count_launch();
        APS_CUDA(cudaEventRecord(ev[2], s));
        unsigned long long cnt[3] = {0, 0, 0};
        int e_h = 0;
        APS_CUDA(cudaMemcpyAsync(cnt, ctr.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaMemcpyAsync(&e_h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        APS_CUDA(cudaStreamSynchronize(s));
        if (e_h) {
            set_error("dense tensor-core kernel: a pipeline wait timed out (code %d)", e_h);
            return APS_ETIMEOUT;
        }
        cudaEventElapsedTime(&ms_gemm, ev[1], ev[2]);
        if (raw) {  // the products are written: no candidates to finish
            out->count = 0;
            return APS_OK;
        }
        nslots = (int64_t)cnt[0];
        npad = (int64_t)cnt[2];
        if (nslots <= cap) break;
        cap = nslots + nslots / 8 + 1024;
    }
    g_dense_hint.store(nslots + nslots / 8 + 1024);
    // sort by (i, j): the slots hold nc candidates and npad CAND_PAD keys, which sort last
    DBuf<uint32_t> dummy;
    APS_TRY(dummy.alloc((size_t)std::max<int64_t>(nslots, 1), s));
    if (nslots > 1) {
        APS_CUDA(cudaMemsetAsync(dummy.p, 0, sizeof(uint32_t) * nslots, s));
        APS_TRY(sort_pairs(reinterpret_cast<uint64_t *>(cand.p), dummy.p, nslots,
                           bits_for((uint64_t)n * (uint64_t)n), s));
    }
    const int64_t nc = nslots - npad;
    APS_CUDA(cudaEventRecord(ev[3], s));
    DBuf<int32_t> keep;
    DBuf<float> sc;
    DBuf<int64_t> pos;
    APS_TRY(keep.alloc((size_t)std::max<int64_t>(nc, 1), s));
    APS_TRY(sc.alloc((size_t)std::max<int64_t>(nc, 1), s));
    APS_TRY(pos.alloc((size_t)nc + 1, s));
    const float beta = (float)std::max(1e-5, (d / 32.0 + 8.0) * std::ldexp(1.0, -23));
    if (nc > 0) {
        k_rescore<<<grid_for(nc * 32, 256, (int64_t)num_sms() * 64), 256, 0, s>>>(cand.p, nc, X, n, d, t, beta,
                                                                                   keep.p, sc.p, ctr.p + 1);
        APS_LAUNCH_CHECK();
    }
    APS_TRY(scan_exclusive(keep.p, pos.p, nc, s));
    int64_t npairs = 0;
    unsigned long long nband = 0;
    APS_CUDA(cudaMemcpyAsync(&npairs, pos.p + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaMemcpyAsync(&nband, ctr.p + 1, sizeof(nband), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    PairsAlloc *pa = new PairsAlloc();
    pa->stream = s;
    const size_t seg = ((size_t)npairs * 4 + 127) & ~(size_t)127;
    aps_status st = dalloc(&pa->block, std::max<size_t>(3 * seg, 256), s);
    if (st != APS_OK) {
        delete pa;
        return st;
    }
    char *b = static_cast<char *>(pa->block);
    int32_t *oi = reinterpret_cast<int32_t *>(b);
    int32_t *oj = reinterpret_cast<int32_t *>(b + seg);
    float *os = reinterpret_cast<float *>(b + 2 * seg);
    if (nc > 0) {
        k_compact<<<grid_for(nc, 256, 65536), 256, 0, s>>>(cand.p, keep.p, sc.p, pos.p, nc, n, oi, oj, os);
        APS_LAUNCH_CHECK();
    }
    APS_CUDA(cudaEventRecord(ev[4], s));
    APS_CUDA(cudaEventSynchronize(ev[4]));
    float ms_total = 0, ms_out = 0;
    cudaEventElapsedTime(&ms_total, ev[0], ev[4]);
    cudaEventElapsedTime(&ms_out, ev[2], ev[4]);
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->candidates = nc;
        stats->verified = nc;
        stats->pairs = npairs;
        stats->band = (int64_t)nband;
        stats->evaluations = (int64_t)n * (n - 1) / 2;
        stats->visits = (int64_t)n * n / 2 * d;  // multiply-adds of the upper triangle
        stats->ms_join = ms_gemm;
        stats->ms_sort = ms_out;
        stats->ms_total = ms_total;
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

// Validate (or normalise) the rows of X and run the dense join.
aps_status dense_all_pairs(const float *X, int32_t n, int32_t d, float t, uint32_t flags, cudaStream_t s,
                           aps_pairs *out, aps_stats *stats) {
    DBuf<float> dx, dy;
    const float *Xd = X;
    if (!(flags & APS_DEVICE_PTRS) || (reinterpret_cast<uintptr_t>(X) & 15)) {  // host, or not 16-byte aligned
        APS_TRY(dx.alloc((size_t)n * d, s));
        if ((int64_t)n * d) APS_CUDA(cudaMemcpyAsync(dx.p, X, sizeof(float) * (size_t)n * d, cudaMemcpyDefault, s));
        Xd = dx.p;
    }
    DBuf<unsigned long long> bad;
    APS_TRY(bad.alloc(1, s));
    APS_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
    const bool norm = (flags & APS_NORMALIZE) != 0;
    if (norm) APS_TRY(dy.alloc((size_t)n * d, s));
    if (n > 0) {
        k_dense_rows<<<grid_for((int64_t)n * 32, 256, 65536), 256, 0, s>>>(Xd, n, d, norm ? 1 : 0, dy.p, bad.p);
        APS_LAUNCH_CHECK();
    }
    unsigned long long b = 0;
    APS_CUDA(cudaMemcpyAsync(&b, bad.p, sizeof(b), cudaMemcpyDeviceToHost, s));
    APS_CUDA(cudaStreamSynchronize(s));
    if (b != ~0ull) {
        set_error(norm ? "row %llu is zero or holds a non-finite value"
                       : "row %llu: L2 norm differs from 1 by more than 1e-3 or a value is not finite "
                         "(pass APS_NORMALIZE)",
                  b);
        return APS_EINVAL;
    }
    return dense_all_pairs_device(norm ? dy.p : Xd, n, d, t, s, out, stats, nullptr);
}

// The tensor cores' float32 products S = X_bf16 . X_bf16^T of the dense path (rows as they
// are, no validation), each computed entry written to raw (row-major n x n); entries of
// 256-row blocks below the diagonal are not computed and left as they were.
aps_status dense_tensor_products(const float *X, int32_t n, int32_t d, cudaStream_t s, float *raw) {
    aps_pairs none;
    memset(&none, 0, sizeof(none));
    return dense_all_pairs_device(X, n, d, 0.f, s, &none, nullptr, raw);
}

}  // namespace aps
