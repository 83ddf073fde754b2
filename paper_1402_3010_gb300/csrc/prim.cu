// Error state, device memory and the generic device primitives (prefix sum, stable
// radix sort) used by the index build and the output stage.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "aps_internal.cuh"

namespace aps {

// ------------------------------------------------------------------ error state
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

aps_status cuda_status(cudaError_t e, const char *what, const char *file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        return APS_ENOMEM;
    }
    return APS_ECUDA;
}

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ------------------------------------------------------------------ memory
static std::mutex g_pool_mu;
static bool g_pool_ready[64];
// test hook: the k-th device allocation from now fails (atomic: serving slots allocate
// from their own threads)
static std::atomic<int64_t> g_alloc_fault{0};

void set_alloc_fault(int64_t k) { g_alloc_fault.store(k); }

static void pool_setup() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready[dev] = true;
}

aps_status dalloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (g_alloc_fault.load() > 0 && g_alloc_fault.fetch_sub(1) == 1) {
        set_error("device allocation of %zu bytes failed (injected)", bytes);
        return APS_ENOMEM;
    }
    pool_setup();
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 1, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? APS_ENOMEM : APS_ECUDA;
    }
    return APS_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------------ pinned host blocks
static std::mutex g_host_mu;
static std::vector<void *> g_host_free[64];  // cached blocks by size class (2^c bytes)
static size_t g_host_cached = 0;
constexpr size_t HOST_CACHE_MAX = (size_t)8 << 30;

static int host_class(size_t bytes) {
    int c = 20;  // 1 MiB
    while (c < 63 && ((size_t)1 << c) < bytes) c++;
    return c;
}

aps_status halloc(void **p, size_t bytes) {
    *p = nullptr;
    const int c = host_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        if (!g_host_free[c].empty()) {
            *p = g_host_free[c].back();
            g_host_free[c].pop_back();
            g_host_cached -= (size_t)1 << c;
            return APS_OK;
        }
    }
    cudaError_t e = cudaMallocHost(p, (size_t)1 << c);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return cuda_status(e, "cudaMallocHost", __FILE__, __LINE__);
    }
    return APS_OK;
}

void hfree(void *p, size_t bytes) {
    if (!p) return;
    const int c = host_class(bytes);
    {
        std::lock_guard<std::mutex> lk(g_host_mu);
        if (g_host_cached + ((size_t)1 << c) <= HOST_CACHE_MAX) {
            g_host_free[c].push_back(p);
            g_host_cached += (size_t)1 << c;
            return;
        }
    }
    cudaFreeHost(p);
}

// ------------------------------------------------------------------ prefix sum
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__global__ void scan_reduce_kernel(const T *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t acc = 0;
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) acc += (int64_t)in[i];
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += warp_tot[w];
        sums[blockIdx.x] = t;
    }
}

// Each block scans its tile (thread t owns items [t*ITEMS, (t+1)*ITEMS) of the tile) and
// adds the scanned block offset.
template <class T>
__global__ void scan_down_kernel(const T *__restrict__ in, int64_t n, const int64_t *__restrict__ offs,
                                 int64_t *__restrict__ out) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t local = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        local += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int64_t wbase = 0;
    for (int w = 0; w < warp; w++) wbase += warp_tot[w];
    int64_t run = offs[blockIdx.x] + wbase + inc - local;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

template <class T>
aps_status scan_impl(const T *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        APS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return APS_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    DBuf<int64_t> offs;
    if (nb == 1) {
        APS_TRY(offs.alloc(1, s));
        APS_CUDA(cudaMemsetAsync(offs.p, 0, sizeof(int64_t), s));
    } else {
        DBuf<int64_t> sums;
        APS_TRY(sums.alloc((size_t)nb, s));
        scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, sums.p);
        APS_LAUNCH_CHECK();
        APS_TRY(offs.alloc((size_t)nb + 1, s));
        APS_TRY(scan_impl<int64_t>(sums.p, offs.p, nb, s));
    }
    scan_down_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, offs.p, out);
    APS_LAUNCH_CHECK();
    return APS_OK;
}

}  // namespace

aps_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
}
aps_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

// ------------------------------------------------------------------ radix sort
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;
constexpr int RS_DIGITS = 256;

// Digit histogram of each tile, stored digit-major: hist[d * nblocks + block], so that an
// exclusive scan of the whole array gives each (digit, block) its output offset.
__global__ void rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t n, int shift,
                               int32_t *__restrict__ hist) {
    __shared__ int32_t h[RS_DIGITS];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: a tile is first ranked into shared memory by digit (items visited in
// input order: round by round, lane order inside a warp, warp order inside a round), then
// written out in digit runs, each run to consecutive addresses after all earlier items of
// its digit. rs_smem holds the tile's keys and values (RS_TILE each).
constexpr int RS_SMEM = RS_TILE * (8 + 4);

__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(const uint64_t *__restrict__ kin,
                                                                  const uint32_t *__restrict__ vin,
                                                                  uint64_t *__restrict__ kout,
                                                                  uint32_t *__restrict__ vout, int64_t n, int shift,
                                                                  const int64_t *__restrict__ offs) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(rs_smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + RS_TILE);
    __shared__ int64_t gbase[RS_DIGITS];  // output offset of (digit, this tile)
    __shared__ int32_t lbase[RS_DIGITS];  // tile-local start of each digit
    __shared__ int32_t cur[RS_DIGITS];    // tile-local cursor of each digit
    __shared__ int32_t wc[RS_WARPS][RS_DIGITS];
    __shared__ int32_t wsum[RS_WARPS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t nb = gridDim.x;
    const int64_t hi = (int64_t)t * nb + blockIdx.x;
    gbase[t] = offs[hi];
    // exclusive scan of the tile's digit counts (offs is the digit-major scan of them)
    const int c = (int)(offs[hi + 1] - offs[hi]);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; w++) before += wsum[w];
    lbase[t] = before + inc - c;
    cur[t] = before + inc - c;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; r++) {
        for (int w = 0; w < RS_WARPS; w++) wc[w][t] = 0;
        __syncthreads();
        const int64_t i = tile + (int64_t)r * RS_THREADS + t;
        const bool valid = i < n;
        const uint64_t k = valid ? kin[i] : 0;
        const uint32_t v = valid ? vin[i] : 0;
        const int d = (int)((k >> shift) & 0xff);
        const unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned peers = 0;
        int rank = 0;
        if (valid) {
            peers = __match_any_sync(vmask, d);
            rank = __popc(peers & lt_mask);
            if (rank == 0) wc[warp][d] = __popc(peers);
        }
        __syncthreads();
        {  // per digit: warp counts -> tile-local warp bases
            int acc = cur[t];
            for (int w = 0; w < RS_WARPS; w++) {
                const int cw = wc[w][t];
                wc[w][t] = acc;
                acc += cw;
            }
            cur[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const int q = wc[warp][d] + rank;
            sk[q] = k;
            sv[q] = v;
        }
        __syncthreads();
    }
    // write out in tile order: consecutive items of a digit go to consecutive addresses
    const int tn = (int)min((int64_t)RS_TILE, n - tile);
    for (int q = t; q < tn; q += RS_THREADS) {
        const uint64_t k = sk[q];
        const int d = (int)((k >> shift) & 0xff);
        const int64_t dst = gbase[d] + (q - lbase[d]);
        kout[dst] = k;
        vout[dst] = sv[q];
    }
}

}  // namespace

aps_status sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return APS_OK;
    int passes = (bits + 7) / 8;
    int64_t nb = (n + RS_TILE - 1) / RS_TILE;
    DBuf<uint64_t> k2;
    DBuf<uint32_t> v2;
    DBuf<int32_t> hist;
    DBuf<int64_t> offs;
    APS_TRY(k2.alloc((size_t)n, s));
    APS_TRY(v2.alloc((size_t)n, s));
    APS_TRY(hist.alloc((size_t)(nb * RS_DIGITS), s));
    APS_TRY(offs.alloc((size_t)(nb * RS_DIGITS + 1), s));
    APS_CUDA(cudaFuncSetAttribute(rs_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM));
    uint64_t *ka = keys, *kb = k2.p;
    uint32_t *va = vals, *vb = v2.p;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        rs_hist_kernel<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, n, shift, hist.p);
        APS_LAUNCH_CHECK();
        APS_TRY(scan_exclusive(hist.p, offs.p, nb * RS_DIGITS, s));
        rs_scatter_kernel<<<(unsigned)nb, RS_THREADS, RS_SMEM, s>>>(ka, va, kb, vb, n, shift, offs.p);
        APS_LAUNCH_CHECK();
        uint64_t *tk = ka;
        ka = kb;
        kb = tk;
        uint32_t *tv = va;
        va = vb;
        vb = tv;
    }
    if (ka != keys) {
        APS_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        APS_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return APS_OK;
}

}  // namespace aps

extern "C" const char *aps_last_error(void) { return aps::g_err; }
extern "C" int64_t aps_launch_count(void) { return aps::g_launches.load(); }
