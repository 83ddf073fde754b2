// Self-join entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc while they join: a serving process whose device
// memory is fully reserved by its own allocator up front, or a host thread that must not
// take the allocator's locks (or trigger an implicit device synchronisation) on its
// latency path. For them aps_all_pairs_noalloc runs the join of an index that already
// exists with all of its scratch taken from one fixed array declared below, and writes the
// pairs into buffers the caller owns.
#include <mutex>

#include "index.cuh"

namespace {

// Scratch for one join: counters, per-(vector, window) counts and offsets, the segment
// table, the per-warp lists of emitted pairs of at most kMaxCtas CTAs, and the pair
// staging buffer in the rest. A file-scope device array: every GPU on which this part of
// the library is loaded holds these 64 MiB until the process exits.
constexpr size_t kArenaBytes = 64ull << 20;
constexpr int kMaxCtas = 32;
__device__ __align__(256) unsigned char g_arena[kArenaBytes];

// In host code `g_arena` names a host-side stand-in, not device memory: kernels get the
// device address looked up once per device.
std::mutex g_mu;
void *g_arena_dev[256];

aps_status arena_address(int dev, void **out) {
    cudaError_t e;
    if (dev < 0 || dev >= 256) {
        aps::set_error("device ordinal %d out of range", dev);
        return APS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_arena_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_arena);
        if (e != cudaSuccess || !p) return aps::cuda_status(e, "cudaGetSymbolAddress(arena)", __FILE__, __LINE__);
        g_arena_dev[dev] = p;
    }
    *out = g_arena_dev[dev];
    return APS_OK;
}

}  // namespace

extern "C" aps_status aps_all_pairs_noalloc(aps_index *index, int32_t *i, int32_t *j, float *score, int64_t capacity,
                                            int64_t *count, void *stream) {
    if (!index || !count) {
        aps::set_error("index and count must not be NULL");
        return APS_EINVAL;
    }
    *count = 0;
    if (capacity < 0 || (capacity > 0 && (!i || !j || !score))) {
        aps::set_error("need capacity >= 0 and device arrays i, j, score when capacity > 0");
        return APS_EINVAL;
    }
    if (index->k != 1) {
        aps::set_error("aps_all_pairs_noalloc needs a single-instance index");
        return APS_EINVAL;
    }
    // The arena used is the current device's; the index's arrays live on index->device.
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return aps::cuda_status(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev != index->device) {
        aps::set_error("the current device (%d) is not the index's device (%d)", dev, index->device);
        return APS_EINVAL;
    }
    // The output arrays are written by kernels: they must be device memory of this device
    // (a host pointer would fault or, where the GPU can reach host memory, write there).
    if (capacity > 0) {
        const void *outs[3] = {i, j, score};
        for (const void *q : outs) {
            cudaPointerAttributes pa;
            e = cudaPointerGetAttributes(&pa, q);
            if (e != cudaSuccess) {
                cudaGetLastError();
                aps::set_error("output array %p is not CUDA memory", q);
                return APS_EINVAL;
            }
            if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev) {
                aps::set_error("output array %p is not device memory of device %d", q, dev);
                return APS_EINVAL;
            }
        }
    }
    void *arena = nullptr;
    APS_TRY(arena_address(dev, &arena));
    return aps::join_noalloc(index, static_cast<unsigned char *>(arena), kArenaBytes, kMaxCtas, i, j, score,
                             capacity, count, static_cast<cudaStream_t>(stream));
}
