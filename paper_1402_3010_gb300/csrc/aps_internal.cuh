// Internal declarations shared by the CUDA sources of libaps.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstddef>
#include <vector>

#include "../../include/aps.h"

namespace aps {

// ---------------------------------------------------------------- error handling
void set_error(const char *fmt, ...);
aps_status cuda_status(cudaError_t e, const char *what, const char *file, int line);

#define APS_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) return ::aps::cuda_status(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define APS_TRY(expr)                      \
    do {                                   \
        aps_status s_ = (expr);            \
        if (s_ != APS_OK) return s_;       \
    } while (0)

// Every kernel launch site is followed by APS_LAUNCH_CHECK(), which also counts launches.
void count_launch();
#define APS_LAUNCH_CHECK()               \
    do {                                 \
        ::aps::count_launch();           \
        APS_CUDA(cudaGetLastError());    \
    } while (0)

// ---------------------------------------------------------------- device memory
// Stream-ordered allocations from the device's default memory pool, whose release
// threshold is raised so that freed blocks are reused by later calls.
aps_status dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
// Host-side fault injection for tests: fail the k-th next allocation (k >= 1), 0 = off.
void set_alloc_fault(int64_t k);
// Pinned host blocks for results copied to the host, recycled through a process-wide cache
// (page-locking fresh memory for every result costs far more than the copy itself). Sizes
// are rounded up to a power of two of at least 1 MiB; at most 8 GiB is kept cached.
aps_status halloc(void **p, size_t bytes);
void hfree(void *p, size_t bytes);

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    aps_status alloc(size_t count, cudaStream_t stream) {
        release();
        s = stream;
        n = count;
        return dalloc(reinterpret_cast<void **>(&p), (count ? count : 1) * sizeof(T), stream);
    }
    void release() {
        if (p) dfree(p, s);
        p = nullptr;
        n = 0;
    }
    T *detach() {
        T *q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

// ---------------------------------------------------------------- primitives
// Exclusive prefix sum of `n` values (int32 or int64 input) into int64 `out` (n + 1
// entries: out[n] = total). `out` may not alias `in`.
aps_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
aps_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
// keys/vals are sorted in place (scratch is allocated internally).
aps_status sort_pairs(uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t s);

inline int bits_for(uint64_t v) {  // bits needed to hold values in [0, v]
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

inline int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace aps
