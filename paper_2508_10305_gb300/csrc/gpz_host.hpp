// gpz_host.hpp -- host-side helpers shared by the single-array and batched
// entry points of libgpz: sizes, the absolute-bound constants, the launch
// counter and the optional per-stage event timer.
#pragma once

#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "gpz.h"
#include "gpz_internal.cuh"

namespace gpz {
namespace host {

inline uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

inline uint64_t nblocks_of(uint64_t n) { return (n + kBlock - 1) / kBlock; }

// The constants of one field from its bound eb: step eb * 63/32 (2 eb less
// 1/64), reciprocal, and the verification threshold RD32(eb * (1 - 2^-22)).
inline FieldParams finalise(double eb) {
    FieldParams p;
    p.eb = (float)eb;
    p.s = (float)(eb * 1.96875);
    p.inv = (float)(1.0 / (double)p.s);
    const double t = eb * (1.0 - std::ldexp(1.0, -22));
    float c = (float)t;
    if ((double)c > t) c = std::nextafterf(c, -INFINITY);
    p.ebchk = c;
    return p;
}

// ---------------------------------------------------------------- stage timing
//
// When enabled for a stream, each call on that stream records one event
// before its first kernel and one after each kernel, from a pool;
// gpz_stage_times resolves the logged pairs into per-stage totals and
// recycles the pool.  Calls on other streams record nothing.

constexpr int kEventPool = 8192;

struct StageTimer {
    std::mutex mu;
    bool enabled = false;
    cudaStream_t stream = nullptr;  // the one stream whose calls are timed
    bool created = false;
    cudaEvent_t ev[kEventPool] = {};
    int used = 0;
    struct Span {
        const char* name;
        int a, b;
    };
    Span spans[kEventPool];
    int nspans = 0;
};
extern StageTimer g_timer;
extern std::atomic<uint64_t> g_launches;

struct Recorder {
    bool on = false;
    cudaStream_t s;
    int last = -1;
    explicit Recorder(cudaStream_t stream) : s(stream) {}
    // Start of the call's first kernel (after its memsets); `marks` events
    // are reserved for the call's kernels.
    void begin(int marks = 8) {
        std::lock_guard<std::mutex> g(g_timer.mu);
        if (!g_timer.enabled || g_timer.stream != s) return;
        if (!g_timer.created) {
            for (auto& e : g_timer.ev) cudaEventCreate(&e);
            g_timer.created = true;
        }
        if (g_timer.used + marks + 1 >= kEventPool) return;  // pool full until the next read
        on = true;
        last = g_timer.used++;
        cudaEventRecord(g_timer.ev[last], s);
    }
    void mark(const char* name) {
        ++g_launches;
        if (!on) return;
        std::lock_guard<std::mutex> g(g_timer.mu);
        if (g_timer.used >= kEventPool) return;
        const int e = g_timer.used++;
        cudaEventRecord(g_timer.ev[e], s);
        g_timer.spans[g_timer.nspans++] = {name, last, e};
        last = e;
    }
};

inline gpz_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GPZ_OK : GPZ_ERR_CUDA; }

// Device allocations made by the library (workspaces of calls given none,
// batch plans, the serving arena) go through these, so that a test can make
// the next ones fail as an exhausted device would (gpz_test_fail_next_allocations).
extern std::atomic<int> g_fail_allocs;
inline bool injected_alloc_failure() {
    int k = g_fail_allocs.load();
    while (k > 0)
        if (g_fail_allocs.compare_exchange_weak(k, k - 1)) return true;
    return false;
}
// Workspaces of calls given none come from the library's own stream-ordered
// pool on the current device (gpz_api.cu), which keeps freed memory for the
// next call instead of returning it to the driver at every synchronisation.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s);
inline cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return pool_malloc_async(p, bytes, s);
}
inline cudaError_t dev_malloc(void** p, size_t bytes) {
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Where gpz_compress's workspace holds the range pass's outputs (byte
// offsets): control words (word 2 counts the finished range CTAs), the
// per-field constants, the CTAs' partial extremes and the block extremes.
struct RangeTargets {
    uint64_t ctrl, params, partials, bext;
};
RangeTargets compress_range_targets(uint64_t n, int F);
constexpr int kRangeCtasMax = 152 * 8;  // partials held for this many CTAs

// gpz_compress, optionally with the range pass already done (gpz_api.cu).
// With `interleaved` (16-byte aligned F-field records, d_fields[f] =
// interleaved + f) the tile kernel reads the records themselves; a relative
// bound then needs the range pass done.
gpz_status compress_impl(const float* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                         uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                         void* d_ws, uint64_t ws_size, void* stream, bool range_done,
                         const float* interleaved = nullptr);

// gpz_decompress; with `interleaved` the values go to F-field records there
// (d_fields[f] = interleaved + f, 4-byte aligned) (gpz_api.cu).
gpz_status decompress_impl(const void* d_in, uint64_t in_size, float* const* d_fields, int F, uint64_t n,
                           void* d_ws, uint64_t ws_size, void* stream, float* interleaved);

}  // namespace host

// The block decoder storing fp64 values (gpz_decode.cu): a.out[f] holds the
// address of a double array.
cudaError_t launch_decompress64(const DecArgs& a, cudaStream_t s);

namespace host {

// The 64-bit form (gpz_wide.cu): its workspace, and compression with
// absolute bounds eb[f] (the header records `mode`).
uint64_t wide_workspace_size(uint64_t n, int F);
gpz_status wide_compress(const double* const* d_fields, uint64_t n, int F, int G, int mode, const double* eb,
                         void* d_out, uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size,
                         uint32_t* d_perm, void* d_ws, uint64_t ws_size, cudaStream_t s);

}  // namespace host
}  // namespace gpz
