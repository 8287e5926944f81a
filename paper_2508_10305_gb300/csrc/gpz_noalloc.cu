// gpz_noalloc.cu -- gpz_compress_noalloc: compression that never allocates.
//
// Some callers cannot allocate device memory at the moment they want to
// compress: an in-situ analysis hook running inside a simulation whose device
// memory is entirely reserved by the simulation's own pool allocator, or a
// latency-critical loop in which an allocation (which may synchronise the
// device) is not acceptable.  For them this entry point takes its scratch
// space -- the per-block temporary output, the block sizes and the prefix-sum
// state of the compaction -- from a fixed array that is part of the library
// image.  Every GPU that loads the library reserves that array until the
// process exits.
#include <mutex>

#include "gpz.h"
#include "gpz_internal.cuh"

namespace {

// 32 MiB of scratch per device: enough for about 8 million fp32 values
// (n * n_fields), e.g. 2.6M particles of 3 fields or 1.3M of 6.
constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Address of this device's scratch array (looked up once per device, with the
// device current; host code must not use the symbol itself as an address).
gpz_status scratch_of_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GPZ_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GPZ_ERR_CUDA;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return GPZ_OK;
}

}  // namespace

extern "C" gpz_status gpz_compress_noalloc(const float* const* d_fields, uint64_t n, const gpz_params* p,
                                           void* d_out, uint64_t out_capacity, uint64_t* d_out_size,
                                           uint64_t* h_out_size, uint32_t* d_perm, void* stream) {
    if (!p || p->n_fields < 1 || p->n_fields > GPZ_MAX_FIELDS) return GPZ_ERR_INVALID_ARG;
    const uint64_t need = gpz_compress_workspace_size(n, p->n_fields);
    if (need == 0 || need > kNoAllocScratchBytes) return GPZ_ERR_CAPACITY;  // too many values for the array
    void* scratch = nullptr;
    const gpz_status st = scratch_of_current_device(&scratch);
    if (st != GPZ_OK) return st;
    // The ordinary entry point with a caller-provided workspace allocates nothing.
    return gpz_compress(d_fields, n, p, d_out, out_capacity, d_out_size, h_out_size, d_perm, scratch,
                        kNoAllocScratchBytes, stream);
}
