// gpz_noalloc.cu -- gpz_compress_noalloc: compression that never allocates.
//
// Some callers cannot allocate device memory at the moment they want to
// compress: an in-situ analysis hook running inside a simulation whose device
// memory is entirely reserved by the simulation's own pool allocator, or a
// latency-critical loop in which an allocation (which may synchronise the
// device) is not acceptable.  For them this entry point takes its scratch
// space -- the per-block temporary output, the block sizes and the prefix-sum
// state of the compaction -- from a fixed array that is part of the library
// image.  The array lives in this file's own module, which holds no kernel:
// under lazy module loading the module, and so the array's 32 MiB, is loaded
// on a device at the first symbol lookup with that device current
// (gpz_noalloc_prepare or the first call), and stays until the process exits.
#include "gpz.h"
#include "gpz_internal.cuh"

namespace {

// 32 MiB of scratch per device: enough for about 8 million fp32 values
// (n * n_fields), e.g. 2.6M particles of 3 fields or 1.3M of 6.
constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the current device's scratch array.  Host code must not
// use the symbol itself as an address.  The lookup is repeated on every call
// (a host-side table lookup once the module is loaded), so no address
// outlives a cudaDeviceReset.
gpz_status scratch_of_current_device(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GPZ_ERR_CUDA;
    *out = p;
    return GPZ_OK;
}

}  // namespace

extern "C" gpz_status gpz_noalloc_prepare(void) {
    void* scratch = nullptr;
    return scratch_of_current_device(&scratch);
}

extern "C" gpz_status gpz_noalloc_sync_status(void* stream) {
    void* scratch = nullptr;
    const gpz_status st = scratch_of_current_device(&scratch);
    if (st != GPZ_OK) return st;
    // the compression workspace's status word is its first word
    return gpz_sync_status(scratch, stream);
}

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
