// gpz_copy.cu -- gpz_copy_stream: a copy whose byte count is read on the
// device (the size word gpz_compress writes), so that a pipeline can move a
// compressed stream to pinned host memory and back without the host waiting
// for the size first.  The copy is done by the SMs (pinned host memory is
// addressable from the device with unified addressing), with 16-byte loads
// and stores when both ends are 16-byte aligned.
#include "gpz.h"
#include "gpz_host.hpp"
#include "gpz_internal.cuh"

using namespace gpz;
using namespace gpz::host;

namespace {

constexpr int kCopyThreads = 256;
constexpr int kCopyCtas = 152 * 4;  // four CTAs per SM of a GB300

template <bool VEC>
__global__ void __launch_bounds__(kCopyThreads) gpz_copy_sized_kernel(void* dst, const void* src,
                                                                      const unsigned long long* d_size,
                                                                      unsigned long long capacity) {
    const unsigned long long want = __ldcg(d_size);
    const unsigned long long bytes = (want < capacity ? want : capacity) & ~3ull;  // streams are whole words
    const unsigned long long tid = (unsigned long long)blockIdx.x * kCopyThreads + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * kCopyThreads;
    unsigned long long done = 0;
    if (VEC) {
        const uint4* s4 = static_cast<const uint4*>(src);
        uint4* d4 = static_cast<uint4*>(dst);
        const unsigned long long n16 = bytes >> 4;
        unsigned long long i = tid;
        for (; i + 3 * nth < n16; i += 4 * nth) {  // four 16-byte words in flight per thread
            const uint4 a = __ldcs(s4 + i), b = __ldcs(s4 + i + nth), c = __ldcs(s4 + i + 2 * nth),
                        d = __ldcs(s4 + i + 3 * nth);
            d4[i] = a;
            d4[i + nth] = b;
            d4[i + 2 * nth] = c;
            d4[i + 3 * nth] = d;
        }
        for (; i < n16; i += nth) d4[i] = __ldcs(s4 + i);
        done = n16 << 4;
    }
    const uint32_t* s = static_cast<const uint32_t*>(src);
    uint32_t* d = static_cast<uint32_t*>(dst);
    for (unsigned long long w = (done >> 2) + tid; w < (bytes >> 2); w += nth) d[w] = __ldcs(s + w);
}

}  // namespace

extern "C" gpz_status gpz_copy_stream(void* dst, const void* src, const uint64_t* d_size, uint64_t capacity,
                                      void* stream) {
    if (!dst || !src || !d_size || !aligned(dst, 4) || !aligned(src, 4) || !aligned(d_size, 8))
        return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const auto* sz = reinterpret_cast<const unsigned long long*>(d_size);
    if (aligned(dst, 16) && aligned(src, 16))
        gpz_copy_sized_kernel<true><<<kCopyCtas, kCopyThreads, 0, s>>>(dst, src, sz, capacity);
    else
        gpz_copy_sized_kernel<false><<<kCopyCtas, kCopyThreads, 0, s>>>(dst, src, sz, capacity);
    ++g_launches;
    return cuda_status(cudaGetLastError());
}
