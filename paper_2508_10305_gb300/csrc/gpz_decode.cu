// gpz_decode.cu -- GPZ decompression (Section 3.2, last paragraph: the
// reverse of compression without sorting; Table 1 "Decompression").
//
// One CTA of 256 threads per 1024-particle block; thread t rebuilds sorted
// positions 4t..4t+3.  Per CTA:
//   1. the block's table entries (one round trip), then its words after the
//      block header by one bulk copy into shared memory (an mbarrier with a
//      bounded wait), while warp 0 checks the stream header, the table
//      entries and the block header;
//   2. raw block: copy the stored values;
//   3. encoded block: every thread extracts two deltas and two counts
//      (fixed-length, one funnel shift each); a CTA-wide prefix sum gives
//      the unique segment ids and the run starts, which are marked in a
//      1024-bit mask;
//   4. the run of position j is the number of run starts <= j (popcount of
//      the mask prefix); its key is the run's id; the record at bit j*W
//      gives the segment offsets and extra-field codes; every value is
//      rebuilt as fma(q, step, min) and stored, four per thread.
// Every read stays inside the stream, every failed check sets
// GPZ_ERR_CORRUPT in the status word, and the kernel never traps.
#include "gpz_decode_block.cuh"

namespace gpz {

template <int F>
__global__ void __launch_bounds__(kDecThreads, 8) gpz_decompress_kernel(DecArgs a) {
    __shared__ DecShared S;
    decode_block<F>(a, S, DecGridBlock{});
}

template <int F>
cudaError_t launch_dec_f(const DecArgs& a, cudaStream_t s) {
    gpz_decompress_kernel<F><<<a.nblocks, kDecThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_decompress(const DecArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    if (a.interleaved) return launch_decompress_aos(a, s);  // gpz_aos.cu
    switch (a.F) {
        case 1: return launch_dec_f<1>(a, s);
        case 2: return launch_dec_f<2>(a, s);
        case 3: return launch_dec_f<3>(a, s);
        case 4: return launch_dec_f<4>(a, s);
        case 5: return launch_dec_f<5>(a, s);
        case 6: return launch_dec_f<6>(a, s);
        case 7: return launch_dec_f<7>(a, s);
        case 8: return launch_dec_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

// The same decoder storing fp64 (gpz_decompress_f64 on a version-1 stream):
// a.out[f] holds the address of field f's double array, and every value is
// the fp32 reconstruction widened exactly.
template <int F>
__global__ void __launch_bounds__(kDecThreads, 8) gpz_decompress64_kernel(DecArgs a) {
    __shared__ DecShared S;
    decode_block<F, DecGridBlock, true>(a, S, DecGridBlock{});
}

cudaError_t launch_decompress64(const DecArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    switch (a.F) {
        case 1: gpz_decompress64_kernel<1><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 2: gpz_decompress64_kernel<2><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 3: gpz_decompress64_kernel<3><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 4: gpz_decompress64_kernel<4><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 5: gpz_decompress64_kernel<5><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 6: gpz_decompress64_kernel<6><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 7: gpz_decompress64_kernel<7><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 8: gpz_decompress64_kernel<8><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gpz
