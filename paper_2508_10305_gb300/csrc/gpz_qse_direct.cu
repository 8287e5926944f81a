// gpz_qse_direct.cu -- the fused compression kernel with fused compaction
// (GPZ_FLAG_FUSED_COMPACTION): the same per-block code (gpz_qse_block.cuh)
// in its fused form, so that a block whose offset its predecessors'
// published sizes already fix is written straight into the stream by its
// own CTA, which waits for them (a decoupled look-back over blocks, the
// in-kernel form of Table 1).  The blocks not placed this way (raw blocks,
// blocks behind one left to the general path, or after a wait that ran out)
// are moved by the copy kernel of the three-step form, which skips the
// placed ones.
#include "gpz_qse_block.cuh"

namespace gpz {

template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 5) gpz_qse_direct_kernel(QseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseFastShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_fast<F, true, GridBlock, kCmDirect, PRE>(a, dsm, S, GridBlock{});
    else
        qse_block_fast<F, false, GridBlock, kCmDirect, PRE>(a, dsm, S, GridBlock{});
}

template <int F, bool PRE>
cudaError_t launch_qse_direct_fp(const QseArgs& a, cudaStream_t s) {
    const size_t smem = qse_fast_smem_bytes();
    auto kern = gpz_qse_direct_kernel<F, PRE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

cudaError_t launch_qse_direct(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    if (!a.direct || !a.bstate) return cudaErrorInvalidValue;
    const bool pre = a.bext != nullptr;
    switch (a.F) {
#define GPZ_CASE(FF) \
    case FF: return pre ? launch_qse_direct_fp<FF, true>(a, s) : launch_qse_direct_fp<FF, false>(a, s);
        GPZ_CASE(1)
        GPZ_CASE(2)
        GPZ_CASE(3)
        GPZ_CASE(4)
        GPZ_CASE(5)
        GPZ_CASE(6)
        GPZ_CASE(7)
        GPZ_CASE(8)
#undef GPZ_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz
