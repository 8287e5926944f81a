// gpz_qse_direct.cu -- the fused compression kernel with fused compaction:
// the same per-block code (gpz_qse_block.cuh) with DIRECT = true, so that a
// block whose offset its predecessors' published sizes already fix is
// written straight into the stream (see the fused-compaction notes in
// gpz_qse_block.cuh).  The three-step compaction of Section 4.4 remains the
// default; this form is selected with gpz_set_fused_compaction().
#include "gpz_qse_block.cuh"

namespace gpz {

template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 5) gpz_qse_direct_kernel(QseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseFastShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_fast<F, true, GridBlock, true, PRE>(a, dsm, S, GridBlock{});
    else
        qse_block_fast<F, false, GridBlock, true, PRE>(a, dsm, S, GridBlock{});
}

template <int F, bool PRE>
cudaError_t launch_qse_direct_fp(const QseArgs& a, cudaStream_t s) {
    const size_t smem = qse_fast_smem_bytes();
    cudaError_t e =
        cudaFuncSetAttribute(gpz_qse_direct_kernel<F, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gpz_qse_direct_kernel<F, PRE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    gpz_qse_direct_kernel<F, PRE><<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

template <int F>
cudaError_t launch_qse_direct_f(const QseArgs& a, cudaStream_t s) {
    return a.bext ? launch_qse_direct_fp<F, true>(a, s) : launch_qse_direct_fp<F, false>(a, s);
}

cudaError_t launch_qse_direct(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    if (!a.direct || !a.bstate || !a.deferred_count) return cudaErrorInvalidValue;
    switch (a.F) {
        case 1: return launch_qse_direct_f<1>(a, s);
        case 2: return launch_qse_direct_f<2>(a, s);
        case 3: return launch_qse_direct_f<3>(a, s);
        case 4: return launch_qse_direct_f<4>(a, s);
        case 5: return launch_qse_direct_f<5>(a, s);
        case 6: return launch_qse_direct_f<6>(a, s);
        case 7: return launch_qse_direct_f<7>(a, s);
        case 8: return launch_qse_direct_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz
