// gpz_qse_pre.cu -- the fused compression kernel for blocks whose extremes
// the range pass has already found (relative bound): the same per-block code
// (gpz_qse_block.cuh) with PRE = true, which reads each block's minimum and
// maximum (and its non-finite mark) instead of reducing them, and so skips
// one barrier and the per-value minimum, maximum and probe.
#include "gpz_qse_block.cuh"

namespace gpz {

template <int F>
__global__ void __launch_bounds__(kThreads, 5) gpz_qse_pre_kernel(QseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseFastShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_fast<F, true, GridBlock, false, true>(a, dsm, S, GridBlock{});
    else
        qse_block_fast<F, false, GridBlock, false, true>(a, dsm, S, GridBlock{});
}

template <int F>
cudaError_t launch_qse_pre_f(const QseArgs& a, cudaStream_t s) {
    const size_t smem = qse_fast_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gpz_qse_pre_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gpz_qse_pre_kernel<F>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    gpz_qse_pre_kernel<F><<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

cudaError_t launch_qse_pre(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    if (!a.bext) return cudaErrorInvalidValue;
    switch (a.F) {
        case 1: return launch_qse_pre_f<1>(a, s);
        case 2: return launch_qse_pre_f<2>(a, s);
        case 3: return launch_qse_pre_f<3>(a, s);
        case 4: return launch_qse_pre_f<4>(a, s);
        case 5: return launch_qse_pre_f<5>(a, s);
        case 6: return launch_qse_pre_f<6>(a, s);
        case 7: return launch_qse_pre_f<7>(a, s);
        case 8: return launch_qse_pre_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz
