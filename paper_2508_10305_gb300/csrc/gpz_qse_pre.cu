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
        qse_block_fast<F, true, GridBlock, kCmTemp, true>(a, dsm, S, GridBlock{});
    else
        qse_block_fast<F, false, GridBlock, kCmTemp, true>(a, dsm, S, GridBlock{});
}

// After the range pass, one thread per block: the widths and flags the fused
// kernel's step 2 would find (block_field_width, the same arithmetic), from
// the block's extremes and the field constants, packed as described at
// kInfoBig.  A block with a non-finite mark is stored raw before its widths
// are read, so those are left at 0.
template <int F>
__global__ void __launch_bounds__(256) gpz_block_info_kernel(const uint2* bext, const FieldParams* params,
                                                             uint32_t nblocks, unsigned long long* info) {
    const uint32_t b = blockIdx.x * 256u + threadIdx.x;
    if (b >= nblocks) return;
    unsigned long long v = 0ull;
    bool big = false, exact = true;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const uint2 e = __ldg(bext + (size_t)b * F + f);
        if (e.x == 0u) continue;  // non-finite
        uint32_t bits;
        bool bg, ex;
        block_field_width(e.x, e.y, params[f], bits, bg, ex);
        v |= (unsigned long long)(bits & 31u) << (5 * f);
        big |= bg;
        exact = exact && ex;
    }
    info[b] = v | ((unsigned long long)big << kInfoBig) | ((unsigned long long)exact << kInfoExact);
}

cudaError_t launch_block_info(const uint2* bext, const FieldParams* d_params, uint32_t nblocks, int F,
                              unsigned long long* binfo, cudaStream_t s) {
    if (nblocks == 0) return cudaSuccess;
    const unsigned grid = (nblocks + 255u) / 256u;
    switch (F) {
        case 1: gpz_block_info_kernel<1><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 2: gpz_block_info_kernel<2><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 3: gpz_block_info_kernel<3><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 4: gpz_block_info_kernel<4><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 5: gpz_block_info_kernel<5><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 6: gpz_block_info_kernel<6><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 7: gpz_block_info_kernel<7><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        case 8: gpz_block_info_kernel<8><<<grid, 256, 0, s>>>(bext, d_params, nblocks, binfo); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
