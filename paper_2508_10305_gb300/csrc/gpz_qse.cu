// gpz_qse.cu -- the fused per-block compression kernel (stages 1-3 of GPZ:
// quantisation, sorting, encoding; Sections 4.1-4.3, the "Q.S.E." kernel of
// Table 1) and the global range pass of the relative error bound.
//
// One CTA of 256 threads owns one block of 1024 particles; every thread
// holds 4 particles of every field in registers (no shared-memory tile).
// Thread (warp w, lane l) owns elements 128w + 32r + l, r = 0..3, so that each
// warp covers 128 consecutive particles in storage order.  Per CTA:
//   1. coalesced streaming loads; per-field exact fp32 minimum (Section 4.1:
//      per-thread, then warp reduction, then a shared atomic per warp);
//   2. quantisation q = floor(fma(x - min, 1/s, 1/2)) with the stream
//      format's fp32 verification (skipped for blocks where it provably
//      passes); blocks that need a fallback candidate, codes >= 2^23 or
//      records wider than 128 bits go to the general kernel; for codes below
//      2^23 the floor and the int<->float conversions are one add in
//      round-down mode against 2^23 (full-rate pipes);
//   3. segId / segOffset by shift and mask (Section 5.1), the linearised
//      segId (key) and the per-particle record of offsets and extra-field
//      codes;
//   4. stable counting sort by key (Section 4.2): each warp ranks its 128
//      elements in storage order with __match_any_sync into a per-warp
//      histogram; a CTA-wide scan over (bin, warp) gives every element its
//      sorted position.  The non-empty bins are the run-length code (unique
//      ids and counts, Section 4.3);
//   5. fixed-length coding (Section 4.3): the sorted records are scattered
//      to shared memory, and each thread packs its run of deltas, counts and
//      records into zeroed staging words with a thread-serial bit appender
//      (words shared with a neighbour are merged with atomicOr); the
//      encoded block is copied out with 16-byte stores;
//   6. the block goes to its temporary slot with its word count (step 1 of
//      the three-step compaction, Section 4.4).
#include "gpz_qse_block.cuh"

namespace gpz {

// ------------------------------------------------------------------ range pass (relative bound)

__global__ void __launch_bounds__(kRangeThreads) gpz_range_kernel(RangeArgs a) {
    __shared__ float2 red[kRangeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int f = 0; f < a.F; ++f) {
        const float* x = a.fields[f];
        float lo = INFINITY, hi = -INFINITY;
        if (a.vec_ok) {
            const float4* x4 = reinterpret_cast<const float4*>(x);
            const uint64_t n4 = a.n >> 2;
            const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
            uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid;
            for (; i + 3 * stride < n4; i += 4 * stride) {  // four 16-byte loads in flight per thread
                const float4 v0 = __ldcs(x4 + i), v1 = __ldcs(x4 + i + stride), v2 = __ldcs(x4 + i + 2 * stride),
                             v3 = __ldcs(x4 + i + 3 * stride);
                lo = fminf(lo, fminf(fminf(fminf(v0.x, v0.y), fminf(v0.z, v0.w)), fminf(fminf(v1.x, v1.y), fminf(v1.z, v1.w))));
                lo = fminf(lo, fminf(fminf(fminf(v2.x, v2.y), fminf(v2.z, v2.w)), fminf(fminf(v3.x, v3.y), fminf(v3.z, v3.w))));
                hi = fmaxf(hi, fmaxf(fmaxf(fmaxf(v0.x, v0.y), fmaxf(v0.z, v0.w)), fmaxf(fmaxf(v1.x, v1.y), fmaxf(v1.z, v1.w))));
                hi = fmaxf(hi, fmaxf(fmaxf(fmaxf(v2.x, v2.y), fmaxf(v2.z, v2.w)), fmaxf(fmaxf(v3.x, v3.y), fmaxf(v3.z, v3.w))));
            }
            for (; i < n4; i += stride) {
                const float4 v = __ldcs(x4 + i);
                lo = fminf(fminf(lo, v.x), fminf(v.y, fminf(v.z, v.w)));
                hi = fmaxf(fmaxf(hi, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
            }
            for (uint64_t i = (n4 << 2) + (uint64_t)blockIdx.x * blockDim.x + tid; i < a.n;
                 i += (uint64_t)gridDim.x * blockDim.x) {
                float v = x[i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        } else {
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
                float v = x[i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        }
        lo = warp_min_f32(lo);
        hi = warp_max_f32(hi);
        if (lane == 0) red[warp] = make_float2(lo, hi);
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kRangeThreads / 32; ++w) {
                lo = fminf(lo, red[w].x);
                hi = fmaxf(hi, red[w].y);
            }
            a.partials[(size_t)blockIdx.x * a.F + f] = make_float2(lo, hi);
        }
        __syncthreads();
    }
    // The last CTA to finish folds the partials and finalises the constants.
    __shared__ bool last;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(a.done_counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int f = 0; f < a.F; ++f) {  // all threads fold the CTAs' partials of field f
        float lo = INFINITY, hi = -INFINITY;
        for (unsigned c = tid; c < gridDim.x; c += blockDim.x) {
            const float2 p = __ldcg(a.partials + (size_t)c * a.F + f);
            lo = fminf(lo, p.x);
            hi = fmaxf(hi, p.y);
        }
        lo = warp_min_f32(lo);
        hi = warp_max_f32(hi);
        if (lane == 0) red[warp] = make_float2(lo, hi);
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kRangeThreads / 32; ++w) {
                lo = fminf(lo, red[w].x);
                hi = fmaxf(hi, red[w].y);
            }
            double rel = a.rel[0];
#pragma unroll
            for (int k = 1; k < kMaxFields; ++k)
                if (k == f) rel = a.rel[k];
            a.d_params[f] = range_params(lo, hi, rel);
        }
        __syncthreads();
    }
}

cudaError_t launch_range(const RangeArgs& a, int grid, cudaStream_t s) {
    gpz_range_kernel<<<grid, kRangeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Blocks the fast kernel leaves to the general path (rare): processed by a
// persistent grid walking the list.
template <int F>
__global__ void __launch_bounds__(kThreads, 2) gpz_qse_general_kernel(QseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseShared S;
    const uint32_t count = *(volatile const uint32_t*)a.general_count;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const uint32_t b = a.general_list[i];
        if ((uint64_t)(b + 1) * kBlock <= a.n)
            qse_block_general<F, true>(a, dsm, S, b);
        else
            qse_block_general<F, false>(a, dsm, S, b);
        __syncthreads();
    }
}

template <int F>
__global__ void __launch_bounds__(kThreads, 5) gpz_qse_kernel(QseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseFastShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_fast<F, true>(a, dsm, S, GridBlock{});
    else
        qse_block_fast<F, false>(a, dsm, S, GridBlock{});
}

template <int F>
cudaError_t launch_qse_f(const QseArgs& a, cudaStream_t s) {
    const size_t smem = qse_fast_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(gpz_qse_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gpz_qse_kernel<F>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    gpz_qse_kernel<F><<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

// the blocks left to the general path (usually none); the grid walks the list
template <int F>
cudaError_t launch_qse_general_f(const QseArgs& a, cudaStream_t s) {
    const size_t gsmem = qse_smem_bytes(F);
    cudaError_t e =
        cudaFuncSetAttribute(gpz_qse_general_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
    if (e != cudaSuccess) return e;
    const unsigned ggrid = a.nblocks < 2u * 152u ? a.nblocks : 2u * 152u;
    gpz_qse_general_kernel<F><<<ggrid, kThreads, gsmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_qse(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    switch (a.F) {
        case 1: return launch_qse_f<1>(a, s);
        case 2: return launch_qse_f<2>(a, s);
        case 3: return launch_qse_f<3>(a, s);
        case 4: return launch_qse_f<4>(a, s);
        case 5: return launch_qse_f<5>(a, s);
        case 6: return launch_qse_f<6>(a, s);
        case 7: return launch_qse_f<7>(a, s);
        case 8: return launch_qse_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_qse_general(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    switch (a.F) {
        case 1: return launch_qse_general_f<1>(a, s);
        case 2: return launch_qse_general_f<2>(a, s);
        case 3: return launch_qse_general_f<3>(a, s);
        case 4: return launch_qse_general_f<4>(a, s);
        case 5: return launch_qse_general_f<5>(a, s);
        case 6: return launch_qse_general_f<6>(a, s);
        case 7: return launch_qse_general_f<7>(a, s);
        case 8: return launch_qse_general_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz
