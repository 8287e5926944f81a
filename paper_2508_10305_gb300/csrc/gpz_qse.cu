// gpz_qse.cu -- the fused per-block compression kernel (stages 1-3 of GPZ:
// quantisation, sorting, encoding; Sections 4.1-4.3, the "Q.S.E." kernel of
// Table 1) and the global range pass of the relative error bound.
//
// One CTA of 256 threads owns one block of 1024 particles; every thread
// holds 4 particles of every field in registers (no shared-memory tile).
// Thread (warp w, lane l) owns elements 128w + 32r + l, r = 0..3, so that each
// warp covers 128 consecutive particles in storage order.  Per CTA:
//   1. coalesced streaming loads; per-field exact fp32 minimum (Section 4.1:
//      per-thread, then warp reduction, then a shared atomic per warp), or,
//      with a relative bound, the block's extremes the range pass already
//      found (gpz_qse_pre.cu);
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
//   5. fixed-length coding (Section 4.3) into staging words cleared at the
//      start: the deltas and counts by thread-serial bit appenders, each
//      record ORed in by its own thread at its sorted position; the encoded
//      block is copied out with 16-byte stores;
//   6. the block goes to its temporary slot with its word count (step 1 of
//      the three-step compaction, Section 4.4).
#include "gpz_qse_block.cuh"

namespace gpz {

// ------------------------------------------------------------------ range pass (relative bound)

// One warp per (block, field) item, field-major, so that consecutive warps
// stream consecutive blocks of a field.  Each item yields the block's
// extremes for the fused kernel (order keys; (0, 0) when the block holds a
// NaN or an infinity in that field) and feeds the CTA's running extremes of
// the field over its non-NaN values.
__global__ void __launch_bounds__(kRangeThreads, 8) gpz_range_kernel(RangeArgs a) {
    __shared__ float2 red[kRangeThreads / 32];
    __shared__ uint32_t s_lo[kMaxFields], s_hi[kMaxFields];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kMaxFields) {
        s_lo[tid] = 0xffffffffu;
        s_hi[tid] = 0u;
    }
    __syncthreads();
    const uint64_t nb = (a.n + kBlock - 1) / kBlock;
    const uint64_t items = nb * (uint64_t)a.F;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kRangeThreads / 32);
    for (uint64_t it = (uint64_t)blockIdx.x * (kRangeThreads / 32) + warp; it < items; it += nwarps) {
        const int f = (int)(it / nb);
        const uint64_t b = it - (uint64_t)f * nb;
        const float* x = a.fields[f] + b * kBlock;
        const int n_b = (int)min((uint64_t)kBlock, a.n - b * kBlock);
        float lo = INFINITY, hi = -INFINITY, probe = 0.0f;  // probe: NaN if any value is NaN or infinite
        if (a.vec_ok && n_b == kBlock) {  // 256 16-byte words: all eight of a lane in flight at once
            const float4* x4 = reinterpret_cast<const float4*>(x);
            float4 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldcs(x4 + lane + 32 * k);
            {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    lo = fminf(lo, fminf(fminf(v[k].x, v[k].y), fminf(v[k].z, v[k].w)));
                    hi = fmaxf(hi, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
                    probe = __fmaf_rn(v[k].x, 0.0f, probe);
                    probe = __fmaf_rn(v[k].y, 0.0f, probe);
                    probe = __fmaf_rn(v[k].z, 0.0f, probe);
                    probe = __fmaf_rn(v[k].w, 0.0f, probe);
                }
            }
        } else {
            for (int i = lane; i < n_b; i += 32) {
                const float v = __ldcs(x + i);
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
                probe = __fmaf_rn(v, 0.0f, probe);
            }
        }
        lo = warp_min_f32(lo);
        hi = warp_max_f32(hi);
        const bool nonfinite = __any_sync(0xffffffffu, probe != probe);
        if (lane == 0) {
            a.bext[b * (uint64_t)a.F + f] = nonfinite ? make_uint2(0u, 0u) : make_uint2(order_key(lo), order_key(hi));
            if (lo <= hi) {  // some value is not NaN
                atomicMin(&s_lo[f], order_key(lo));
                atomicMax(&s_hi[f], order_key(hi));
            }
        }
    }
    __syncthreads();
    if (tid < a.F) {
        const uint32_t kl = s_lo[tid], kh = s_hi[tid];
        const bool any = kl != 0xffffffffu || kh != 0u;
        a.partials[(size_t)blockIdx.x * a.F + tid] =
            any ? make_float2(from_order_key(kl), from_order_key(kh)) : make_float2(INFINITY, -INFINITY);
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
    if (a.bext) return launch_qse_pre(a, s);
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
