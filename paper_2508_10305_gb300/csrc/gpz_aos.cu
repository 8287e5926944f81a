// gpz_aos.cu -- interleaved (array-of-structures) input and output: particle
// i's fields at aos[i*F .. i*F+F-1], the layout of LAS-style point records.
// The stream is the one gpz_compress writes for the same values.
//   - Compression of 16-byte aligned records: the tile kernel's body takes a
//     block's 1024 F contiguous values as its tile (one bulk copy), and a
//     relative bound's range pass reads the records; no copy is made.
//     Records only 4-byte aligned (or with fused compaction) are first
//     transposed into structure-of-arrays form in the workspace, the range
//     pass folded into the transpose (one CTA per tile of 1024 particles,
//     staged through shared memory).
//   - Decompression: the block decoder stores each value at its place in the
//     records (field f of sorted position j at aos[j*F + f]).
#include "gpz.h"
#include "gpz_host.hpp"
#include "gpz_internal.cuh"
#include "gpz_qse_tile.cuh"
#include "gpz_decode_block.cuh"

using namespace gpz;
using namespace gpz::host;

namespace gpz {

constexpr int kAosTile = 1024;     // particles per tile
constexpr int kAosThreads = 256;

// soa[f * ld + i] = aos[i * F + f] for i < n
template <int F>
__global__ void __launch_bounds__(kAosThreads) gpz_aos_to_soa_kernel(const float* __restrict__ aos,
                                                                     float* __restrict__ soa, uint64_t n,
                                                                     uint64_t ld, bool vec) {
    __shared__ float tile[(kAosTile + 1) * F];
    const uint64_t ntiles = (n + kAosTile - 1) / kAosTile;
    for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const uint64_t first = tl * kAosTile;
        const int cnt = (int)min((uint64_t)kAosTile, n - first);
        const int words = cnt * F;
        const float* src = aos + first * (uint64_t)F;
        if (vec && cnt == kAosTile) {  // whole tile, 16-byte aligned on both sides: 16-byte loads and stores
            const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
            for (int k4 = threadIdx.x; k4 < kAosTile * F / 4; k4 += kAosThreads) {
                const float4 v = __ldcs(s4 + k4);
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = 4 * k4 + c, i = k / F, f = k - i * F;
                    tile[f * (kAosTile + 1) + i] = e[c];  // field-major in shared memory, padded rows
                }
            }
            __syncthreads();
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const float* row = tile + f * (kAosTile + 1);
                const int i = 4 * threadIdx.x;  // 256 threads x 4 = the tile
                __stcs(reinterpret_cast<float4*>(soa + (uint64_t)f * ld + first + i),
                       make_float4(row[i], row[i + 1], row[i + 2], row[i + 3]));
            }
        } else {
            for (int k = threadIdx.x; k < words; k += kAosThreads) {
                const int i = k / F, f = k - i * F;
                tile[f * (kAosTile + 1) + i] = __ldcs(src + k);
            }
            __syncthreads();
#pragma unroll
            for (int f = 0; f < F; ++f)
                for (int i = threadIdx.x; i < cnt; i += kAosThreads)
                    soa[(uint64_t)f * ld + first + i] = tile[f * (kAosTile + 1) + i];
        }
        __syncthreads();
    }
}

// The interleaved-to-fields transpose that also does the relative bound's
// range pass: while a tile (one 1,024-particle block) sits in shared memory,
// warp f reduces field f's row to the block's extremes (order keys, or
// (0, 0) when the row holds a NaN or an infinity) and the CTA's running
// extremes over the non-NaN values; the last CTA folds the CTAs' partials
// into the per-field constants.  The outputs are those of the range pass of
// gpz_compress, in the same places of its workspace, so compression then
// skips that pass and its read of the fields.  With soa == nullptr the
// kernel is the range pass alone (compression then reads the records).
template <int F>
__global__ void __launch_bounds__(kAosThreads) gpz_aos_range_kernel(const float* __restrict__ aos,
                                                                    float* __restrict__ soa, uint64_t n,
                                                                    uint64_t ld, bool vec, RangeArgs ra) {
    __shared__ float tile[(kAosTile + 1) * F];
    __shared__ uint32_t s_lo[kMaxFields], s_hi[kMaxFields];
    __shared__ float2 red[kAosThreads / 32];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kMaxFields) {
        s_lo[tid] = 0xffffffffu;
        s_hi[tid] = 0u;
    }
    const uint64_t ntiles = (n + kAosTile - 1) / kAosTile;
    for (uint64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const uint64_t first = tl * kAosTile;
        const int cnt = (int)min((uint64_t)kAosTile, n - first);
        const int words = cnt * F;
        const float* src = aos + first * (uint64_t)F;
        if (vec && cnt == kAosTile) {
            const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
            for (int k4 = tid; k4 < kAosTile * F / 4; k4 += kAosThreads) {
                const float4 v = __ldcs(s4 + k4);
                const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = 4 * k4 + c, i = k / F, f = k - i * F;
                    tile[f * (kAosTile + 1) + i] = e[c];
                }
            }
        } else {
            for (int k = tid; k < words; k += kAosThreads) {
                const int i = k / F, f = k - i * F;
                tile[f * (kAosTile + 1) + i] = __ldcs(src + k);
            }
        }
        __syncthreads();
        if (warp < F) {  // the block's extremes of field `warp`
            const float* row = tile + warp * (kAosTile + 1);
            float lo = INFINITY, hi = -INFINITY, probe = 0.0f;  // probe: NaN if a value is NaN or infinite
            for (int i = lane; i < cnt; i += 32) {
                const float v = row[i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
                probe = __fmaf_rn(v, 0.0f, probe);
            }
            lo = warp_min_f32(lo);
            hi = warp_max_f32(hi);
            const bool nonfinite = __any_sync(0xffffffffu, probe != probe);
            if (lane == 0) {
                ra.bext[tl * (uint64_t)F + warp] =
                    nonfinite ? make_uint2(0u, 0u) : make_uint2(order_key(lo), order_key(hi));
                if (lo <= hi) {  // some value is not NaN
                    atomicMin(&s_lo[warp], order_key(lo));
                    atomicMax(&s_hi[warp], order_key(hi));
                }
            }
        }
        if (!soa) {
            // the range pass alone
        } else if (vec && cnt == kAosTile) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const float* row = tile + f * (kAosTile + 1);
                const int i = 4 * tid;
                __stcs(reinterpret_cast<float4*>(soa + (uint64_t)f * ld + first + i),
                       make_float4(row[i], row[i + 1], row[i + 2], row[i + 3]));
            }
        } else {
#pragma unroll
            for (int f = 0; f < F; ++f)
                for (int i = tid; i < cnt; i += kAosThreads)
                    soa[(uint64_t)f * ld + first + i] = tile[f * (kAosTile + 1) + i];
        }
        __syncthreads();
    }
    if (tid < F) {
        const uint32_t kl = s_lo[tid], kh = s_hi[tid];
        const bool any = kl != 0xffffffffu || kh != 0u;
        ra.partials[(size_t)blockIdx.x * F + tid] =
            any ? make_float2(from_order_key(kl), from_order_key(kh)) : make_float2(INFINITY, -INFINITY);
    }
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(ra.done_counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int f = 0; f < F; ++f) {  // the last CTA folds every CTA's partial extremes of field f
        float lo = INFINITY, hi = -INFINITY;
        for (unsigned c = tid; c < gridDim.x; c += kAosThreads) {
            const float2 pp = __ldcg(ra.partials + (size_t)c * F + f);
            lo = fminf(lo, pp.x);
            hi = fmaxf(hi, pp.y);
        }
        lo = warp_min_f32(lo);
        hi = warp_max_f32(hi);
        if (lane == 0) red[warp] = make_float2(lo, hi);
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kAosThreads / 32; ++w) {
                lo = fminf(lo, red[w].x);
                hi = fmaxf(hi, red[w].y);
            }
            ra.d_params[f] = range_params(lo, hi, ra.rel[f]);
        }
        __syncthreads();
    }
}

// Compression straight from 16-byte aligned interleaved records: the tile
// kernel's body with the block's records as its tile (one bulk copy of
// 1024 F contiguous values), so no structure-of-arrays copy is made.
template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 6) gpz_qse_tile_aos_kernel(QseArgs a) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ __align__(8) TileShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_tile<F, true, PRE, GridBlock, true>(a, dsm, S, GridBlock{});
    else
        qse_block_tile<F, false, PRE, GridBlock, true>(a, dsm, S, GridBlock{});
}

template <int F, bool PRE>
cudaError_t launch_qse_tile_aos_fp(const QseArgs& a, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(F);
    auto kern = gpz_qse_tile_aos_kernel<F, PRE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

cudaError_t launch_qse_tile_aos(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    const bool pre = a.bext != nullptr;
    switch (a.F) {
#define GPZ_CASE(FF) \
    case FF: return pre ? launch_qse_tile_aos_fp<FF, true>(a, s) : launch_qse_tile_aos_fp<FF, false>(a, s);
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

// Decompression into interleaved records: the block decoder stages the
// block's values in record order in shared memory and writes the block's
// records with contiguous stores (4-byte aligned records; 16-byte stores
// when they are 16-byte aligned).
template <int F>
__global__ void __launch_bounds__(kDecThreads, 8) gpz_decompress_aos_kernel(DecArgs a) {
    __shared__ DecSharedRec<F> S;
    decode_block<F, DecGridBlock, false, true, DecSharedRec<F>>(a, S, DecGridBlock{});
}

cudaError_t launch_decompress_aos(const DecArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    switch (a.F) {
        case 1: gpz_decompress_aos_kernel<1><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 2: gpz_decompress_aos_kernel<2><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 3: gpz_decompress_aos_kernel<3><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 4: gpz_decompress_aos_kernel<4><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 5: gpz_decompress_aos_kernel<5><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 6: gpz_decompress_aos_kernel<6><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 7: gpz_decompress_aos_kernel<7><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        case 8: gpz_decompress_aos_kernel<8><<<a.nblocks, kDecThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int F>
cudaError_t launch_transpose_range_f(const float* src, float* dst, uint64_t n, uint64_t ld, unsigned grid,
                                     const RangeArgs& ra, cudaStream_t s) {
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 && ld % 4 == 0;
    gpz_aos_range_kernel<F><<<grid, kAosThreads, 0, s>>>(src, dst, n, ld, vec, ra);
    return cudaGetLastError();
}

cudaError_t launch_transpose_range(const float* src, float* dst, uint64_t n, int F, uint64_t ld, unsigned grid,
                                   const RangeArgs& ra, cudaStream_t s) {
    switch (F) {
        case 1: return launch_transpose_range_f<1>(src, dst, n, ld, grid, ra, s);
        case 2: return launch_transpose_range_f<2>(src, dst, n, ld, grid, ra, s);
        case 3: return launch_transpose_range_f<3>(src, dst, n, ld, grid, ra, s);
        case 4: return launch_transpose_range_f<4>(src, dst, n, ld, grid, ra, s);
        case 5: return launch_transpose_range_f<5>(src, dst, n, ld, grid, ra, s);
        case 6: return launch_transpose_range_f<6>(src, dst, n, ld, grid, ra, s);
        case 7: return launch_transpose_range_f<7>(src, dst, n, ld, grid, ra, s);
        case 8: return launch_transpose_range_f<8>(src, dst, n, ld, grid, ra, s);
    }
    return cudaErrorInvalidValue;
}

template <int F>
cudaError_t launch_transpose_f(const float* src, float* dst, uint64_t n, uint64_t ld, unsigned grid,
                               cudaStream_t s) {
    // 16-byte accesses when both bases are 16-byte aligned: a whole tile of the
    // interleaved array starts at a multiple of 1024 F floats, a field of the
    // other at a multiple of ld (a multiple of 4) plus a multiple of 1024
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0 && ld % 4 == 0;
    gpz_aos_to_soa_kernel<F><<<grid, kAosThreads, 0, s>>>(src, dst, n, ld, vec);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float* src, float* dst, uint64_t n, int F, uint64_t ld,
                             unsigned grid, cudaStream_t s) {
    switch (F) {
        case 1: return launch_transpose_f<1>(src, dst, n, ld, grid, s);
        case 2: return launch_transpose_f<2>(src, dst, n, ld, grid, s);
        case 3: return launch_transpose_f<3>(src, dst, n, ld, grid, s);
        case 4: return launch_transpose_f<4>(src, dst, n, ld, grid, s);
        case 5: return launch_transpose_f<5>(src, dst, n, ld, grid, s);
        case 6: return launch_transpose_f<6>(src, dst, n, ld, grid, s);
        case 7: return launch_transpose_f<7>(src, dst, n, ld, grid, s);
        case 8: return launch_transpose_f<8>(src, dst, n, ld, grid, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz

namespace {

constexpr uint64_t kAosAlign = 256;

// Leading dimension of the structure-of-arrays copy: every field 16-byte aligned.
uint64_t soa_ld(uint64_t n) { return align_up(n, 4); }

uint64_t soa_bytes(uint64_t n, int F) { return align_up(4ull * soa_ld(n) * (uint64_t)F, kAosAlign); }

unsigned transpose_grid(uint64_t n) {
    const uint64_t tiles = (n + kAosTile - 1) / kAosTile;
    const uint64_t cap = (uint64_t)kRangeCtasMax;  // eight CTAs per SM of a GB300
    return (unsigned)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}

}  // namespace

extern "C" {

uint64_t gpz_compress_aos_workspace_size(uint64_t n, int n_fields) {
    const uint64_t c = gpz_compress_workspace_size(n, n_fields);
    if (c == 0) return 0;
    return align_up(c, kAosAlign) + soa_bytes(n, n_fields);
}

uint64_t gpz_decompress_aos_workspace_size(uint64_t n, int n_fields) {
    (void)n;
    if (n_fields < 1 || n_fields > kMaxFields) return 0;
    return align_up(gpz_decompress_workspace_size(), kAosAlign);
}

gpz_status gpz_compress_aos(const float* d_aos, uint64_t n, const gpz_params* p, void* d_out,
                            uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                            void* d_ws, uint64_t ws_size, void* stream) {
    if (!p || p->n_fields < 1 || p->n_fields > kMaxFields) return GPZ_ERR_INVALID_ARG;
    const int F = p->n_fields;
    if (n > 0 && (!d_aos || (reinterpret_cast<uintptr_t>(d_aos) & 3u))) return GPZ_ERR_INVALID_ARG;
    const uint64_t need = gpz_compress_aos_workspace_size(n, F);
    cudaStream_t s = (cudaStream_t)stream;
    bool own = false;
    if (d_ws) {
        if (ws_size < need) return GPZ_ERR_CAPACITY;
        if (reinterpret_cast<uintptr_t>(d_ws) % kAosAlign) return GPZ_ERR_INVALID_ARG;
    } else {
        if (dev_malloc_async(&d_ws, need, s) != cudaSuccess) return GPZ_ERR_OOM;
        own = true;
    }
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    const uint64_t cws = align_up(gpz_compress_workspace_size(n, F), kAosAlign);
    float* soa = reinterpret_cast<float*>(ws + cws);
    const uint64_t ld = soa_ld(n);
    gpz_status rc = GPZ_OK;
    bool range_done = false;
    // 16-byte aligned records go straight to the tile kernel (no
    // structure-of-arrays copy); otherwise, or with fused compaction, they are
    // transposed first
    const bool direct = (reinterpret_cast<uintptr_t>(d_aos) & 15u) == 0 &&
                        (p->flags & GPZ_FLAG_FUSED_COMPACTION) == 0u;
    if (n > 0) {
        Recorder rec(s);
        rec.begin(1);
        if (p->mode == GPZ_EB_REL) {
            // the range pass over the records (with the transpose when there is
            // one), into the compression workspace
            const RangeTargets rt = compress_range_targets(n, F);
            RangeArgs ra{};
            ra.n = n;
            ra.F = F;
            for (int f = 0; f < F; ++f) ra.rel[f] = p->eb[f];
            ra.partials = reinterpret_cast<float2*>(ws + rt.partials);
            ra.done_counter = reinterpret_cast<uint32_t*>(ws + rt.ctrl) + 2;
            ra.d_params = reinterpret_cast<FieldParams*>(ws + rt.params);
            ra.bext = reinterpret_cast<uint2*>(ws + rt.bext);
            rc = cuda_status(cudaMemsetAsync(ws + rt.ctrl, 0, 64, s));
            const unsigned grid = transpose_grid(n);  // <= kRangeCtasMax CTAs: their partials fit
            if (rc == GPZ_OK)
                rc = cuda_status(launch_transpose_range(d_aos, direct ? nullptr : soa, n, F, ld, grid, ra, s));
            range_done = rc == GPZ_OK;
            if (rc == GPZ_OK) rec.mark(direct ? "aos_range" : "aos");
        } else if (!direct) {
            rc = cuda_status(launch_transpose(d_aos, soa, n, F, ld, transpose_grid(n), s));
            if (rc == GPZ_OK) rec.mark("aos");
        }
    }
    if (rc == GPZ_OK) {
        const float* fields[kMaxFields];
        for (int f = 0; f < F; ++f) fields[f] = direct ? d_aos + f : soa + (uint64_t)f * ld;
        // the compression workspace sits at the start, so gpz_sync_status(d_ws) reads its status
        rc = compress_impl(fields, n, p, d_out, out_capacity, d_out_size, h_out_size, d_perm, ws, cws, stream,
                           range_done, direct && n > 0 ? d_aos : nullptr);
    }
    if (own) {  // as gpz_compress without a workspace: synchronise and return the device-side status
        if (rc == GPZ_OK) {
            uint32_t st = 0;
            if (cudaMemcpyAsync(&st, d_ws, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = GPZ_ERR_CUDA;
            else if (st != 0)
                rc = (gpz_status)st;
        }
        cudaFreeAsync(d_ws, s);
        if (cudaStreamSynchronize(s) != cudaSuccess && rc == GPZ_OK) rc = GPZ_ERR_CUDA;
    }
    return rc;
}

gpz_status gpz_decompress_aos(const void* d_in, uint64_t in_size, float* d_aos, int n_fields, uint64_t n,
                              void* d_ws, uint64_t ws_size, void* stream) {
    if (n_fields < 1 || n_fields > kMaxFields) return GPZ_ERR_INVALID_ARG;
    const int F = n_fields;
    if (n > 0 && (!d_aos || (reinterpret_cast<uintptr_t>(d_aos) & 3u))) return GPZ_ERR_INVALID_ARG;
    if (d_ws) {
        if (ws_size < gpz_decompress_aos_workspace_size(n, F)) return GPZ_ERR_CAPACITY;
        if (reinterpret_cast<uintptr_t>(d_ws) % kAosAlign) return GPZ_ERR_INVALID_ARG;
    }
    // the values go straight to their records; without a workspace the call
    // allocates one, synchronises and returns the device-side status
    float* fields[kMaxFields];
    for (int f = 0; f < F; ++f) fields[f] = n ? d_aos + f : nullptr;
    return decompress_impl(d_in, in_size, fields, F, n, d_ws, d_ws ? ws_size : 0, stream, n ? d_aos : nullptr);
}

}  // extern "C"
