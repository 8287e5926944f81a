// gpz_batch_compress.cu -- batched compression: for each group of chunks of
// one field count, one launch of range items (relative bounds), one launch
// with one CTA per block running the single-array fused quantise/sort/encode
// code (Sections 4.1-4.3), and the rare general-path blocks; then one 64-bit
// look-back scan over all blocks and one compaction pass that also writes
// every chunk's header and block table (Section 4.4, steps 2 and 3).  Each
// chunk's stream is the one a call of its own produces.
#include "gpz_batch.cuh"
#include "gpz_qse_block.cuh"
#include "gpz_qse_tile.cuh"
#include "gpz_copy_block.cuh"

namespace gpz {

namespace {

// Per-chunk argument block of the per-block code, built in shared memory by
// the CTA's threads in parallel (d_params stays null: the constants are
// copied in, read from L2).  Thread 64 also stores the block's index within
// its chunk in *slot.
__device__ __forceinline__ void load_chunk_args(const BatchCompressArgs& g, uint32_t c, uint32_t gb, QseArgs& A,
                                                uint32_t* slot) {
    const int t = threadIdx.x;
    const BatchChunk* ch = g.chunks + c;
    if (t < kMaxFields) A.fields[t] = ch->in[t];
    if (t >= 32 && t < 32 + 4 * kMaxFields) {
        const int f = (t - 32) >> 2, k = (t - 32) & 3;
        const uint32_t* src = ch->mode ? reinterpret_cast<const uint32_t*>(g.rparams + (size_t)c * kMaxFields + f)
                                       : reinterpret_cast<const uint32_t*>(ch->params + f);
        reinterpret_cast<uint32_t*>(A.params + f)[k] = __ldcg(src + k);
    }
    if (t == 64) {
        const uint32_t base = ch->block_base;
        slot[0] = gb - base;
        slot[1] = gb;
        A.n = ch->n;
        A.nblocks = ch->nblocks;
        A.F = ch->F;
        A.G = ch->G;
        A.bulk_ok = ch->bulk_ok;
        A.interleaved = 0;
        A.d_params = nullptr;
        A.bext = g.pre ? g.bext + (size_t)ch->block_base * kMaxFields : nullptr;
        A.binfo = nullptr;  // the fused kernel derives the widths from the extremes
        A.temp = g.temp + ch->temp_base;
        A.slot_words = batch_slot_words(ch->F);
        A.sizes = g.sizes + base;
        A.perm = ch->perm;
        A.status = g.chunk_status + c;
        A.general_list = g.general_list;
        A.general_count = g.general_count;
        A.direct = nullptr;  // the batched form keeps the three-step compaction
        A.direct_capacity = 0;
        A.bstate = nullptr;
        A.deferred_count = nullptr;
    }
}

// One range item: minimum and maximum of one slice of one field of a
// relative-bound chunk, merged into the chunk's order keys; the CTA that
// finishes the chunk's last item writes the chunk's constants.
__device__ __forceinline__ void range_item(const BatchCompressArgs& g, uint32_t c, uint32_t local, float2* red) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const BatchChunk* ch = g.chunks + c;
    const uint32_t slices = ch->range_slices;
    const uint32_t f = local / slices, sl = local - f * slices;
    const uint64_t n = ch->n;
    const uint64_t start = (uint64_t)sl * g.slice;  // a multiple of 1024: the slice holds whole blocks
    const uint64_t end = start + g.slice < n ? start + g.slice : n;
    const float* x = ch->in[f];
    const int F = ch->F;
    uint2* bext = g.bext + (size_t)ch->block_base * kMaxFields;
    // a warp per block: the block's extremes (order keys, or (0, 0) when it
    // holds a NaN or an infinity), and the warp's running extremes of the
    // slice over its non-NaN values
    float lo = INFINITY, hi = -INFINITY;
    const uint64_t b_first = start / kBlock, b_end = (end + kBlock - 1) / kBlock;
    for (uint64_t b = b_first + warp; b < b_end; b += kWarps) {
        const float* xb = x + b * kBlock;
        const int n_b = (int)min((uint64_t)kBlock, n - b * kBlock);
        float blo = INFINITY, bhi = -INFINITY, probe = 0.0f;
        if (ch->bulk_ok && n_b == kBlock) {  // two rounds of four 16-byte loads per lane
            const float4* x4 = reinterpret_cast<const float4*>(xb);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float4 v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = __ldcs(x4 + lane + 32 * (4 * h + k));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    blo = fminf(blo, fminf(fminf(v[k].x, v[k].y), fminf(v[k].z, v[k].w)));
                    bhi = fmaxf(bhi, fmaxf(fmaxf(v[k].x, v[k].y), fmaxf(v[k].z, v[k].w)));
                    probe = __fmaf_rn(v[k].x, 0.0f, probe);
                    probe = __fmaf_rn(v[k].y, 0.0f, probe);
                    probe = __fmaf_rn(v[k].z, 0.0f, probe);
                    probe = __fmaf_rn(v[k].w, 0.0f, probe);
                }
            }
        } else {
            for (int i = lane; i < n_b; i += 32) {
                const float v = __ldcs(xb + i);
                blo = fminf(blo, v);
                bhi = fmaxf(bhi, v);
                probe = __fmaf_rn(v, 0.0f, probe);
            }
        }
        blo = warp_min_f32(blo);
        bhi = warp_max_f32(bhi);
        const bool nonfinite = __any_sync(0xffffffffu, probe != probe);
        if (lane == 0 && bext)
            bext[b * (uint64_t)F + f] = nonfinite ? make_uint2(0u, 0u) : make_uint2(order_key(blo), order_key(bhi));
        lo = fminf(lo, blo);
        hi = fmaxf(hi, bhi);
    }
    lo = warp_min_f32(lo);
    hi = warp_max_f32(hi);
    if (lane == 0) red[warp] = make_float2(lo, hi);
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < kWarps; ++w) {
            lo = fminf(lo, red[w].x);
            hi = fmaxf(hi, red[w].y);
        }
        uint32_t* keys = g.rkeys + ((size_t)c * kMaxFields + f) * 2;
        if (lo <= hi) {  // NaNs are ignored, as fminf / fmaxf do
            atomicMax(keys, ~order_key(lo));
            atomicMax(keys + 1, order_key(hi));
        }
        __threadfence();
        const uint32_t items = (uint32_t)ch->F * slices;
        if (atomicAdd(g.rdone + c, 1u) == items - 1) {
            __threadfence();
            for (int ff = 0; ff < ch->F; ++ff) {
                const volatile uint32_t* k = g.rkeys + ((size_t)c * kMaxFields + ff) * 2;
                const uint32_t kmin = k[0], kmax = k[1];
                const float flo = kmax ? from_order_key(~kmin) : INFINITY;
                const float fhi = kmax ? from_order_key(kmax) : -INFINITY;
                g.rparams[(size_t)c * kMaxFields + ff] = range_params(flo, fhi, ch->rel[ff]);
            }
        }
    }
}

}  // namespace

// The chunk of every global block (one CTA per chunk).
__global__ void __launch_bounds__(256) gpz_batch_map_kernel(BatchMapArgs a) {
    const BatchChunk* ch = a.chunks + blockIdx.x;
    const uint32_t base = ch->block_base, nb = ch->nblocks;
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) a.block_map[base + j] = blockIdx.x;
    if (a.block_loc) {  // decompression: each block's place, gathered where it is coalesced
        const uint64_t table_start = kHeaderWords + 2ull * (uint64_t)ch->F;
        const bool fits = table_start + nb + 1 <= ch->words;  // the table lies inside the stream
        const uint32_t pw = fits ? __ldg(ch->src + 9) : 0u;
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
            a.block_loc[base + j] = fits ? make_uint4(pw, __ldg(ch->src + table_start + j),
                                                      __ldg(ch->src + table_start + j + 1), 0u)
                                         : make_uint4(0u, 0u, 0u, 0u);
    }
}

// One CTA per range item of the group.
__global__ void __launch_bounds__(kThreads) gpz_batch_range_kernel(BatchCompressArgs g) {
    __shared__ float2 red[kWarps];
    const uint32_t r = g.range_first + blockIdx.x;
    const uint32_t c = g.first + search_chunk(g.range_end + g.first, g.nchunks, r);
    range_item(g, c, r - g.chunks[c].range_base, red);
}

// One CTA per block of the group: the single-array fused kernel's code, with
// the chunk's arguments in shared memory.
template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 5) gpz_batch_compress_kernel(BatchCompressArgs g) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseFastShared S;
    __shared__ QseArgs A;
    __shared__ uint32_t slot[2];  // block within its chunk, global block id
    const uint32_t gb = g.block_first + blockIdx.x;
    load_chunk_args(g, __ldg(g.block_map + gb), gb, A, slot);
    __syncthreads();
    const SlotBlock idx{slot};
    if ((uint64_t)(idx.b() + 1) * kBlock <= A.n)
        qse_block_fast<F, true, SlotBlock, kCmTemp, PRE>(A, dsm, S, idx);
    else
        qse_block_fast<F, false, SlotBlock, kCmTemp, PRE>(A, dsm, S, idx);
}

// The same with the shared-memory tile body (gpz_qse_tile.cuh): groups whose
// chunks all have 16-byte aligned fields.
template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 6) gpz_batch_tile_kernel(BatchCompressArgs g) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ __align__(8) TileShared S;
    __shared__ QseArgs A;
    __shared__ uint32_t slot[2];  // block within its chunk, global block id
    const uint32_t gb = g.block_first + blockIdx.x;
    load_chunk_args(g, __ldg(g.block_map + gb), gb, A, slot);
    __syncthreads();
    const SlotBlock idx{slot};
    if ((uint64_t)(idx.b() + 1) * kBlock <= A.n)
        qse_block_tile<F, true, PRE>(A, dsm, S, idx);
    else
        qse_block_tile<F, false, PRE>(A, dsm, S, idx);
}

// Blocks the fast path left to the general one (rare); the grid walks the
// group's list.
template <int F>
__global__ void __launch_bounds__(kThreads, 2) gpz_batch_general_kernel(BatchCompressArgs g) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ QseShared S;
    __shared__ QseArgs A;
    __shared__ uint32_t slot[2];
    const uint32_t count = *(volatile const uint32_t*)g.general_count;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
        const uint32_t gb = __ldcg(g.general_list + i);
        load_chunk_args(g, __ldg(g.block_map + gb), gb, A, slot);
        __syncthreads();
        const uint32_t b = slot[0];
        if ((uint64_t)(b + 1) * kBlock <= A.n)
            qse_block_general<F, true>(A, dsm, S, b);
        else
            qse_block_general<F, false>(A, dsm, S, b);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ 64-bit look-back scan over all blocks

namespace {

constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr unsigned long long kAggregate = 1ull << 62;
constexpr unsigned long long kPrefix = 2ull << 62;
constexpr uint32_t kMaxBlockWords = 1u + (uint32_t)kMaxFields * (uint32_t)kBlock;

__device__ unsigned long long lookback64(const BatchScanArgs& a, uint32_t tile) {
    const long long limit = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;
    unsigned long long excl = 0;
    int p = (int)tile - 1;
    while (p >= 0) {
        const long long t0 = clock64();
        unsigned long long st;
        for (;;) {
            st = ld_relaxed_u64(a.tile_state + p);
            if ((st >> 62) != 0ull) break;
            if (clock64() - t0 > limit) {
                set_status(a.status, kStTimeout);
                st = kPrefix;  // give up: treat the predecessor's prefix as 0
                break;
            }
            __nanosleep(32);
        }
        excl += st & kValMask;
        if ((st >> 62) == 2ull) break;
        --p;
    }
    return excl;
}

}  // namespace

__global__ void __launch_bounds__(kScanThreads) gpz_batch_scan_kernel(BatchScanArgs a) {
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t start = (uint64_t)tile * kScanTile + (uint64_t)tid * kScanItems;
    uint32_t v[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        v[k] = (start + k < a.total_blocks) ? min(__ldcg(a.sizes + start + k), kMaxBlockWords) : 0u;
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += v[k];
    const uint32_t incl = warp_incl_sum(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t warp_base = 0, aggregate = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const uint32_t x = s_warp[w];
        if (w < warp) warp_base += x;
        aggregate += x;
    }
    if (tid == 0) {
        unsigned long long excl = 0;
        if (tile == 0) {
            st_release_u64(a.tile_state, kPrefix | aggregate);
        } else {
            st_release_u64(a.tile_state + tile, kAggregate | aggregate);
            excl = lookback64(a, tile);
            st_release_u64(a.tile_state + tile, kPrefix | (excl + aggregate));
        }
        s_excl = excl;
    }
    __syncthreads();
    unsigned long long run = s_excl + warp_base + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (start + k <= a.total_blocks) a.offsets[start + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------------ compaction, tables and headers

__global__ void __launch_bounds__(32 * kCompactWarps) gpz_batch_compact_kernel(BatchCompactArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kCompactWarps;
    const uint32_t items = a.total_blocks + a.nchunks;
    for (uint32_t qi = blockIdx.x * kCompactWarps + warp; qi < items; qi += nwarps) {
        // the blocks from the last one down (the last slots written are the
        // likeliest still in L2), then the chunks' headers
        const uint32_t q = qi < a.total_blocks ? a.total_blocks - 1u - qi : qi;
        if (q < a.total_blocks) {
            const uint32_t cur = __ldg(a.block_map + q);
            const BatchChunk* ch = a.chunks + cur;
            const uint32_t F = (uint32_t)ch->F, nb = ch->nblocks, b = q - ch->block_base;
            const uint64_t n = ch->n;
            const unsigned long long base = __ldcg(a.offsets + ch->block_base);
            const unsigned long long o0 = __ldcg(a.offsets + q), o1 = __ldcg(a.offsets + q + 1);
            const uint64_t first = (uint64_t)b * kBlock;
            const uint32_t n_b = (uint32_t)(n - first < (uint64_t)kBlock ? n - first : (uint64_t)kBlock);
            const uint64_t table_start = kHeaderWords + 2ull * F;
            const uint64_t payload_start = table_start + nb + 1;
            const unsigned long long rel = o0 - base, len = o1 - o0;
            uint32_t* dst = ch->dst;
            if (len > 1ull + F * n_b || payload_start + rel + len > ch->words) {
                if (lane == 0) set_status(a.chunk_status + cur, kStCapacity);
                continue;
            }
            if (lane == 0) dst[table_start + b] = (uint32_t)rel;
            const uint32_t* src = a.temp + ch->temp_base + (uint64_t)b * batch_slot_words((int)F);
            uint32_t* out = dst + payload_start + rel;
            copy_block(src, out, (uint32_t)len, lane);  // src 16-byte aligned: slots of whole 16-byte words
        } else {
            // the chunk's stream header, constants, closing table entry and size
            const uint32_t c = q - a.total_blocks;
            const BatchChunk* ch = a.chunks + c;
            const uint32_t F = (uint32_t)ch->F, nb = ch->nblocks;
            const unsigned long long payload = __ldcg(a.offsets + ch->block_base + nb) - __ldcg(a.offsets + ch->block_base);
            const uint64_t table_start = kHeaderWords + 2ull * F;
            const uint64_t payload_start = table_start + nb + 1;
            uint32_t* dst = ch->dst;
            if (payload_start + payload > ch->words) {
                if (lane == 0) {
                    set_status(a.chunk_status + c, kStCapacity);
                    a.out_sizes[ch->index] = 0ull;
                }
                continue;
            }
            if (lane < kHeaderWords) {
                uint32_t v = 0;
                switch (lane) {
                    case 0: v = kMagic; break;
                    case 1: v = kVersion; break;
                    case 2: v = F; break;
                    case 3: v = (uint32_t)ch->G; break;
                    case 4: v = (uint32_t)kBlock; break;
                    case 5: v = (uint32_t)ch->mode; break;
                    case 6: v = (uint32_t)(ch->n & 0xffffffffull); break;
                    case 7: v = (uint32_t)(ch->n >> 32); break;
                    case 8: v = nb; break;
                    case 9: v = (uint32_t)payload; break;
                    default: v = 0; break;
                }
                dst[lane] = v;
            }
            if ((uint32_t)lane < 2 * F) {
                const int f = lane >> 1;
                const FieldParams* p = ch->mode ? a.rparams + (size_t)c * kMaxFields + f : ch->params + f;
                const uint32_t* pw = reinterpret_cast<const uint32_t*>(p);
                dst[kHeaderWords + lane] = __ldcg((lane & 1) ? pw + 1 : pw);  // eb, then the step
            }
            if (lane == 0) {
                dst[table_start + nb] = (uint32_t)payload;
                a.out_sizes[ch->index] = 4ull * (payload_start + payload);
            }
        }
    }
}

// ------------------------------------------------------------------ launches

template <int F>
bool prepare_f() {
    return cudaFuncSetAttribute(gpz_batch_compress_kernel<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)qse_fast_smem_bytes()) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_compress_kernel<F, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                100) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_compress_kernel<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)qse_fast_smem_bytes()) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_compress_kernel<F, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                100) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_tile_kernel<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem_bytes(F)) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_tile_kernel<F, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                100) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_tile_kernel<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tile_smem_bytes(F)) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_tile_kernel<F, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                100) == cudaSuccess &&
           cudaFuncSetAttribute(gpz_batch_general_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)qse_smem_bytes(F)) == cudaSuccess;
}

bool batch_prepare_kernels(int F) {
    switch (F) {
        case 1: return prepare_f<1>();
        case 2: return prepare_f<2>();
        case 3: return prepare_f<3>();
        case 4: return prepare_f<4>();
        case 5: return prepare_f<5>();
        case 6: return prepare_f<6>();
        case 7: return prepare_f<7>();
        case 8: return prepare_f<8>();
    }
    return false;
}

template <int F>
void launch_f(const BatchCompressArgs& a, int grid, cudaStream_t s, bool general) {
    if (general)
        gpz_batch_general_kernel<F><<<grid, kThreads, qse_smem_bytes(F), s>>>(a);
    else if (a.tile && a.pre)
        gpz_batch_tile_kernel<F, true><<<grid, kThreads, tile_smem_bytes(F), s>>>(a);
    else if (a.tile)
        gpz_batch_tile_kernel<F, false><<<grid, kThreads, tile_smem_bytes(F), s>>>(a);
    else if (a.pre)
        gpz_batch_compress_kernel<F, true><<<grid, kThreads, qse_fast_smem_bytes(), s>>>(a);
    else
        gpz_batch_compress_kernel<F, false><<<grid, kThreads, qse_fast_smem_bytes(), s>>>(a);
}

cudaError_t launch_group(const BatchCompressArgs& a, int F, int grid, cudaStream_t s, bool general) {
    switch (F) {
        case 1: launch_f<1>(a, grid, s, general); break;
        case 2: launch_f<2>(a, grid, s, general); break;
        case 3: launch_f<3>(a, grid, s, general); break;
        case 4: launch_f<4>(a, grid, s, general); break;
        case 5: launch_f<5>(a, grid, s, general); break;
        case 6: launch_f<6>(a, grid, s, general); break;
        case 7: launch_f<7>(a, grid, s, general); break;
        case 8: launch_f<8>(a, grid, s, general); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_map(const BatchMapArgs& a, cudaStream_t s) {
    gpz_batch_map_kernel<<<a.nchunks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_range(const BatchCompressArgs& a, cudaStream_t s) {
    gpz_batch_range_kernel<<<a.range_items, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_compress(const BatchCompressArgs& a, int F, cudaStream_t s) {
    return launch_group(a, F, (int)a.total_blocks, s, false);
}

cudaError_t launch_batch_general(const BatchCompressArgs& a, int F, int grid, cudaStream_t s) {
    return launch_group(a, F, grid, s, true);
}

cudaError_t launch_batch_scan(const BatchScanArgs& a, cudaStream_t s, unsigned grid) {
    const unsigned tiles = (unsigned)(((uint64_t)a.total_blocks + 1 + kScanTile - 1) / kScanTile);
    gpz_batch_scan_kernel<<<grid ? grid : tiles, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_compact(const BatchCompactArgs& a, int grid, cudaStream_t s) {
    gpz_batch_compact_kernel<<<grid, 32 * kCompactWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpz
