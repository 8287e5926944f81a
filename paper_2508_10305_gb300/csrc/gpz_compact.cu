// gpz_compact.cu -- steps 2 and 3 of GPZ's three-step compaction (Section
// 4.4, Table 1 "C."): a device-level prefix sum of the per-block word counts,
// then a copy of every block from its temporary slot to its final offset --
// except, with fused compaction, the blocks the fused kernel already wrote
// into the stream (kPlaced in their word count).
//
// The prefix sum is a single-pass decoupled look-back scan: CTAs take tiles
// in order from an atomic counter, publish their aggregate, then walk back
// over their predecessors' published aggregates / inclusive prefixes.  Every
// wait is bounded (about a second of SM clock); on expiry the status word
// records GPZ_ERR_TIMEOUT and the CTA continues as if the predecessor's
// prefix were zero, so no CTA waits forever.  Its output is written straight
// into the stream's block-offset table.
#include "gpz_internal.cuh"
#include "gpz_copy_block.cuh"

namespace gpz {

constexpr unsigned long long kFlagAggregate = 1ull << 32;
constexpr unsigned long long kFlagPrefix = 2ull << 32;

__device__ uint32_t lookback(const ScanArgs& a, uint32_t tile) {
    const long long limit = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;
    uint32_t excl = 0;
    int p = (int)tile - 1;
    while (p >= 0) {
        const long long t0 = clock64();
        unsigned long long st;
        for (;;) {
            st = ld_relaxed_u64(a.tile_state + p);
            if ((st >> 32) != 0ull) break;
            if (clock64() - t0 > limit) {
                set_status(a.status, kStTimeout);
                st = kFlagPrefix;  // give up: treat the predecessor's prefix as 0
                break;
            }
            __nanosleep(32);
        }
        excl += (uint32_t)st;
        if ((st >> 32) == 2ull) break;
        --p;
    }
    return excl;
}

__global__ void __launch_bounds__(kScanThreads) gpz_scan_kernel(ScanArgs a) {
    __shared__ uint32_t s_tile, s_excl;
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t start = (uint64_t)tile * kScanTile + (uint64_t)tid * kScanItems;

    // A block's words never exceed its raw size 1 + F*n_b; clamping keeps the
    // offsets (and the copy) inside the bound even if a size were corrupt.
    const uint32_t raw_full = 1u + (uint32_t)a.F * kBlock;
    const uint32_t raw_last = 1u + (uint32_t)a.F * (uint32_t)(a.n - (uint64_t)(a.nblocks ? a.nblocks - 1 : 0) * kBlock);
    uint32_t v[kScanItems];
    if (start + kScanItems <= a.nblocks) {
        const uint4* src = reinterpret_cast<const uint4*>(a.sizes + start);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            const uint4 q = __ldcg(src + k);
            v[4 * k] = q.x;
            v[4 * k + 1] = q.y;
            v[4 * k + 2] = q.z;
            v[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (start + k < a.nblocks) ? __ldcg(a.sizes + start + k) : 0u;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = min(v[k] & ~kPlaced, start + k + 1 == a.nblocks ? raw_last : raw_full);
        sum += v[k];
    }
    const uint32_t incl = warp_incl_sum(sum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t warp_base = 0, aggregate = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const uint32_t t = s_warp[w];
        if (w < warp) warp_base += t;
        aggregate += t;
    }
    if (tid == 0) {
        uint32_t excl = 0;
        if (tile == 0) {
            st_release_u64(a.tile_state, kFlagPrefix | aggregate);
        } else {
            st_release_u64(a.tile_state + tile, kFlagAggregate | aggregate);
            excl = lookback(a, tile);
            st_release_u64(a.tile_state + tile, kFlagPrefix | (uint32_t)(excl + aggregate));
        }
        s_excl = excl;
    }
    __syncthreads();
    // Exclusive prefixes; index nblocks (past the last block, whose item is
    // 0) receives the total, closing the table.
    uint32_t run = s_excl + warp_base + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (start + k <= a.nblocks) a.table[start + k] = run;
        run += v[k];
    }
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t s, unsigned grid) {
    const unsigned tiles = (unsigned)((a.nblocks + 1 + kScanTile - 1) / kScanTile);
    gpz_scan_kernel<<<grid ? grid : tiles, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ copy to final positions

__global__ void __launch_bounds__(32 * kCompactWarps) gpz_compact_kernel(CompactArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * kCompactWarps;
    if (blockIdx.x == 0 && warp == 0) {
        // Stream header and per-field constants.
        const uint32_t payload_words = __ldcg(a.table + a.nblocks);
        if (lane < kHeaderWords) {
            uint32_t v = 0;
            switch (lane) {
                case 0: v = kMagic; break;
                case 1: v = a.version; break;
                case 2: v = (uint32_t)a.F; break;
                case 3: v = (uint32_t)a.G; break;
                case 4: v = (uint32_t)kBlock; break;
                case 5: v = (uint32_t)a.mode; break;
                case 6: v = (uint32_t)(a.n & 0xffffffffull); break;
                case 7: v = (uint32_t)(a.n >> 32); break;
                case 8: v = a.nblocks; break;
                case 9: v = payload_words; break;
                default: v = 0; break;
            }
            a.stream[lane] = v;
        }
        if (a.ext_words) {
            if ((uint32_t)lane < a.ext_words) a.stream[kHeaderWords + lane] = a.ext[lane];
        } else if (lane < 2 * a.F) {
            const int f = lane >> 1;
            FieldParams p = a.params[0];
#pragma unroll
            for (int k = 1; k < kMaxFields; ++k)
                if (k == f) p = a.params[k];
            if (a.d_params) p = a.d_params[f];
            a.stream[kHeaderWords + lane] = __float_as_uint((lane & 1) ? p.s : p.eb);
        }
        if (lane == 0 && a.d_out_size)
            *a.d_out_size = 4ull * ((unsigned long long)a.payload_start + payload_words);
    }
    uint32_t* payload = a.stream + a.payload_start;
    // from the last block down: the fused kernel wrote the last blocks' slots
    // most recently, so the first reads here still find them in L2
    for (uint32_t bi = blockIdx.x * kCompactWarps + warp; bi < a.nblocks; bi += nwarps) {
        const uint32_t b = a.nblocks - 1u - bi;
        if (__ldcg(a.sizes + b) & kPlaced) continue;  // written into the stream by the fused kernel
        if (a.unplaced && lane == 0) atomicAdd(a.unplaced, 1u);
        const uint32_t len = __ldcg(a.table + b + 1) - __ldcg(a.table + b);  // clamped by the scan
        const uint32_t* src = a.temp + (size_t)b * a.slot_words;  // 16-byte aligned
        uint32_t* dst = payload + __ldcg(a.table + b);
        copy_block(src, dst, len, lane);
    }
}

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s) {
    unsigned grid = (a.nblocks + kCompactWarps - 1) / kCompactWarps;
    if (grid == 0) grid = 1;
    if (grid > 152u * 16u) grid = 152u * 16u;
    gpz_compact_kernel<<<grid, 32 * kCompactWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpz
