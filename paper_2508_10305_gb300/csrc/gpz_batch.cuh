// gpz_batch.cuh -- device-side descriptors and argument blocks of the batched
// path: many independent arrays ("chunks") compressed or decompressed by a
// few persistent launches, each chunk producing exactly the stream (or the
// values) a call of its own would produce.
//
// The chunks of one field count F form a group, served by one persistent
// launch of the kernel compiled for that F.  Its work is claimed from the
// group's atomic ticket counters over a flattened item list, ordered by
// chunk: in compression the range-pass slices of the group's relative-bound
// chunks come first (claimed one at a time from their own counter), then
// every block of every chunk; in decompression every block of every chunk.
// A CTA claims `claim` consecutive blocks per ticket and finds each item's
// chunk by a forward search from the chunk of its previous item (tickets only
// grow).  A block of a relative-bound chunk waits for that chunk's constants;
// those come from range items claimed before any block (by CTAs that are
// already running and never wait themselves), so the wait always ends (it is
// bounded anyway).
#pragma once

#include "gpz_internal.cuh"

namespace gpz {

struct BatchChunk {
    const float* in[kMaxFields];     // compression: input fields
    float* out[kMaxFields];          // decompression: output fields
    const uint32_t* src;             // decompression: the stream
    uint32_t* dst;                   // compression: the stream buffer
    uint64_t words;                  // compression: capacity; decompression: stream length (words)
    uint64_t n;                      // particles
    uint64_t temp_base;              // compression: first temporary word of the chunk
    uint32_t* perm;                  // compression: [n] or nullptr
    FieldParams params[kMaxFields];  // absolute bound: the constants
    double rel[kMaxFields];          // relative bound: the factors
    uint32_t block_base;             // global index of the chunk's first block
    uint32_t nblocks;
    uint32_t range_base;             // first range item of the chunk (relative bound)
    uint32_t range_slices;           // range items per field (relative bound), else 0
    uint32_t index;                  // position in the caller's descriptor array
    int F, G, mode;
    int bulk_ok;                     // every field pointer 16-byte aligned
};

// One launch covers the chunks of one field count F (a "group"): chunk
// indices c below are positions in the plan's chunk array, which holds the
// groups one after another; the group is chunks [first, first + nchunks).
struct BatchCompressArgs {
    const BatchChunk* chunks;    // the plan's chunk array
    uint32_t first, nchunks;     // the group
    const uint32_t* range_end;   // [all chunks] inclusive prefix of range items (plan order)
    const uint32_t* block_end;   // [all chunks] inclusive prefix of blocks (plan order)
    uint32_t range_first;        // the group's first range item
    uint32_t range_items;        // the group's range items
    uint32_t block_first;        // the group's first block
    uint32_t total_blocks;       // the group's blocks
    uint32_t slice;              // elements per range item
    uint32_t claim;              // items per ticket
    uint32_t* ticket;            // the group's block counter (ticket[24]: its range-item counter), zeroed
    uint32_t* rkeys;             // [chunks][kMaxFields][2]: ~order key of the min, order key of the max; zeroed
    uint32_t* rdone;             // [chunks] range items finished; zeroed
    uint32_t* ready;             // [chunks] 1 once the chunk's relative constants are written; zeroed
    FieldParams* rparams;        // [chunks][kMaxFields]
    uint32_t* temp;
    uint32_t* sizes;             // [all blocks] words per block
    uint32_t* general_list;      // [the group's blocks] global block ids left to the general kernel
    uint32_t* general_count;     // the group's count, zeroed
    uint32_t* chunk_status;      // [chunks] zeroed
};

struct BatchScanArgs {
    const uint32_t* sizes;       // [total_blocks]
    uint32_t total_blocks;
    unsigned long long* offsets; // [total_blocks + 1] exclusive prefix (words)
    unsigned long long* tile_state; // zeroed
    uint32_t* tile_counter;      // zeroed
    uint32_t* status;
};

struct BatchCompactArgs {
    const BatchChunk* chunks;
    uint32_t nchunks;
    const uint32_t* block_end;
    uint32_t total_blocks;
    const uint32_t* temp;
    const unsigned long long* offsets;
    const FieldParams* rparams;
    const uint32_t* ready;
    unsigned long long* out_sizes;  // [nchunks] stream bytes, in descriptor order (BatchChunk::index)
    uint32_t* chunk_status;
};

struct BatchDecompressArgs {
    const BatchChunk* chunks;    // the plan's chunk array
    uint32_t first, nchunks;     // the group (one field count)
    const uint32_t* block_end;   // [all chunks] inclusive prefix of blocks
    uint32_t block_first;        // the group's first block
    uint32_t total_blocks;       // the group's blocks
    uint32_t claim;
    uint32_t* ticket;            // the group's block counter (ticket[24]: its range-item counter), zeroed
    uint32_t* chunk_status;      // [chunks] zeroed
};

// Words of a block's temporary slot: the raw form 1 + F * 1024, rounded to 4.
__host__ __device__ constexpr uint32_t batch_slot_words(int F) {
    return (1u + (uint32_t)F * (uint32_t)kBlock + 3u) & ~3u;
}

// Smallest c >= lo with end[c] > item, for a non-decreasing end[0..nchunks)
// whose last entry exceeds item (so the answer exists).  Galloping from lo, then a
// binary search; at most 2 * 32 probes.
__device__ __forceinline__ uint32_t find_chunk(const uint32_t* end, uint32_t nchunks, uint32_t item, uint32_t lo) {
    if (__ldg(end + lo) > item) return lo;
    uint32_t below = lo, step = 1, above = nchunks - 1;  // end[below] <= item < end[above]
    for (int k = 0; k < 32; ++k) {
        const uint32_t probe = below + step;
        if (probe >= nchunks - 1) break;
        if (__ldg(end + probe) > item) {
            above = probe;
            break;
        }
        below = probe;
        step <<= 1;
    }
    for (int k = 0; k < 32 && above - below > 1; ++k) {
        const uint32_t mid = below + ((above - below) >> 1);
        if (__ldg(end + mid) > item)
            above = mid;
        else
            below = mid;
    }
    return above;
}

// Launch wrappers (gpz_batch_compress.cu, gpz_batch_decode.cu).
cudaError_t launch_batch_compress(const BatchCompressArgs& a, int F, int grid, cudaStream_t s);
cudaError_t launch_batch_general(const BatchCompressArgs& a, int F, int grid, cudaStream_t s);
cudaError_t launch_batch_scan(const BatchScanArgs& a, cudaStream_t s);
cudaError_t launch_batch_compact(const BatchCompactArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_decompress(const BatchDecompressArgs& a, int F, int grid, cudaStream_t s);
int batch_compress_max_ctas_per_sm(int F);   // 0 on error
int batch_decompress_max_ctas_per_sm(int F);

}  // namespace gpz
