// gpz_batch.cuh -- device-side descriptors and argument blocks of the batched
// path: many independent arrays ("chunks") compressed or decompressed by a
// few launches, each chunk producing exactly the stream (or the values) a
// call of its own would produce.
//
// The chunks of one field count F form a group, served by the kernels compiled
// for that F.  Every block of every chunk has a global index (the chunks of
// all groups one after another); a map kernel writes, for every global block,
// the plan position of its chunk, so that a CTA finds its chunk with one load.
// Compression of a group: one launch of range items (relative-bound chunks:
// one slice of one field each; the last slice of a chunk to finish writes the
// chunk's constants), one launch with one CTA per block (the fused
// quantise/sort/encode of the single-array path), and the rare general-path
// blocks; then one 64-bit look-back scan over all blocks and one compaction
// pass for all chunks.  Decompression of a group: one launch with one CTA per
// block.
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

// chunks[] holds the groups one after another; a group is chunks
// [first, first + nchunks).
struct BatchCompressArgs {
    const BatchChunk* chunks;    // the plan's chunk array
    uint32_t first, nchunks;     // the group
    const uint32_t* range_end;   // [all chunks] inclusive prefix of range items (plan order)
    const uint32_t* block_map;   // [all blocks] plan position of each block's chunk
    uint32_t range_first;        // the group's first range item
    uint32_t range_items;        // the group's range items
    uint32_t block_first;        // the group's first block
    uint32_t total_blocks;       // the group's blocks
    uint32_t slice;              // values per range item
    uint32_t* rkeys;             // [chunks][kMaxFields][2]: ~order key of the min, order key of the max; zeroed
    uint32_t* rdone;             // [chunks] range items finished; zeroed
    FieldParams* rparams;        // [chunks][kMaxFields]
    uint2* bext;                 // [all blocks][kMaxFields]: each block's extremes from the range items
                                 // (a chunk's blocks from block_base * kMaxFields, b * F + f), or nullptr
    int pre;                     // the group's blocks read their extremes from bext (relative bounds)
    int tile;                    // every chunk's fields 16-byte aligned: the shared-memory tile kernel
    uint32_t* temp;
    uint32_t* sizes;             // [all blocks] words per block
    uint32_t* general_list;      // [the group's blocks] global block ids left to the general kernel
    uint32_t* general_count;     // the group's count, zeroed
    uint32_t* chunk_status;      // [chunks] zeroed
};

struct BatchMapArgs {
    const BatchChunk* chunks;
    uint32_t nchunks;
    uint32_t* block_map;         // [all blocks]
    uint4* block_loc;            // decompression: [all blocks] (payload words, table entries b and b + 1, 0)
                                 // read from the stream when its table lies inside it, else zeros; or nullptr
};

struct BatchScanArgs {
    const uint32_t* sizes;       // [total_blocks]
    uint32_t total_blocks;
    unsigned long long* offsets; // [total_blocks + 1] exclusive prefix (words)
    unsigned long long* tile_state; // zeroed
    uint32_t* tile_counter;      // zeroed
    uint32_t* status;
    long long wait_cycles;       // limit of a look-back wait in SM cycles; 0: kWaitCycles
};

struct BatchCompactArgs {
    const BatchChunk* chunks;
    uint32_t nchunks;
    const uint32_t* block_map;
    uint32_t total_blocks;
    const uint32_t* temp;
    const unsigned long long* offsets;
    const FieldParams* rparams;
    unsigned long long* out_sizes;  // [nchunks] stream bytes, in descriptor order (BatchChunk::index)
    uint32_t* chunk_status;
};

struct BatchDecompressArgs {
    const BatchChunk* chunks;    // the plan's chunk array
    const uint32_t* block_map;   // [all blocks]
    const uint4* block_loc;      // [all blocks] as BatchMapArgs
    uint32_t block_first;        // the group's first block
    uint32_t total_blocks;       // the group's blocks
    uint32_t* chunk_status;      // [chunks] zeroed
};

// Words of a block's temporary slot: the raw form 1 + F * 1024, rounded to 4.
__host__ __device__ constexpr uint32_t batch_slot_words(int F) {
    return (1u + (uint32_t)F * (uint32_t)kBlock + 3u) & ~3u;
}

// Smallest c in [0, n) with end[c] > item, for a non-decreasing end[] whose
// last entry exceeds item: a binary search, at most 32 probes.
__device__ __forceinline__ uint32_t search_chunk(const uint32_t* end, uint32_t n, uint32_t item) {
    uint32_t lo = 0, hi = n - 1;
    for (int k = 0; k < 32 && lo < hi; ++k) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(end + mid) > item)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Launch wrappers (gpz_batch_compress.cu, gpz_batch_decode.cu).
cudaError_t launch_batch_map(const BatchMapArgs& a, cudaStream_t s);
cudaError_t launch_batch_range(const BatchCompressArgs& a, cudaStream_t s);
cudaError_t launch_batch_compress(const BatchCompressArgs& a, int F, cudaStream_t s);
cudaError_t launch_batch_general(const BatchCompressArgs& a, int F, int grid, cudaStream_t s);
cudaError_t launch_batch_scan(const BatchScanArgs& a, cudaStream_t s, unsigned grid = 0);  // grid 0: one CTA per tile
cudaError_t launch_batch_compact(const BatchCompactArgs& a, int grid, cudaStream_t s);
cudaError_t launch_batch_decompress(const BatchDecompressArgs& a, int F, cudaStream_t s);
bool batch_prepare_kernels(int F);  // shared-memory attributes of the compression kernels; false on error

}  // namespace gpz
