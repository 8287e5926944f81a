// gpz_batch_core.hpp -- host side of one batched compression or decompression:
// the chunk descriptors in plan order (grouped by field count), the flattened
// work lists, the workspace layout, and the enqueue of one run on a stream.
// Shared by the plan API (gpz_batch_api.cu) and the serving engine
// (gpz_serve.cu); it owns no device memory: the caller places the device
// copy of the descriptors and the workspace.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "gpz.h"
#include "gpz_batch.h"
#include "gpz_batch.cuh"

namespace gpz {
namespace host {

struct BatchGroup {
    int F;
    int pre;                            // relative-bound chunks: block extremes from the range items
    int bulk;                           // every chunk's fields 16-byte aligned: the tile kernel
    uint32_t first, count;              // plan positions of the group's chunks
    uint32_t range_first, range_items;  // the group's range items
    uint32_t block_first, blocks;       // the group's blocks
};

struct BatchLayout {  // byte offsets into the workspace
    uint64_t ctrl, status, rkeys, rdone, states, zero_bytes;
    uint64_t map, loc, rparams, bext, offsets, sizes, list, out_sizes, temp, total;
};

struct BatchDevice {  // the device copy of the descriptors
    BatchChunk* chunks;
    uint32_t* range_end;
};

struct BatchCore {
    int kind = 0;  // 0 compression, 1 decompression
    std::vector<BatchChunk> chunks;  // caller order until finish(), then plan order
    std::vector<BatchGroup> groups;
    std::vector<uint32_t> range_end;  // inclusive prefix of range items, plan order
    uint32_t total_blocks = 0;
    uint64_t temp_words = 0;
    bool any_rel = false;
    int sms = 0;
    gpz_batch_config cfg{};
    BatchLayout L{};
    uint32_t launches = 0;  // kernels per run

    uint32_t count() const { return (uint32_t)chunks.size(); }
};

// Append one chunk (its position in the caller's order is its index).
// Checks it as gpz_compress / gpz_decompress would.
gpz_status core_add_compress(BatchCore& c, const gpz_compress_chunk& d);
gpz_status core_add_decompress(BatchCore& c, const gpz_decompress_chunk& d);

// Group by field count, number the blocks and range items, lay out the
// workspace.  Queries the current device (SM count; cached) and sets the
// kernels' shared-memory attributes (once per device and field count).
gpz_status core_finish(BatchCore& c, const gpz_batch_config* cfg);

// Change the launch shape; re-lays the range items (the descriptors change:
// upload them again when this returns true in *redo).
gpz_status core_set_config(BatchCore& c, const gpz_batch_config& cfg, bool* redo);

// Bytes of the device copy of the descriptors, and their host image / device view.
uint64_t core_device_bytes(const BatchCore& c);
void core_pack(const BatchCore& c, uint8_t* host);
BatchDevice core_device_view(const BatchCore& c, uint8_t* device);

// Enqueue one run on s: clear the workspace's control words, then the kernels.
// timed: record per-kernel events when stage timing is on.
gpz_status core_enqueue(const BatchCore& c, const BatchDevice& dev, uint8_t* ws, uint64_t* d_out_sizes,
                        cudaStream_t s, bool timed);

}  // namespace host
}  // namespace gpz
