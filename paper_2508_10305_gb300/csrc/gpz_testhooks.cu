// gpz_testhooks.cu -- the failure-injection hooks of include/gpz_test.h: an
// allocation-failure counter read by every device allocation of the library,
// and launches of the look-back kernels with a predecessor that never
// publishes and a short wait limit, so that tests see the bounded waits run
// out (and the GPU keep answering) without any fault.
#include <atomic>

#include "gpz.h"
#include "gpz_batch.cuh"
#include "gpz_host.hpp"
#include "gpz_qse_block.cuh"
#include "gpz_test.h"

namespace gpz {
namespace host {
std::atomic<int> g_fail_allocs{0};
}  // namespace host
}  // namespace gpz

using namespace gpz;
using namespace gpz::host;

namespace {

constexpr uint32_t kTestBlocks = 2u * (uint32_t)kScanTile + 1u;  // nblocks + 1 items: three tiles
constexpr uint32_t kTestTiles = 3u;
constexpr uint64_t kA = 256;

// Workspace of the scan test: control words (status, tile counter), the tile
// states, the block sizes and the offsets (64-bit, enough for either scan).
struct ScanTestLayout {
    uint64_t ctrl = 0, states = 256, sizes, offsets, total;
    ScanTestLayout() {
        sizes = states + align_up(kTestTiles * 8ull, kA);
        offsets = sizes + align_up(kTestBlocks * 4ull, kA);
        total = offsets + align_up((kTestBlocks + 1ull) * 8ull, kA);
    }
};

__global__ void gpz_test_lookback_kernel(const unsigned long long* bstate, uint32_t b, long long limit,
                                         uint32_t* result) {
    const uint32_t off = block_lookback(bstate, b, limit);
    if (threadIdx.x == 0) *result = off == kNotPlaced ? 0u : 1u;
}

gpz_status sync_read_u32(const uint32_t* d, uint32_t* h, cudaStream_t s) {
    if (cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GPZ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GPZ_ERR_CUDA;
    return GPZ_OK;
}

}  // namespace

extern "C" {

int gpz_test_fail_next_allocations(int count) { return g_fail_allocs.exchange(count > 0 ? count : 0); }

uint64_t gpz_test_scan_workspace_size(void) { return ScanTestLayout().total; }

gpz_status gpz_test_scan_timeout(int batched, uint32_t wait_cycles, void* d_ws, uint64_t ws_size, void* stream) {
    const ScanTestLayout L;
    if (!d_ws || ws_size < L.total || !aligned(d_ws, kA) || wait_cycles < 1 || wait_cycles > (1u << 24))
        return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.ctrl);
    uint32_t* counter = status + 1;
    // every size 0x01010101 (clamped by the kernels to a block's largest
    // size); no tile state published; the tile counter at 1, so that the two
    // CTAs launched take tiles 1 and 2 and nobody ever processes tile 0
    if (cudaMemsetAsync(ws, 0, L.sizes, s) != cudaSuccess) return GPZ_ERR_CUDA;
    if (cudaMemsetAsync(ws + L.sizes, 1, kTestBlocks * 4ull, s) != cudaSuccess) return GPZ_ERR_CUDA;
    if (cudaMemsetAsync(counter, 1, 1, s) != cudaSuccess) return GPZ_ERR_CUDA;
    cudaError_t e;
    if (batched) {
        BatchScanArgs a{};
        a.sizes = reinterpret_cast<const uint32_t*>(ws + L.sizes);
        a.total_blocks = kTestBlocks;
        a.offsets = reinterpret_cast<unsigned long long*>(ws + L.offsets);
        a.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
        a.tile_counter = counter;
        a.status = status;
        a.wait_cycles = wait_cycles;
        e = launch_batch_scan(a, s, kTestTiles - 1);
    } else {
        ScanArgs a{};
        a.sizes = reinterpret_cast<const uint32_t*>(ws + L.sizes);
        a.nblocks = kTestBlocks;
        a.n = (uint64_t)kTestBlocks * kBlock;
        a.F = 1;
        a.table = reinterpret_cast<uint32_t*>(ws + L.offsets);
        a.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
        a.tile_counter = counter;
        a.status = status;
        a.wait_cycles = wait_cycles;
        e = launch_scan(a, s, kTestTiles - 1);
    }
    if (e != cudaSuccess) return GPZ_ERR_CUDA;
    uint32_t st = 0;
    const gpz_status rc = sync_read_u32(status, &st, s);
    return rc != GPZ_OK ? rc : (gpz_status)st;
}

gpz_status gpz_test_block_lookback_timeout(uint32_t block, uint32_t wait_cycles, void* d_ws, uint64_t ws_size,
                                           int* h_placed, void* stream) {
    if (!d_ws || !h_placed || block < 1 || block > 4096 || ws_size < 8ull * (block + 1) || !aligned(d_ws, kA) ||
        wait_cycles < 1 || wait_cycles > (1u << 24))
        return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    // states of blocks 0..block-1: none published; the result word after them
    if (cudaMemsetAsync(ws, 0, 8ull * (block + 1), s) != cudaSuccess) return GPZ_ERR_CUDA;
    uint32_t* result = reinterpret_cast<uint32_t*>(ws + 8ull * block);
    gpz_test_lookback_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const unsigned long long*>(ws), block,
                                              (long long)wait_cycles, result);
    if (cudaGetLastError() != cudaSuccess) return GPZ_ERR_CUDA;
    uint32_t placed = 0;
    const gpz_status rc = sync_read_u32(result, &placed, s);
    if (rc != GPZ_OK) return rc;
    *h_placed = (int)placed;
    return GPZ_OK;
}

}  // extern "C"
