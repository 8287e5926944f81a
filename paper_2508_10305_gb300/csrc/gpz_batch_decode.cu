// gpz_batch_decode.cu -- batched decompression: every block of every chunk of
// a group (one field count) in one launch, one CTA per block (Section 3.2,
// the reverse of compression without sorting).  The per-block code is the
// single-stream code, so each chunk's values are the ones a call of its own
// produces; a chunk whose stream fails a check gets GPZ_ERR_CORRUPT in its
// own status word.
#include "gpz_batch.cuh"
#include "gpz_decode_block.cuh"

namespace gpz {

// One CTA per block of the group.  The map kernel has gathered every
// block's table entries (block_loc), so a CTA needs one round trip for its
// chunk and its place, and one for its words.
template <int F>
__global__ void __launch_bounds__(kDecThreads, 8) gpz_batch_decompress_kernel(BatchDecompressArgs g) {
    __shared__ DecShared S;
    __shared__ DecArgs A;
    __shared__ uint32_t s_b;  // block within its chunk
    const int t = threadIdx.x, lane = t & 31;
    const uint32_t gb = g.block_first + blockIdx.x;
    // the block's place (gathered by the map kernel) in the same round trip
    // as its chunk: lanes 0, 1, 2 of every warp take the payload size and the
    // block's two table entries
    const uint32_t hw_pre = lane < 3 ? __ldg(reinterpret_cast<const uint32_t*>(g.block_loc + gb) + lane) : 0u;
    const uint32_t c = __ldg(g.block_map + gb);
    const BatchChunk* ch = g.chunks + c;
    if (t < F) A.out[t] = ch->out[t];
    if (t == 32) {
        A.stream = ch->src;
        A.total_words = ch->words;
        A.n = ch->n;
        A.F = F;
        A.nblocks = ch->nblocks;
        A.status = g.chunk_status + c;
        A.interleaved = 0;
        s_b = gb - ch->block_base;
    }
    __syncthreads();
    decode_block<F, DecSlotBlock, false, false, DecShared, true>(A, S, DecSlotBlock{&s_b}, hw_pre);
}

cudaError_t launch_batch_decompress(const BatchDecompressArgs& a, int F, cudaStream_t s) {
    const unsigned grid = a.total_blocks;
    switch (F) {
        case 1: gpz_batch_decompress_kernel<1><<<grid, kDecThreads, 0, s>>>(a); break;
        case 2: gpz_batch_decompress_kernel<2><<<grid, kDecThreads, 0, s>>>(a); break;
        case 3: gpz_batch_decompress_kernel<3><<<grid, kDecThreads, 0, s>>>(a); break;
        case 4: gpz_batch_decompress_kernel<4><<<grid, kDecThreads, 0, s>>>(a); break;
        case 5: gpz_batch_decompress_kernel<5><<<grid, kDecThreads, 0, s>>>(a); break;
        case 6: gpz_batch_decompress_kernel<6><<<grid, kDecThreads, 0, s>>>(a); break;
        case 7: gpz_batch_decompress_kernel<7><<<grid, kDecThreads, 0, s>>>(a); break;
        case 8: gpz_batch_decompress_kernel<8><<<grid, kDecThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gpz
