// gpz_batch_decode.cu -- batched decompression: every block of every chunk of
// a batch in one persistent launch (Section 3.2, the reverse of compression
// without sorting).  The per-block code is the single-stream code, so each
// chunk's values are the ones a call of its own produces; a chunk whose
// stream fails a check gets GPZ_ERR_CORRUPT in its own status word.
#include "gpz_batch.cuh"
#include "gpz_decode_block.cuh"

namespace gpz {

template <int F>
__global__ void __launch_bounds__(kDecThreads, 5) gpz_batch_decompress_kernel(BatchDecompressArgs g) {
    __shared__ DecShared S;
    __shared__ DecArgs A;
    __shared__ uint32_t s_ticket;
    const int t = threadIdx.x;
    const uint32_t* block_end = g.block_end + g.first;
    uint32_t cur = 0, loaded = 0xffffffffu;  // group-relative
    if (t == 0) s_ticket = atomicAdd(g.ticket, g.claim);
    __syncthreads();
    uint32_t base = s_ticket;
    while (base < g.total_blocks) {
        uint32_t next = 0;
        if (t == 0) next = atomicAdd(g.ticket, g.claim);  // in flight while the blocks decode
        const uint32_t stop = g.total_blocks - base < g.claim ? g.total_blocks : base + g.claim;
        for (uint32_t q = base; q < stop; ++q) {
            const uint32_t gb = g.block_first + q;
            cur = find_chunk(block_end, g.nchunks, gb, cur);
            const BatchChunk* ch = g.chunks + g.first + cur;
            if (cur != loaded) {
                if (t < kMaxFields) A.out[t] = ch->out[t];
                if (t == 32) {
                    A.stream = ch->src;
                    A.total_words = ch->words;
                    A.n = ch->n;
                    A.F = F;
                    A.nblocks = ch->nblocks;
                    A.status = g.chunk_status + g.first + cur;
                }
                __syncthreads();
                loaded = cur;
            }
            decode_block<F>(A, S, gb - ch->block_base);
            __syncthreads();
        }
        if (t == 0) s_ticket = next;
        __syncthreads();
        base = s_ticket;
    }
}

int batch_decompress_max_ctas_per_sm(int F) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (F) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<1>, kDecThreads, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<2>, kDecThreads, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<3>, kDecThreads, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<4>, kDecThreads, 0); break;
        case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<5>, kDecThreads, 0); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<6>, kDecThreads, 0); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<7>, kDecThreads, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gpz_batch_decompress_kernel<8>, kDecThreads, 0); break;
    }
    return e == cudaSuccess ? n : 0;
}

cudaError_t launch_batch_decompress(const BatchDecompressArgs& a, int F, int grid, cudaStream_t s) {
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
