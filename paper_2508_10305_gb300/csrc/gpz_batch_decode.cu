// gpz_batch_decode.cu -- batched decompression: every block of every chunk of
// a batch in one persistent launch (Section 3.2, the reverse of compression
// without sorting).  The per-block code is the single-stream code, so each
// chunk's values are the ones a call of its own produces; a chunk whose
// stream fails a check gets GPZ_ERR_CORRUPT in its own status word.
#include "gpz_batch.cuh"
#include "gpz_decode_block.cuh"

namespace gpz {

// The loop state lives in shared memory: thread 0 claims and decodes each
// item between barriers, so that no register stays live across the inlined
// block code (the block index is re-read from the slot where it is used).
struct DecLoopState {
    uint32_t q, stop, seen;  // current block, end of the claimed run, the counter as of the last claim
    uint32_t cur, loaded;    // chunk of the current block, chunk whose arguments are in A
    uint32_t cbase, cend;    // global blocks [cbase, cend) of chunk cur
    uint32_t b;              // block within its chunk
};

template <int F>
__global__ void __launch_bounds__(kDecThreads, 5) gpz_batch_decompress_kernel(BatchDecompressArgs g) {
    __shared__ DecShared S;
    __shared__ DecArgs A;
    __shared__ DecLoopState L;
    const int t = threadIdx.x;
    if (t == 0) {
        L.q = L.stop = L.seen = L.cur = 0u;
        L.cbase = L.cend = 0u;
        L.loaded = 0xffffffffu;
    }
    for (;;) {
        if (t == 0) {
            if (L.q >= L.stop) {  // claim the next run of blocks (shorter runs near the end)
                const uint32_t left = g.total_blocks > L.seen ? g.total_blocks - L.seen : 0u;
                uint32_t k = left / (2u * gridDim.x);
                k = k < 1u ? 1u : (k < g.claim ? k : g.claim);
                const uint32_t b0 = atomicAdd(g.ticket, k);
                L.seen = b0 + k;
                L.q = b0;
                L.stop = g.total_blocks - min(b0, g.total_blocks) < k ? g.total_blocks : b0 + k;
            }
            if (L.q < g.total_blocks) {
                const uint32_t gb = g.block_first + L.q;
                if (gb < L.cbase || gb >= L.cend) {  // another chunk: search (usually one probe)
                    const uint32_t cur = find_chunk(g.block_end + g.first, g.nchunks, gb, L.cur);
                    L.cur = cur;
                    L.cend = __ldg(g.block_end + g.first + cur);
                    L.cbase = g.chunks[g.first + cur].block_base;
                }
                L.b = gb - L.cbase;
            }
        }
        __syncthreads();
        if (L.q >= g.total_blocks) break;
        const uint32_t cur = L.cur;
        if (cur != L.loaded) {
            __syncthreads();  // every thread has read L.loaded
            const BatchChunk* ch = g.chunks + g.first + cur;
            if (t < kMaxFields) A.out[t] = ch->out[t];
            if (t == 32) {
                A.stream = ch->src;
                A.total_words = ch->words;
                A.n = ch->n;
                A.F = F;
                A.nblocks = ch->nblocks;
                A.status = g.chunk_status + g.first + cur;
            }
            if (t == 64) L.loaded = cur;
            __syncthreads();
        }
        decode_block<F>(A, S, DecSlotBlock{&L.b});
        __syncthreads();
        if (t == 0) L.q = L.q + 1u;
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
