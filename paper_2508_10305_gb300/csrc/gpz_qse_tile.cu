// gpz_qse_tile.cu -- the fused compression kernel (quantisation, sorting,
// encoding; Sections 4.1-4.3) of single-array calls whose fields are 16-byte
// aligned, with the block's input in shared memory instead of registers.
//
// One CTA of 256 threads owns one block of 1024 particles, as in
// gpz_qse_block.cuh's fast path, and produces the same words; what differs
// is where the data lives:
//   - thread 0 loads the block's F x 1024 values into a shared tile with one
//     bulk copy per field, completing on an mbarrier (the few values of a
//     ragged last block beyond a multiple of four are loaded by plain loads);
//   - threads 0..F-1 derive their field's constants (minimum, code width,
//     segment split, record offset) once, into shared memory: with a
//     relative bound from the block extremes of the range pass, loaded with
//     the field's step constants in one round trip while the tile is in
//     flight; otherwise from the tile;
//   - each thread quantises its 4 particles of every field from the tile;
//   - once every value is quantised the tile is dead, and the encoded
//     block's staging words are assembled in the same bytes, then written to
//     the block's temporary slot by one bulk copy.
// Holding no input in registers, a thread needs about 40 registers instead
// of 48, and with the staging words overlaying the tile a CTA needs about 36
// KB of shared memory for F = 6: six CTAs per SM instead of five.  The
// kernel is latency-bound (instruction issue waits on shared memory, warp
// collectives and barriers), so residency is what pays.
//
// With a relative bound the block's extremes come from the range pass and
// must bound the block's values (they are exact there): codes are monotone in
// the value, so every code then fits the width derived from the maximum, and
// every key stays below 2^keybits, which the histogram's indexing relies on.
//
// Blocks the fast path cannot take (a value needing a fallback candidate, a
// code >= 2^23, a record > 128 bits) go to the general kernel's list; blocks
// with a non-finite value or no gain are stored raw -- both exactly as in
// gpz_qse_block.cuh.
#include "gpz_qse_tile.cuh"

namespace gpz {

template <int F, bool PRE>
__global__ void __launch_bounds__(kThreads, 6) gpz_qse_tile_kernel(QseArgs a) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ __align__(8) TileShared S;
    if ((uint64_t)(blockIdx.x + 1) * kBlock <= a.n)
        qse_block_tile<F, true, PRE>(a, dsm, S, GridBlock{});
    else
        qse_block_tile<F, false, PRE>(a, dsm, S, GridBlock{});
}

template <int F, bool PRE>
cudaError_t launch_qse_tile_fp(const QseArgs& a, cudaStream_t s) {
    const size_t smem = tile_smem_bytes(F);
    auto kern = gpz_qse_tile_kernel<F, PRE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    kern<<<a.nblocks, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_qse_general(a, s);
}

cudaError_t launch_qse_tile(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    if (!a.bulk_ok) return cudaErrorInvalidValue;
    if (a.interleaved) return launch_qse_tile_aos(a, s);  // gpz_aos.cu
    const bool pre = a.bext != nullptr;
    switch (a.F) {
#define GPZ_CASE(FF) \
    case FF: return pre ? launch_qse_tile_fp<FF, true>(a, s) : launch_qse_tile_fp<FF, false>(a, s);
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

}  // namespace gpz
