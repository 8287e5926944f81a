// gpz_internal.cuh -- device-side constants, kernel argument blocks and warp
// helpers of libgpz (sm_103a).  The stream format implemented here is the one
// of include/gpz.h: a 16-word header, (eb, step) per field, a table of block
// word offsets, then one encoded or raw block per 1024 particles.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gpz {

constexpr int kBlock = 1024;             // particles per block (Section 4.2: 32 threads x 32 points)
constexpr uint32_t kMagic = 0x315A5047u; // 'G','P','Z','1'
constexpr uint32_t kVersion = 1;
constexpr int kHeaderWords = 16;
constexpr int kMaxFields = 8;
constexpr int kMaxSegBits = 3;
constexpr int kMaxBins = 512;            // 2^(3 * kMaxSegBits) linearised segment ids
constexpr int kRow = 33;                 // padded shared-memory row of 32 values
constexpr int kPadWords = 32 * kRow;     // 1056: 1024 values in padded rows
constexpr int kQseThreads = 256;         // one CTA per particle block, 4 particles per thread
constexpr int kDecThreads = 256;         // one CTA per particle block, 4 positions per thread
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kRangeThreads = 256;
constexpr int kCompactWarps = 8;

// Status codes written to the workspace status word (values of gpz_status).
constexpr uint32_t kStCapacity = 2;
constexpr uint32_t kStCorrupt = 3;
constexpr uint32_t kStTimeout = 6;

// Limit of every device-side wait on another CTA, in SM cycles (about a
// second at 2 GHz): a wait that runs out records kStTimeout and the waiting
// CTA carries on without the value it waited for.
constexpr long long kWaitCycles = 1ll << 31;

struct FieldParams {
    float eb;    // RN32(eb), stored in the header
    float s;     // quantisation step RN32(eb * 63/32)
    float inv;   // RN32(1 / s): the precomputed reciprocal (Section 5.1)
    float ebchk; // RD32(eb * (1 - 2^-22)): the verification threshold
};

// Argument blocks (passed by value).
struct RangeArgs {
    const float* fields[kMaxFields];
    uint64_t n;
    int F;
    int vec_ok;                 // every field pointer 16-byte aligned
    double rel[kMaxFields];
    float2* partials;           // [gridDim.x][F] (min, max)
    uint32_t* done_counter;
    FieldParams* d_params;      // out
    uint2* bext;                // out, [nblocks][F]: each block's extremes (order keys), (0, 0) if non-finite
};

struct QseArgs {
    const float* fields[kMaxFields];
    uint64_t n;
    uint32_t nblocks;
    int F;
    int G;
    int bulk_ok;                // every field pointer 16-byte aligned: stage tiles with bulk copies
    int interleaved;            // fields[0] holds F-field records: field f of particle i at fields[0][i * F + f]
    FieldParams params[kMaxFields];
    const FieldParams* d_params; // device constants (relative bound) or nullptr
    const uint2* bext;          // each block's extremes from the range pass, or nullptr
    const unsigned long long* binfo; // each block's widths and flags (gpz_block_info_kernel), or nullptr
    uint32_t* temp;             // [nblocks][slot_words]
    uint32_t slot_words;
    uint32_t* sizes;            // [nblocks] words per block
    uint32_t* perm;             // [n] or nullptr
    uint32_t* status;
    uint32_t* general_list;     // [nblocks] blocks left to the general kernel
    uint32_t* general_count;    // zeroed
    // Fused compaction only (gpz_qse_direct_kernel): the stream's payload,
    // the words it can hold, the per-block look-back states (zeroed) and a
    // count of the blocks that could not be placed directly.
    uint32_t* direct;
    uint64_t direct_capacity;
    unsigned long long* bstate;
    uint32_t* deferred_count;
};

constexpr uint32_t kPlaced = 0x80000000u;  // in a block's word count: already in the stream

// Compaction forms of the per-block code: the temporary slot only (Section
// 4.4's three steps), or fused (placed by the block itself after its
// look-back over its predecessors' published sizes).
constexpr int kCmTemp = 0, kCmDirect = 1;

struct F64Args {                // fp64 input and output (gpz_f64.cu)
    const double* in[kMaxFields];
    float* out32[kMaxFields];
    const float* in32[kMaxFields];
    double* out64[kMaxFields];
    uint64_t n;
    int F;
    unsigned long long* res;    // [F][3]: min key, max key, largest rounding error (bits)
};

struct ScanArgs {
    const uint32_t* sizes;      // [nblocks]
    uint32_t nblocks;
    uint64_t n;                 // particles (a block's size never exceeds its raw size)
    int F;
    uint32_t* table;            // [nblocks + 1] in the stream
    unsigned long long* tile_state; // [ntiles], zeroed
    uint32_t* tile_counter;     // zeroed
    uint32_t* status;
    long long wait_cycles;      // limit of a look-back wait in SM cycles; 0: kWaitCycles
};

struct CompactArgs {
    const uint32_t* temp;
    uint32_t slot_words;
    const uint32_t* sizes;
    const uint32_t* table;      // [nblocks + 1]
    uint32_t* stream;           // stream base
    uint32_t payload_start;     // words
    uint32_t nblocks;
    uint64_t n;
    int F;
    int G;
    int mode;
    FieldParams params[kMaxFields];
    const FieldParams* d_params;
    unsigned long long* d_out_size; // nullable
    uint32_t* unplaced;         // nullable: counts the blocks this kernel moves (in-kernel compaction forms)
    uint32_t version;           // header word 1
    uint32_t ext_words;         // nonzero: the header extension is ext[0..ext_words) instead of (eb, s) per field
    uint32_t ext[4 * kMaxFields];
};

struct DecArgs {
    const uint32_t* stream;
    uint64_t total_words;
    float* out[kMaxFields];
    uint64_t n;
    int F;
    uint32_t nblocks;
    uint32_t* status;
    int interleaved;            // out[0] receives F-field records: field f of particle i at out[0][i * F + f]
};

// The constants of one field under a relative bound rel, from the field's
// range [lo, hi] (lo > hi when the field holds no value): eb = rel * (hi - lo)
// when that is a finite positive number, else eb = rel; then the step
// eb * 63/32, its reciprocal and the verification threshold, all from the
// double eb (one rounding each).
__device__ __forceinline__ FieldParams range_params(float lo, float hi, double rel) {
    double eb = rel;
    if (lo <= hi) {
        const double range = (double)hi - (double)lo;
        if (range > 0.0 && range < HUGE_VAL) {
            const double e = rel * range;
            if (e > 0.0 && e < HUGE_VAL) eb = e;
        }
    }
    FieldParams p;
    p.eb = __double2float_rn(eb);
    p.s = __double2float_rn(eb * 1.96875);
    p.inv = __double2float_rn(1.0 / (double)p.s);
    p.ebchk = __double2float_rd(eb * (1.0 - 0x1p-22));
    return p;
}

// ---------------------------------------------------------------- helpers

// ceil(2^32 / d) for d = 1..255 (entry 0 unused), built at compile time: with
// m = ceil(2^32 / d), floor(n / d) = floor(n * m / 2^32) exactly for n < 2^18
// (the multiply's relative error stays below 2^-14 < 1/d).
struct DivMagic {
    unsigned long long m[256];
    constexpr DivMagic() : m() {
        for (int d = 1; d < 256; ++d) m[d] = ((1ull << 32) + (unsigned long long)d - 1ull) / (unsigned long long)d;
    }
};
__constant__ DivMagic kDivMagic = DivMagic();

// floor(n / d) for n < 2^18, 1 <= d <= 255.
__device__ __forceinline__ uint32_t div_small(uint32_t n, uint32_t d) {
    const unsigned long long m = kDivMagic.m[d];
    return __umulhi(n, (uint32_t)m) + ((m >> 32) ? n : 0u);
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t code) {
    atomicCAS(st, 0u, code);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int pad_idx(int j) { return (j >> 5) * kRow + (j & 31); }

__device__ __forceinline__ uint32_t bit_width(uint32_t v) { return 32u - (uint32_t)__clz(v); }

__device__ __forceinline__ uint32_t ceil_words(uint32_t bits) { return (bits + 31u) >> 5; }

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
    return __reduce_max_sync(0xffffffffu, v);
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
    return __reduce_add_sync(0xffffffffu, v);
}

__device__ __forceinline__ float warp_min_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_max_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Inclusive prefix sum over the warp.
__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Inclusive prefix maximum over the warp (signed).
__device__ __forceinline__ int warp_incl_max(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = max(v, t);
    }
    return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier + bulk copy global -> shared

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive (the one expected arrival) and announce `bytes` of bulk copies.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of the mbarrier, for at most kWaitCycles SM
// cycles; on expiry record kStTimeout, wait once more as long (so that bulk
// copies still in flight into this CTA's shared memory are not left behind
// by an exiting CTA), and return false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            set_status(status, kStTimeout);
            t0 = clock64();
            while (!mbar_try_wait(bar, parity))
                if (clock64() - t0 > kWaitCycles) break;
            return false;
        }
    }
    return true;
}

// One-dimensional bulk copy global -> shared, completing on the mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- bulk copy shared -> global (async proxy)

// Orders this thread's earlier shared-memory writes before later reads of
// them by the async proxy (a bulk copy issued after a barrier).
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread: copy `bytes` (a multiple of 16) from shared memory to global
// memory, both 16-byte aligned, with one bulk copy, and wait until the copy
// has read its source (so that the CTA may exit or reuse the words).
__device__ __forceinline__ void bulk_s2g(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// ---------------------------------------------------------------- acquire / release (look-back scan)

// A look-back reads other CTAs' published states with relaxed loads: the
// value it needs is in the state word itself, and a gpu-scope acquire load
// would also invalidate the SM's L1 for every CTA resident there.  A reader
// that goes on to read data the state vouches for issues one fence first.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------- launch wrappers (defined in the .cu files)

cudaError_t launch_range(const RangeArgs& a, int grid, cudaStream_t s);
cudaError_t launch_qse(const QseArgs& a, cudaStream_t s);         // fast kernel, then the general list
cudaError_t launch_qse_direct(const QseArgs& a, cudaStream_t s);  // the same with blocks placed directly
cudaError_t launch_qse_general(const QseArgs& a, cudaStream_t s);
cudaError_t launch_qse_pre(const QseArgs& a, cudaStream_t s);     // fast kernel reading a.bext
cudaError_t launch_qse_tile(const QseArgs& a, cudaStream_t s);    // shared-memory tile kernel (16-byte aligned fields)
cudaError_t launch_qse_tile_aos(const QseArgs& a, cudaStream_t s); // the same on interleaved records (16-byte aligned)
cudaError_t launch_decompress_aos(const DecArgs& a, cudaStream_t s); // decompression into interleaved records
cudaError_t launch_block_info(const uint2* bext, const FieldParams* d_params, uint32_t nblocks, int F,
                              unsigned long long* binfo, cudaStream_t s);
cudaError_t launch_scan(const ScanArgs& a, cudaStream_t s, unsigned grid = 0);  // grid 0: one CTA per tile
cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);
cudaError_t launch_decompress(const DecArgs& a, cudaStream_t s);

}  // namespace gpz
