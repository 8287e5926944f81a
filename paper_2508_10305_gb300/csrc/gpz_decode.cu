// gpz_decode.cu -- GPZ decompression (Section 3.2, last paragraph: the
// reverse of compression without sorting; Table 1 "Decompression").
//
// One warp per 1024-particle block, kDecWarps warps per CTA.  Per warp:
//   1. check the stream header and the block's table entries;
//   2. raw block: copy the stored values;
//   3. encoded block: decode the delta and count arrays 32 entries at a time
//      (each lane extracts one fixed-length value with a funnel shift), warp
//      prefix sums give the unique segment ids and the run starts; the run
//      starts are marked in a 1024-bit mask;
//   4. for sorted position j, its run is the number of run starts <= j
//      (popcount of the mask prefix), its key the run's id; the record at
//      bit j*W gives the offsets and extra-field codes; every value is
//      rebuilt as fma(q, step, min) and stored coalesced.
// Every read stays inside the stream and every check failure sets
// GPZ_ERR_CORRUPT in the status word; the kernel never traps.
#include "gpz_internal.cuh"

namespace gpz {

struct DecMeta {
    float mn[kMaxFields];
    float s[kMaxFields];
    uint32_t w[kMaxFields];       // record width per field
    uint32_t o[kMaxFields];       // offset bits (positions)
    uint32_t gmask[kMaxFields];   // segId mask (positions)
    uint32_t kshift[kMaxFields];
    uint32_t rshift[kMaxFields];
};

__device__ __forceinline__ uint32_t mask_bits(uint32_t w) { return w >= 32u ? 0xffffffffu : ((1u << w) - 1u); }

// Value k of a fixed-length array of width w (<= 31) starting at A.
__device__ __forceinline__ uint32_t extract(const uint32_t* A, uint32_t k, uint32_t w) {
    if (w == 0u) return 0u;
    const uint32_t p = k * w;
    const uint32_t wi = p >> 5, sh = p & 31u;
    const uint32_t lo = __ldg(A + wi);
    const uint32_t hi = (sh + w > 32u) ? __ldg(A + wi + 1) : 0u;
    return __funnelshift_r(lo, hi, sh) & mask_bits(w);
}

__global__ void __launch_bounds__(32 * kDecWarps) gpz_decompress_kernel(DecArgs a) {
    __shared__ uint32_t s_uniq[kDecWarps][kMaxBins];
    __shared__ uint32_t s_mask[kDecWarps][32];
    __shared__ DecMeta s_meta[kDecWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b = blockIdx.x * kDecWarps + warp;
    if (b >= a.nblocks) return;
    const uint32_t* S = a.stream;
    const int F = a.F;
    const int P = F < 3 ? F : 3;
    DecMeta* m = &s_meta[warp];
    uint32_t* uniq = s_uniq[warp];
    uint32_t* mask = s_mask[warp];

    // ---- 1. header (16 words were checked present by the host)
    const uint32_t hw = lane < kHeaderWords ? __ldg(S + lane) : 0u;
    bool ok = true;
    switch (lane) {
        case 0: ok = hw == kMagic; break;
        case 1: ok = hw == kVersion; break;
        case 2: ok = hw == (uint32_t)F; break;
        case 3: ok = hw <= (uint32_t)kMaxSegBits; break;
        case 4: ok = hw == (uint32_t)kBlock; break;
        case 5: ok = hw <= 1u; break;
        case 6: ok = hw == (uint32_t)(a.n & 0xffffffffull); break;
        case 7: ok = hw == (uint32_t)(a.n >> 32); break;
        case 8: ok = hw == a.nblocks; break;
        case 9: break;
        default: ok = lane >= kHeaderWords || hw == 0u; break;
    }
    const uint32_t G = __shfl_sync(0xffffffffu, hw, 3);
    const uint32_t payload_words = __shfl_sync(0xffffffffu, hw, 9);
    const uint64_t table_start = kHeaderWords + 2ull * F;
    const uint64_t payload_start = table_start + a.nblocks + 1;
    if (!__all_sync(0xffffffffu, ok) || payload_start + payload_words > a.total_words) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    const uint32_t off = __ldg(S + table_start + b), end = __ldg(S + table_start + b + 1);
    if (off > end || end > payload_words || (b == 0 && off != 0) || (b + 1 == a.nblocks && end != payload_words) ||
        end == off) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    const uint32_t* blk = S + payload_start + off;
    const uint32_t nw = end - off;
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = (int)((a.n - first) < (uint64_t)kBlock ? (a.n - first) : (uint64_t)kBlock);
    const uint32_t mode = __ldg(blk);

    // ---- 2. raw block
    if (mode & 1u) {
        if (mode != 1u || nw != 1u + (uint32_t)F * (uint32_t)n_b) {
            if (lane == 0) set_status(a.status, kStCorrupt);
            return;
        }
        for (int f = 0; f < F; ++f) {
            float* dst = nullptr;
#pragma unroll
            for (int k = 0; k < kMaxFields; ++k)
                if (k == f) dst = a.out[k];
            for (int i = lane; i < n_b; i += 32) dst[first + i] = __uint_as_float(__ldg(blk + 1 + f * n_b + i));
        }
        return;
    }

    // ---- 3. encoded block header
    const uint32_t U = (mode >> 1) & 0x7ffu, wd = (mode >> 12) & 31u, wc = (mode >> 17) & 31u;
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    if ((mode >> 22) != 0u || nw < hdr) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    uint32_t bits_lane = 0;
    if (lane < 4 * ((F + 3) >> 2)) bits_lane = (__ldg(blk + 1 + F + (lane >> 2)) >> (8 * (lane & 3))) & 0xffu;
    ok = lane < F ? bits_lane <= 31u : bits_lane == 0u;
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    uint32_t keybits = 0, W = 0;
    // widths are warp-uniform: gather them with shuffles
    uint32_t bitsv[kMaxFields];
#pragma unroll
    for (int f = 0; f < kMaxFields; ++f) bitsv[f] = __shfl_sync(0xffffffffu, bits_lane, f);
    {
        uint32_t ks = 0, rs = 0;
#pragma unroll
        for (int f = kMaxFields - 1; f >= 0; --f) {
            if (f < F) {
                const uint32_t g = f < P ? min(G, bitsv[f]) : 0u;
                const uint32_t w = f < P ? bitsv[f] - g : bitsv[f];
                if (lane == 0) {
                    m->w[f] = w;
                    m->o[f] = f < P ? w : 0u;
                    m->gmask[f] = mask_bits(g);
                    m->kshift[f] = ks;
                    m->rshift[f] = rs;
                }
                ks += g;
                rs += w;
            }
        }
        keybits = ks;
        W = rs;
    }
    if (lane < F) {
        m->mn[lane] = __uint_as_float(__ldg(blk + 1 + lane));
        m->s[lane] = __uint_as_float(__ldg(S + kHeaderWords + 2 * lane + 1));
    }
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = ceil_words((uint32_t)n_b * W);
    if (U < 1u || U > (uint32_t)n_b || U > (1u << keybits) || nw != hdr + dwords + cwords + rwords) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    const uint32_t* D = blk + hdr;
    const uint32_t* C = D + dwords;
    const uint32_t* R = C + cwords;
    mask[lane] = 0u;
    __syncwarp();

    // ---- 3b. unique ids and run starts
    bool bad = false;
    uint32_t carry_u = 0, carry_c = 0;
    const uint32_t idlimit = 1u << keybits;
    for (uint32_t s0 = 0; s0 < U; s0 += 32) {
        const uint32_t k = s0 + lane;
        const bool valid = k < U;
        const uint32_t d = valid ? extract(D, k, wd) : 0u;
        const uint32_t c = valid ? extract(C, k, wc) : 0u;
        if (valid && (d >= idlimit || c == 0u || c > (uint32_t)n_b || (k > 0 && d == 0u))) bad = true;
        const uint32_t dd = d < idlimit ? d : 0u;
        const uint32_t cc = c <= (uint32_t)n_b ? c : 0u;
        const uint32_t iu = warp_incl_sum(dd) + carry_u;
        const uint32_t ic = warp_incl_sum(cc) + carry_c;
        if (valid) {
            const uint32_t start = ic - cc;
            if (iu >= idlimit || start >= (uint32_t)n_b) {
                bad = true;
            } else {
                uniq[k] = iu;
                atomicOr(&mask[start >> 5], 1u << (start & 31u));
            }
        }
        carry_u = __shfl_sync(0xffffffffu, iu, 31);
        carry_c = __shfl_sync(0xffffffffu, ic, 31);
        if (carry_u >= idlimit) carry_u = idlimit;  // stays bounded for corrupt input
        if (carry_c > (uint32_t)n_b) carry_c = (uint32_t)n_b + 1u;
    }
    if (__any_sync(0xffffffffu, bad) || carry_c != (uint32_t)n_b) {
        if (lane == 0) set_status(a.status, kStCorrupt);
        return;
    }
    __syncwarp();

    // ---- 4. expand runs, decode records, rebuild values
    const uint32_t mrow = mask[lane];
    const uint32_t pre = warp_incl_sum(__popc(mrow)) - __popc(mrow);
    const bool fast = W <= 64u;
    const unsigned long long wmask = W >= 64u ? ~0ull : ((1ull << W) - 1ull);
    for (int r = 0; r < (n_b + 31) / 32; ++r) {
        const int j = 32 * r + lane;
        const bool valid = j < n_b;
        const uint32_t m_r = __shfl_sync(0xffffffffu, mrow, r);
        const uint32_t p_r = __shfl_sync(0xffffffffu, pre, r);
        int run = (int)(p_r + __popc(m_r & lanemask_le())) - 1;
        run = run < 0 ? 0 : (run >= (int)U ? (int)U - 1 : run);
        const uint32_t key = uniq[run];
        unsigned long long rec = 0ull;
        if (fast && valid && W > 0u) {
            const uint32_t p = (uint32_t)j * W;
            const uint32_t wi = p >> 5, sh = p & 31u;
            const uint32_t w0 = __ldg(R + wi);
            const uint32_t w1 = wi + 1 < rwords ? __ldg(R + wi + 1) : 0u;
            const uint32_t w2 = wi + 2 < rwords ? __ldg(R + wi + 2) : 0u;
            const unsigned long long lo = ((unsigned long long)w1 << 32) | w0;
            rec = sh ? ((lo >> sh) | ((unsigned long long)w2 << (64u - sh))) : lo;
            rec &= wmask;
        }
        for (int f = 0; f < F; ++f) {
            const uint32_t wf = m->w[f];
            uint32_t code = 0u;
            if (wf) {
                if (fast) {
                    code = (uint32_t)(rec >> m->rshift[f]) & mask_bits(wf);
                } else if (valid) {
                    const uint32_t p = (uint32_t)j * W + m->rshift[f];
                    const uint32_t wi = p >> 5, sh = p & 31u;
                    const uint32_t lo = __ldg(R + wi);
                    const uint32_t hi = (sh + wf > 32u) ? __ldg(R + wi + 1) : 0u;
                    code = __funnelshift_r(lo, hi, sh) & mask_bits(wf);
                }
            }
            uint32_t q = code;
            if (f < P) q |= ((key >> m->kshift[f]) & m->gmask[f]) << m->o[f];
            if (valid) {
                float* dst = nullptr;
#pragma unroll
                for (int k = 0; k < kMaxFields; ++k)
                    if (k == f) dst = a.out[k];
                dst[first + j] = __fmaf_rn(__uint2float_rn(q), m->s[f], m->mn[f]);
            }
        }
    }
}

cudaError_t launch_decompress(const DecArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    const unsigned grid = (a.nblocks + kDecWarps - 1) / kDecWarps;
    gpz_decompress_kernel<<<grid, 32 * kDecWarps, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpz
