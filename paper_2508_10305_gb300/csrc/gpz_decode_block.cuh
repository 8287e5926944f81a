// gpz_decode_block.cuh -- the per-block body of GPZ decompression (Section
// 3.2: the reverse of compression, without sorting), shared by the
// single-stream kernel (gpz_decode.cu) and the batched kernel
// (gpz_batch_decode.cu).  See gpz_decode.cu for the design.
#pragma once

#include "gpz_internal.cuh"

namespace gpz {


constexpr int kDecWarps = kDecThreads / 32;
// deltas (<= 512 x 9 bits) + counts (<= 512 x 11 bits) + records (<= 1024 x 128 bits)
constexpr uint32_t kDecStageWords = 144u + 176u + 4096u;
// words read past the staged ones: a value or record is extracted from a
// window of words that may reach past its array; those bits are never used
constexpr uint32_t kDecStagePad = 8u;


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

// Value k of a fixed-length array of width w (<= 31) held in shared memory
// (the word after the value's first may lie past the array: its bits are
// masked off).
__device__ __forceinline__ uint32_t extract_s(const uint32_t* A, uint32_t k, uint32_t w) {
    const uint32_t p = k * w;
    const uint32_t wi = p >> 5, sh = p & 31u;
    return __funnelshift_r(A[wi], A[wi + 1], sh) & mask_bits(w);
}

// (float)q for q < 2^23 with two full-rate operations.
__device__ __forceinline__ float small_u2f(uint32_t q) {
    return __fsub_rn(__uint_as_float(q + 0x4B000000u), 8388608.0f);
}

// Rebuild four consecutive values x = fma((float)q, step, min) and store them
// at out[first .. first + 3]: fp32, or widened to fp64 (exact) when OUT64 --
// then `out` holds a double array's address.
template <bool OUT64>
__device__ __forceinline__ void store4(float* out, uint64_t first, const uint32_t* qv, uint32_t bits, float s, float mn,
                                       int left) {
    if (OUT64) {
        float v[4];
        if (bits <= 23u) {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(small_u2f(qv[e]), s, mn);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(__uint2float_rn(qv[e]), s, mn);
        }
        double* dst = reinterpret_cast<double*>(out) + first;
        if (left >= 4 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
            reinterpret_cast<double2*>(dst)[0] = make_double2((double)v[0], (double)v[1]);
            reinterpret_cast<double2*>(dst)[1] = make_double2((double)v[2], (double)v[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e < left) dst[e] = (double)v[e];
        }
        return;
    }
    float* dst = out + first;
    float v[4];
    if (bits <= 23u) {  // uniform: codes below 2^23 convert with one add
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(small_u2f(qv[e]), s, mn);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = __fmaf_rn(__uint2float_rn(qv[e]), s, mn);
    }
    if (left >= 4 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
        __stcs(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < left) dst[e] = v[e];
    }
}

// Interleaved output: a block's values in record order in shared memory,
// value (j, f) at word j * F + f + j / 8 (the padding word every eight
// records spreads a warp's four-apart records over the banks).
template <int F>
__device__ __forceinline__ int rec_slot(int j, int f) { return j * F + f + (j >> 3); }
template <int F>
constexpr uint32_t rec_words() { return (uint32_t)(kBlock * F + kBlock / 8); }

// store4's values, for records j .. j + 3 of field f, into that staging.
template <int F>
__device__ __forceinline__ void store4_rec(float* recs, int j, int f, const uint32_t* qv, uint32_t bits, float s,
                                           float mn, int left) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float q = bits <= 23u ? small_u2f(qv[e]) : __uint2float_rn(qv[e]);
        if (e < left) recs[rec_slot<F>(j + e, f)] = __fmaf_rn(q, s, mn);
    }
}

// Records wider than 128 bits (rare): every code is read field by field from
// the stream itself; the block header is re-read here so that the common path
// passes nothing through memory.
template <int F, bool OUT64 = false, bool AOS = false>
__device__ __forceinline__ void decode_wide(const DecArgs& a, const uint32_t* blk, uint32_t rwords_off,
                                         uint32_t rwords, uint32_t W, uint32_t G, int j0, int n_b, uint64_t first,
                                         uint32_t key0, uint32_t key1, uint32_t key2, uint32_t key3,
                                         float* recs = nullptr) {
    constexpr int P = F < 3 ? F : 3;
    const uint32_t* R = blk + rwords_off;
    const uint32_t key[4] = {key0, key1, key2, key3};
    uint32_t rs = W;
    uint32_t ks = 0;
    // walk the fields from the top of the record down: field 0 is most significant
    uint32_t kacc[F], racc[F], wfv[F], gv[F];
    {
        uint32_t r = 0, k = 0;
        for (int f = F - 1; f >= 0; --f) {
            const uint32_t bf = (__ldg(blk + 1 + F + (f >> 2)) >> (8 * (f & 3))) & 0xffu;
            const uint32_t g = f < P ? min(G, bf) : 0u;
            gv[f] = g;
            wfv[f] = f < P ? bf - g : bf;
            racc[f] = r;
            kacc[f] = k;
            r += wfv[f];
            k += g;
        }
    }
    (void)rs;
    (void)ks;
    for (int f = 0; f < F; ++f) {
        const uint32_t bf = (__ldg(blk + 1 + F + (f >> 2)) >> (8 * (f & 3))) & 0xffu;
        const float mnf = __uint_as_float(__ldg(blk + 1 + f));
        const float sf = __uint_as_float(__ldg(a.stream + kHeaderWords + 2 * f + 1));
        const uint32_t cm = mask_bits(wfv[f]), gm = mask_bits(gv[f]);
        uint32_t qv[4];
        for (int e = 0; e < 4; ++e) {
            uint32_t code = 0u;
            if (cm && j0 + e < n_b) {
                const uint32_t p = (uint32_t)(j0 + e) * W + racc[f];
                const uint32_t wi = p >> 5, sh = p & 31u;
                const uint32_t lo = __ldg(R + wi);
                const uint32_t hi = (sh + wfv[f] > 32u) && (wi + 1 < rwords) ? __ldg(R + wi + 1) : 0u;
                code = __funnelshift_r(lo, hi, sh) & cm;
            }
            qv[e] = f < P ? (code | (((key[e] >> kacc[f]) & gm) << wfv[f])) : code;
        }
        if (AOS)
            store4_rec<F>(recs, j0, f, qv, bf, sf, mnf, n_b - j0);
        else
            store4<OUT64>(a.out[f], first + j0, qv, bf, sf, mnf, n_b - j0);
    }
}

struct DecCore {  // everything a block's decoding keeps in shared memory but its staged words
    uint16_t uniq[kMaxBins];
    uint32_t mask[32];
    uint32_t warp_uc[kDecWarps];  // per warp: id sum | count sum << 15
    uint32_t bad;
    // the block's constants, checked by warp 0 and read by every warp
    uint32_t ok, raw, U, wd, wc, W, keybits, G;
    uint4 lay[kMaxFields];      // per field: bits in the record, segId bits of a position axis,
                                // segId mask shifted above the segOffset bits, code width
    float2 ms[kMaxFields];      // per field: block minimum, step
};

struct DecShared : DecCore {
    uint64_t bar;  // the staging bulk copy
    // the block's words after its header, from word `shift` (the source's
    // offset from a 16-byte boundary, 0..3)
    alignas(16) uint32_t stage[kDecStageWords + kDecStagePad + 4];
};

// The same for interleaved output: the stage also takes the block's values
// in record order once its words are consumed.
constexpr uint32_t cmax(uint32_t x, uint32_t y) { return x > y ? x : y; }
template <int F>
struct DecSharedRec : DecCore {
    uint64_t bar;
    alignas(16) uint32_t stage[cmax(kDecStageWords + kDecStagePad + 4, 4 + rec_words<F>())];
};

// Codes of fields F-1 .. 0 of four records, consumed from the least
// significant end: field F-1 sits at bit 0 of the record and field 0 at the
// top.  rr[e] holds record e in its low bits (two words when W <= 64, else
// four); after each field the record is shifted right by the field's width
// and the key right by the axis' segId bits.  q = segId * 2^o + segOffset for
// a position axis, the whole code otherwise.
template <int F, bool WIDE, bool OUT64 = false, bool AOS = false>
__device__ __forceinline__ void decode_fields(const DecArgs& a, uint32_t (&rr)[4][4], uint32_t (&key)[4],
                                              const DecCore& L, uint64_t first, int left, float* recs = nullptr,
                                              int jl = 0) {
    constexpr int P = F < 3 ? F : 3;
#pragma unroll
    for (int f = F - 1; f >= 0; --f) {
        const uint4 lay = L.lay[f];
        const uint32_t wf = lay.x, cm = mask_bits(wf);
        uint32_t qv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint32_t q = rr[e][0] & cm;
            if (f < P) {
                q |= (key[e] << wf) & lay.z;
                key[e] >>= lay.y;
            }
            qv[e] = q;
            if (f > 0) {
                rr[e][0] = __funnelshift_r(rr[e][0], rr[e][1], wf);
                if (WIDE) {
                    rr[e][1] = __funnelshift_r(rr[e][1], rr[e][2], wf);
                    rr[e][2] = __funnelshift_r(rr[e][2], rr[e][3], wf);
                    rr[e][3] >>= wf;
                } else {
                    rr[e][1] >>= wf;
                }
            }
        }
        const float2 ms = L.ms[f];
        if (AOS)
            store4_rec<F>(recs, jl, f, qv, lay.w, ms.y, ms.x, left);
        else
            store4<OUT64>(a.out[f], first, qv, lay.w, ms.y, ms.x, left);
    }
}


// Where a CTA gets its block's index: the grid (one CTA per block), or a
// shared-memory slot (the batched kernel's block within its chunk) re-read at
// each use, so that the index holds no register through the block code.
struct DecGridBlock {
    __device__ __forceinline__ uint32_t b() const { return blockIdx.x; }
};
struct DecSlotBlock {
    const volatile uint32_t* slot;
    __device__ __forceinline__ uint32_t b() const { return *slot; }
};

// Decode block idx.b() of the stream described by a (every thread of the CTA).
// The format checks and the block's constants (warp 0 alone; every lane
// calls): from the stream header words hv (lane k holds word k), the block's
// first words bw (lane k holds word k, up to the block header's end) and the
// steps (lane f holds field f's), and the block's table entries; into S.
template <int F>
__device__ __forceinline__ void decode_checks(const DecArgs& a, DecCore& S, uint32_t hv, uint32_t bw, float step,
                                              bool inside, uint32_t b, uint32_t off, uint32_t end,
                                              uint32_t payload_words, int n_b) {
    constexpr int P = F < 3 ? F : 3;
    const int lane = threadIdx.x & 31;
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    const uint32_t nw = end - off;
        bool ok = true;
    switch (lane) {
        case 0: ok = hv == kMagic; break;
        case 1: ok = hv == kVersion; break;
        case 2: ok = hv == (uint32_t)F; break;
        case 3: ok = hv <= (uint32_t)kMaxSegBits; break;
        case 4: ok = hv == (uint32_t)kBlock; break;
        case 5: ok = hv <= 1u; break;
        case 6: ok = hv == (uint32_t)(a.n & 0xffffffffull); break;
        case 7: ok = hv == (uint32_t)(a.n >> 32); break;
        case 8: ok = hv == a.nblocks; break;
        case 9: break;
        default: ok = lane >= 10 + 6 || hv == 0u; break;
    }
    const uint32_t G = __shfl_sync(0xffffffffu, hv, 3);
    ok = __all_sync(0xffffffffu, ok) && inside && !(b == 0 && off != 0) &&
         !(b + 1 == a.nblocks && end != payload_words) && end != off;
    // the block header: mode word, minima, width bytes
    const uint32_t mode = __shfl_sync(0xffffffffu, bw, 0);
    const bool raw = ok && (mode & 1u);
    if (raw) ok = mode == 1u && nw == 1u + (uint32_t)F * (uint32_t)n_b;
    // lane f holds field f: its code width, minimum and step, and its
    // layout -- bits in the record, segId bits and mask
    const bool fl = lane < F;
    const uint32_t wword = __shfl_sync(0xffffffffu, bw, (1 + F + (lane >> 2)) & 31);
    const uint32_t bits = fl ? (wword >> (8 * (lane & 3))) & 0xffu : 0u;
    const float mn = __uint_as_float(__shfl_sync(0xffffffffu, bw, (1 + lane) & 31));
    const uint32_t bf = bits <= 31u ? bits : 0u;
    const uint32_t g = lane < P ? min(G, bf) : 0u;
    const uint32_t wf = fl ? bf - g : 0u;
    uint32_t U = 0, wd = 0, wc = 0, W = 0, keybits = 0;
    if (ok && !raw) {
        U = (mode >> 1) & 0x7ffu;
        wd = (mode >> 12) & 31u;
        wc = (mode >> 17) & 31u;
        ok = (mode >> 22) == 0u && nw >= hdr && !__any_sync(0xffffffffu, bits > 31u);
        // padding bytes of the last width word are zero
        const uint32_t lastw = __shfl_sync(0xffffffffu, bw, hdr - 1);
        if ((F & 3) != 0) ok = ok && (lastw >> (8 * (F & 3))) == 0u;
        keybits = __reduce_add_sync(0xffffffffu, g);
        W = __reduce_add_sync(0xffffffffu, wf);
        // ids are below 2^keybits and counts at most 1024, so their widths
        // are at most keybits and 11 bits: the deltas and counts then fit
        // the words reserved for them in the staging area
        ok = ok && U >= 1u && U <= (uint32_t)n_b && U <= (1u << keybits) && wd <= keybits && wc <= 11u &&
             nw == hdr + ceil_words(U * wd) + ceil_words(U * wc) + ceil_words((uint32_t)n_b * W);
    }
    if (lane == 0) {
        S.ok = ok;
        S.raw = raw;
        S.U = U;
        S.wd = wd;
        S.wc = wc;
        S.W = W;
        S.keybits = keybits;
        S.G = G;
    }
    if (fl) {
        S.lay[lane] = make_uint4(wf, g, mask_bits(g) << wf, bf);  // g + wf = bits <= 31
        S.ms[lane] = make_float2(mn, step);
    }
}

// Decode a block whose constants warp 0 has published in S (after a
// barrier): stage holds the block's words after its header, blk the block in
// the stream (read directly for raw blocks and records wider than 128 bits).
// The block's values, staged in record order (rec_slot), to out[0] with
// contiguous 16-byte stores when the records are 16-byte aligned (every
// thread, after the values are staged).
template <int F>
__device__ __forceinline__ void store_records(const DecArgs& a, const float* recs, uint32_t b, int n_b) {
    __syncthreads();  // every value is staged
    const int t = threadIdx.x, total = n_b * F;
    float* dst = a.out[0] + (uint64_t)b * kBlock * F;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        for (int k = 4 * t; k < total; k += 4 * kDecThreads) {
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = (k + c) / F;
                v[c] = k + c < total ? recs[k + c + (j >> 3)] : 0.0f;  // rec_slot(j, (k + c) - j F)
            }
            if (k + 4 <= total)
                __stcs(reinterpret_cast<float4*>(dst + k), make_float4(v[0], v[1], v[2], v[3]));
            else
                for (int c = 0; c < 4 && k + c < total; ++c) dst[k + c] = v[c];
        }
    } else {
        for (int k = t; k < total; k += kDecThreads) dst[k] = recs[k + ((k / F) >> 3)];
    }
}

// AOS: the values go to interleaved records at out[0]; `stage` must then
// hold rec_words<F>() words.
template <int F, bool OUT64 = false, bool AOS = false>
__device__ __forceinline__ void decode_tail(const DecArgs& a, DecCore& S, uint32_t* stage,
                                            const uint32_t* blk, uint32_t b, int n_b) {
    uint16_t* uniq = S.uniq;
    uint32_t* mask = S.mask;
    uint32_t& s_bad = S.bad;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    if (!S.ok) {
        if (t == 0) set_status(a.status, kStCorrupt);
        return;  // uniform across the CTA
    }

    // ---- 2. raw block
    if (S.raw) {
        if (AOS) {  // field-major in the stream: gather each record's fields
            float* dst = a.out[0] + (uint64_t)b * kBlock * F;
            for (int k = t; k < n_b * F; k += kDecThreads) {
                const int j = k / F, f = k - j * F;
                dst[k] = __uint_as_float(__ldg(blk + 1 + f * n_b + j));
            }
            return;
        }
#pragma unroll
        for (int f = 0; f < F; ++f)
            for (int i = t; i < n_b; i += kDecThreads)
            {
                const float v = __uint_as_float(__ldg(blk + 1 + f * n_b + i));
                if (OUT64)
                    reinterpret_cast<double*>(a.out[f])[(uint64_t)b * kBlock + i] = (double)v;
                else if (AOS)
                    a.out[0][((uint64_t)b * kBlock + i) * F + f] = v;
                else
                    a.out[f][(uint64_t)b * kBlock + i] = v;
            }
        return;
    }

    const uint32_t U = S.U, wd = S.wd, wc = S.wc, W = S.W, keybits = S.keybits;
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc), rwords = ceil_words((uint32_t)n_b * W);
    const uint32_t idlimit = 1u << keybits;

    // the deltas, counts and (when at most 128 bits wide) the records are in
    // the staging area, contiguous as in the stream
    const bool fast = W <= 128u;  // then dwords + cwords + rwords <= the staged words
    const uint32_t ndc = dwords + cwords;
    const uint32_t* sD = stage;
    const uint32_t* sC = stage + dwords;
    const uint32_t* sR = stage + ndc;
    const uint32_t k0 = 2u * t, k1 = k0 + 1u;
    const bool v0 = k0 < U, v1 = k1 < U;
    uint32_t d0 = v0 ? extract_s(sD, k0, wd) : 0u, d1 = v1 ? extract_s(sD, k1, wd) : 0u;
    uint32_t c0 = v0 ? extract_s(sC, k0, wc) : 0u, c1 = v1 ? extract_s(sC, k1, wc) : 0u;

    // ---- 3. unique ids and run starts
    {
        bool bad = (v0 && (d0 >= idlimit || c0 == 0u || c0 > (uint32_t)n_b || (k0 > 0 && d0 == 0u))) ||
                   (v1 && (d1 >= idlimit || c1 == 0u || c1 > (uint32_t)n_b || d1 == 0u));
        if (bad) d0 = d1 = c0 = c1 = 0u;  // keep the sums small; the block is rejected below
        // one scan of both sums: a warp's id sum is below 2^15 (32 x 2 x 511)
        // and its count sum at most 2^16 (32 x 2 x 1024), so they share a word
        const uint32_t su = d0 + d1, sc = c0 + c1;
        const uint32_t iuc = warp_incl_sum(su | (sc << 15));
        const uint32_t iu = iuc & 0x7fffu, ic = iuc >> 15;
        if (lane == 31) S.warp_uc[w] = iuc;
        __syncthreads();
        uint32_t bu = 0, bc = 0, total = 0;
#pragma unroll
        for (int ww = 0; ww < kDecWarps; ++ww) {
            const uint32_t uc = S.warp_uc[ww], cu = uc & 0x7fffu, cc = uc >> 15;
            if (ww < w) {
                bu += cu;
                bc += cc;
            }
            total += cc;
        }
        const uint32_t u0 = bu + iu - su + d0, u1 = u0 + d1;
        const uint32_t s0 = bc + ic - sc, s1 = s0 + c0;
        if (v0) {
            if (u0 >= idlimit || s0 >= (uint32_t)n_b) {
                bad = true;
            } else {
                uniq[k0] = (uint16_t)u0;
                atomicOr(&mask[s0 >> 5], 1u << (s0 & 31u));
            }
        }
        if (v1) {
            if (u1 >= idlimit || s1 >= (uint32_t)n_b) {
                bad = true;
            } else {
                uniq[k1] = (uint16_t)u1;
                atomicOr(&mask[s1 >> 5], 1u << (s1 & 31u));
            }
        }
        if (t == 0 && total != (uint32_t)n_b) bad = true;
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&s_bad, 1u);
    }
    __syncthreads();
    if (s_bad) {
        if (t == 0) set_status(a.status, kStCorrupt);
        return;
    }
    // every warp scans the 32 mask words itself (no further barrier): lane i
    // holds word i and the run starts before it; thread t's positions lie in
    // word t/8
    uint32_t mrow, prow;
    {
        const uint32_t mw = mask[lane];
        const uint32_t pc = __popc(mw);
        const uint32_t pre = warp_incl_sum(pc) - pc;
        const int src = (t >> 3) & 31;
        mrow = __shfl_sync(0xffffffffu, mw, src);
        prow = __shfl_sync(0xffffffffu, pre, src);
    }

    // ---- 4. positions 4t..4t+3 (with interleaved output every thread stays
    // for the barriers of the staging in record order)
    const int j0 = 4 * t;
    if (!AOS && j0 >= n_b) return;
    const bool act = j0 < n_b;
    float* recs = reinterpret_cast<float*>(stage);  // AOS, once the stage's words are consumed
    uint32_t key[4] = {0u, 0u, 0u, 0u};
    if (act) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t bit = (uint32_t)(j0 + e) & 31u;
            int run = (int)(prow + __popc(mrow & ((2u << bit) - 1u))) - 1;
            run = run < 0 ? 0 : (run >= (int)U ? (int)U - 1 : run);
            key[e] = uniq[run];
        }
    }
    if (!fast) {
        if (AOS) __syncthreads();  // the staged deltas and counts are consumed
        if (act)
            decode_wide<F, OUT64, AOS>(a, blk, hdr + dwords + cwords, rwords, W, S.G, j0, n_b, (uint64_t)b * kBlock,
                                       key[0], key[1], key[2], key[3], recs);
        if (AOS) store_records<F>(a, recs, b, n_b);
        return;
    }
    // records j0..j0+3 from the staged words; words past the record array
    // (inside the staging pad) hold bits above W, which are never consumed
    const bool wide = W > 64u;
    uint32_t rr[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t p = (uint32_t)((act ? j0 : 0) + e) * W;
        const uint32_t wi = p >> 5, sh = p & 31u;
        const uint32_t x0 = sR[wi], x1 = sR[wi + 1], x2 = sR[wi + 2];
        rr[e][0] = __funnelshift_r(x0, x1, sh);
        rr[e][1] = __funnelshift_r(x1, x2, sh);
        if (wide) {
            const uint32_t x3 = sR[wi + 3], x4 = sR[wi + 4];
            rr[e][2] = __funnelshift_r(x2, x3, sh);
            rr[e][3] = __funnelshift_r(x3, x4, sh);
        } else {
            rr[e][2] = rr[e][3] = 0u;
        }
    }
    const uint64_t first = (uint64_t)b * kBlock + j0;
    if (AOS) __syncthreads();  // every record is in registers: the stage takes the values
    if (act) {
        if (wide)
            decode_fields<F, true, OUT64, AOS>(a, rr, key, S, first, n_b - j0, recs, j0);
        else
            decode_fields<F, false, OUT64, AOS>(a, rr, key, S, first, n_b - j0, recs, j0);
    }
    if (AOS) store_records<F>(a, recs, b, n_b);
}


// AOS: out[0] receives interleaved records of F fields (Sh then a
// DecSharedRec<F>).  PREHW: lanes 0, 1, 2 of every warp pass in hw_pre the
// words round trip 1 would load (the payload size and the block's two table
// entries), loaded earlier by the caller.
template <int F, class Idx, bool OUT64 = false, bool AOS = false, class Sh = DecShared, bool PREHW = false>
__device__ __forceinline__ void decode_block(const DecArgs& a, Sh& S, Idx idx, uint32_t hw_pre = 0u) {
    uint32_t* stage = S.stage;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t* Sw = a.stream;
    const uint32_t b = idx.b();
    const int n_b = (int)((a.n - (uint64_t)b * kBlock) < (uint64_t)kBlock ? (a.n - (uint64_t)b * kBlock) : (uint64_t)kBlock);
    const uint64_t table_start = kHeaderWords + 2ull * F;
    const uint64_t payload_start = table_start + a.nblocks + 1;
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    if (t < 32) S.mask[t] = 0u;
    if (t == 0) S.bad = 0u;

    // ---- 1. where the block is (every warp, one round trip): the payload
    // size and the block's two table entries, checked only as far as staging
    // the block safely needs
    const bool header_fits = payload_start <= a.total_words;
    uint32_t hw = 0;
    if (PREHW)
        hw = header_fits && lane < 3 ? hw_pre : 0u;
    else if (header_fits && lane < 3)
        hw = __ldg(lane == 0 ? Sw + 9 : Sw + table_start + b + (uint32_t)(lane - 1));
    const uint32_t payload_words = __shfl_sync(0xffffffffu, hw, 0);
    const uint32_t off = __shfl_sync(0xffffffffu, hw, 1);
    const uint32_t end = __shfl_sync(0xffffffffu, hw, 2);
    const bool inside =
        header_fits && payload_start + payload_words <= a.total_words && off <= end && end <= payload_words;
    const uint32_t* blk = Sw + payload_start + off;
    const uint32_t nw = end - off;
    // round trip 2: warp 0 fetches the stream header, the block header and the
    // steps (all in bounds once the block is inside the stream), and the
    // block's words after its header are staged in shared memory (all of them
    // when they fit; the deltas and counts always fit) by one bulk copy that
    // thread 0 issues, its last few words by plain loads where the copy's
    // 16-byte units would reach past the stream
    uint32_t hv = 0, bw = 0;
    float step = 0.0f;
    if (w == 0) {
        if (lane < kHeaderWords) hv = __ldg(Sw + lane);  // the host checked total_words >= kHeaderWords
        if (inside && (uint32_t)lane < min(hdr, nw)) bw = __ldg(blk + lane);
        if (header_fits && lane < F) step = __uint_as_float(__ldg(Sw + kHeaderWords + 2 * lane + 1));
    }
    // the copy: 16-byte units from the boundary at or below the first word,
    // as many as end inside the stream; the words after them by plain loads
    const uint32_t* src = blk + hdr;
    const uint32_t shift = (uint32_t)((reinterpret_cast<uintptr_t>(src) >> 2) & 3u);
    uint32_t nst = 0, units = 0;
    if (inside && nw > hdr) {
        nst = min(nw - hdr, kDecStageWords);
        const uint64_t avail = a.total_words - (uint64_t)(src - Sw) + shift;  // words from the boundary to the stream's end
        units = (uint32_t)(min((uint64_t)(nst + shift + 3u), avail) >> 2);
        if (units * 4u < shift) units = 0;
    }
    if (units && t == 0) {
        mbar_init(&S.bar, 1);
        mbar_arrive_expect_tx(&S.bar, units * 16u);
        bulk_g2s(S.stage, src - shift, units * 16u, &S.bar);
    }
    const uint32_t kb = units ? units * 4u - shift : 0u;  // first word not in the copy
    for (uint32_t k = kb + t; k < nst; k += kDecThreads) stage[shift + k] = __ldg(src + k);

    if (w == 0) decode_checks<F>(a, S, hv, bw, step, inside, b, off, end, payload_words, n_b);
    __syncthreads();
    if (units && !__syncthreads_and(mbar_wait_bounded(&S.bar, 0, a.status))) return;  // uniform
    decode_tail<F, OUT64, AOS>(a, S, stage + shift, blk, b, n_b);
}

}  // namespace gpz
