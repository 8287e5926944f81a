// gpz_qse_block.cuh -- the per-block body of the fused compression kernel
// (quantisation, sorting, encoding; Sections 4.1-4.3), shared by the
// single-array kernels (gpz_qse.cu) and the batched kernels
// (gpz_batch_compress.cu).  See gpz_qse.cu for the design.
#pragma once

#include "gpz_internal.cuh"

namespace gpz {

// ------------------------------------------------------------------ fused Q.S.E. kernel

constexpr int kThreads = kQseThreads;        // 256
constexpr int kWarps = kThreads / 32;        // 8
constexpr uint32_t kHistBytes = kWarps * kMaxBins * 2u;  // u16 per-warp histograms
constexpr uint32_t kMagic23 = 0x4B000000u;   // bit pattern of 2^23

__host__ __device__ constexpr uint32_t qse_region_bytes(int F) {
    const uint32_t rec = kHistBytes + kBlock * 16u;         // histograms + 128-bit sorted records
    const uint32_t codes = (uint32_t)F * kBlock * 4u;        // u32 sorted codes per field (W > 128)
    return rec > codes ? rec : codes;
}

// The whole encoded block of the packed path: header (<= 11 words), deltas
// (<= 512 x 9 bits), counts (<= 512 x 11 bits), records (<= 1024 x 128 bits).
constexpr uint32_t kStageWords = 4432u;
constexpr uint32_t kFastRecordBits = 128u;

__host__ __device__ constexpr uint32_t qse_smem_bytes(int F) {
    return qse_region_bytes(F) + kMaxBins * 2u /*uniq*/ + kMaxBins * 2u /*counts*/ + kBlock * 2u /*perm*/ +
           kStageWords * 4u /*packed records*/;
}

struct QseShared {
    uint32_t minkey[kMaxFields];
    uint32_t maxq[kMaxFields];
    uint32_t flags;                 // bit 0: non-finite value, bit 1: no code within the bound
    uint32_t maxcnt, maxdelta;
    uint32_t warp_tot[kWarps], warp_nz[kWarps];
};

// Where the fast path gets its block's index: the grid (one CTA per block),
// or a shared-memory slot (the batched kernel's block within its chunk)
// re-read at each use, so that the index holds no register through the
// block code.
struct GridBlock {
    __device__ __forceinline__ uint32_t b() const { return blockIdx.x; }   // block within its array
    __device__ __forceinline__ uint32_t id() const { return blockIdx.x; }  // entry for the general list
};
struct SlotBlock {
    const volatile uint32_t* slot;  // [0]: block within its array, [1]: entry for the general list
    __device__ __forceinline__ uint32_t b() const { return slot[0]; }
    __device__ __forceinline__ uint32_t id() const { return slot[1]; }
};

// Order-preserving map of finite floats to u32 (-0 < +0).
__device__ __forceinline__ uint32_t order_key(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_order_key(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Verification of one candidate code: the decompressor's reconstruction.
__device__ __forceinline__ bool code_ok(float x, uint32_t q, const FieldParams& p, float mn) {
    const float xh = __fmaf_rn(__uint2float_rn(q), p.s, mn);
    return fabsf(__fsub_rn(x, xh)) <= p.ebchk;
}

// General quantiser (codes >= 2^23, or a first candidate that fails):
// candidates q0, q0 - 1, q0 + 1; returns 0xffffffff when none is within the
// bound (valid codes are below 2^31).
static __device__ __noinline__ uint32_t quantise_general(float x, FieldParams p, float mn) {
    const float t = __fmaf_rn(__fsub_rn(x, mn), p.inv, 0.5f);
    if (!(t < 2147483648.0f)) return 0xffffffffu;
    const uint32_t q = __float2uint_rd(t);
    if (code_ok(x, q, p, mn)) return q;
    if (q > 0u && code_ok(x, q - 1u, p, mn)) return q - 1u;
    if (code_ok(x, q + 1u, p, mn)) return q + 1u;
    return 0xffffffffu;
}


// Thread-serial fixed-length appender into zeroed shared words: appends the
// low w (<= 32) bits of v at the current bit position.  Every completed word
// is merged with atomicOr (a word at the edge of a thread's range is shared
// with its neighbour); the updates are predicated, so the warp never diverges.
struct BitAppender {
    unsigned long long acc;
    uint32_t nb;   // bits pending in acc (< 32)
    uint32_t wi;   // shared word index of acc's low word
    __device__ __forceinline__ BitAppender(uint32_t bitpos) : acc(0ull), nb(bitpos & 31u), wi(bitpos >> 5) {}
    __device__ __forceinline__ void put(uint32_t* sw, uint32_t v, uint32_t w) {
        acc |= (unsigned long long)v << nb;
        nb += w;
        const bool full = nb >= 32u;
        if (full) atomicOr(sw + wi, (uint32_t)acc);
        acc = full ? (acc >> 32) : acc;
        nb = full ? nb - 32u : nb;
        wi += full ? 1u : 0u;
    }
    __device__ __forceinline__ void finish(uint32_t* sw) {
        if (nb) atomicOr(sw + wi, (uint32_t)acc);
    }
};

template <int F>
__device__ __forceinline__ void write_raw(const QseArgs& a, uint32_t b, int n_b, int t) {
    const uint64_t first = (uint64_t)b * kBlock;
    uint32_t* out = a.temp + (size_t)b * a.slot_words;
    if (t == 0) out[0] = 1u;
    if (a.interleaved) {  // value k of the block's records is field k % F of particle k / F
        const float* src = a.fields[0] + first * F;
        for (int k = t; k < F * n_b; k += kThreads) {
            const int i = k / F, f = k - i * F;
            out[1 + f * n_b + i] = __float_as_uint(__ldg(src + k));
        }
    } else {
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const float* src = a.fields[f] + first;
            for (int i = t; i < n_b; i += kThreads) out[1 + f * n_b + i] = __float_as_uint(__ldg(src + i));
        }
    }
    if (a.perm)
        for (int i = t; i < n_b; i += kThreads) a.perm[first + i] = (uint32_t)(first + i);
    if (t == 0) a.sizes[b] = 1u + (uint32_t)F * (uint32_t)n_b;
}

// The general per-block path: any block, including codes >= 2^23, values
// that need a fallback candidate, and records wider than 128 bits.
template <int F, bool FULL>
__device__ __forceinline__ void qse_block_general(const QseArgs& a, uint8_t* dsm, QseShared& S, uint32_t b) {
    constexpr int P = F < 3 ? F : 3;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = FULL ? kBlock : (int)(a.n - first);
    constexpr uint32_t region = qse_region_bytes(F);
    uint16_t* hist = reinterpret_cast<uint16_t*>(dsm);                     // [8][512]
    uint4* recs = reinterpret_cast<uint4*>(dsm + kHistBytes);               // [1024] 128-bit records
    uint32_t* codes = reinterpret_cast<uint32_t*>(dsm);                      // [F][1024], wide records
    uint16_t* uniq = reinterpret_cast<uint16_t*>(dsm + region);             // [512]
    uint16_t* cnt = uniq + kMaxBins;                                         // [512]
    uint16_t* sperm = cnt + kMaxBins;                                        // [1024]
    uint32_t* stage = reinterpret_cast<uint32_t*>(sperm + kBlock);           // [kStageWords]
    uint32_t* out = a.temp + (size_t)b * a.slot_words;

    if (t < F) {
        S.minkey[t] = 0xffffffffu;
        S.maxq[t] = 0u;
    }
    if (t == 0) {
        S.flags = 0u;
        S.maxcnt = 0u;
        S.maxdelta = 0u;
    }
    {
        uint32_t* h32 = reinterpret_cast<uint32_t*>(hist + w * kMaxBins);
#pragma unroll
        for (int k = 0; k < kMaxBins / 64; ++k) h32[lane + 32 * k] = 0u;
        for (uint32_t k = t; k < kStageWords; k += kThreads) stage[k] = 0u;
    }

    // ---- 1. load (coalesced, streaming) and block minimum
    bool valid[4];
    float x[F][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) valid[r] = FULL || (128 * w + 32 * r + lane < n_b);
#pragma unroll
    for (int f = 0; f < F; ++f) {
        // separate fields, or interleaved records (stride F)
        const uint64_t stride = a.interleaved ? (uint64_t)F : 1u;
        const float* src = a.interleaved ? a.fields[0] + (first + 128 * w + lane) * F + f
                                         : a.fields[f] + first + 128 * w + lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) x[f][r] = valid[r] ? __ldcs(src + 32 * r * stride) : 0.0f;
    }
    FieldParams prm[F];
#pragma unroll
    for (int f = 0; f < F; ++f) prm[f] = a.d_params ? a.d_params[f] : a.params[f];
    __syncthreads();  // shared reduction slots initialised (the loads are in flight)
    float probe = 0.0f;  // becomes NaN if any value is NaN or infinite (x * 0)
#pragma unroll
    for (int f = 0; f < F; ++f) {
        float m = valid[0] ? x[f][0] : INFINITY;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (valid[r]) {
                probe = __fmaf_rn(x[f][r], 0.0f, probe);
                m = fminf(m, x[f][r]);
            }
        }
        const uint32_t mk = __reduce_min_sync(0xffffffffu, m == INFINITY ? 0xffffffffu : order_key(m));
        if (lane == 0) atomicMin(&S.minkey[f], mk);
    }
    if (__any_sync(0xffffffffu, probe != probe) && lane == 0) atomicOr(&S.flags, 1u);
    __syncthreads();  // A
    if (S.flags & 1u) {
        write_raw<F>(a, b, n_b, t);
        return;
    }

    // ---- 2. quantisation with verification (fast path for codes < 2^23)
    float mn[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const float m = from_order_key(S.minkey[f]);
        mn[f] = m == 0.0f ? 0.0f : m;  // a zero minimum is stored as +0
    }
    uint32_t q[F][4];
    uint32_t pending = 0;  // bit 4f + r: value needs the general quantiser
#pragma unroll
    for (int f = 0; f < F; ++f) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float xv = x[f][r];
            const float tt = __fmaf_rn(__fsub_rn(xv, mn[f]), prm[f].inv, 0.5f);
            // 2^23 + floor(t), exactly, while t < 2^23 (the sum lies in [2^23, 2^24))
            const float u = __fadd_rd(tt, 8388608.0f);
            q[f][r] = __float_as_uint(u) - kMagic23;
            const float xh = __fmaf_rn(__fsub_rn(u, 8388608.0f), prm[f].s, mn[f]);
            const bool ok = (tt < 8388608.0f) && (fabsf(__fsub_rn(xv, xh)) <= prm[f].ebchk);
            if (valid[r] && !ok) pending |= 1u << (4 * f + r);
            if (!valid[r]) q[f][r] = 0u;
        }
    }
    bool fail = false;
    if (__any_sync(0xffffffffu, pending != 0u)) {
#pragma unroll
        for (int f = 0; f < F; ++f) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (pending & (1u << (4 * f + r))) {
                    const uint32_t g = quantise_general(x[f][r], prm[f], mn[f]);
                    fail |= g == 0xffffffffu;
                    q[f][r] = g == 0xffffffffu ? 0u : g;
                }
            }
        }
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
        uint32_t qmax = max(max(q[f][0], q[f][1]), max(q[f][2], q[f][3]));
        qmax = __reduce_max_sync(0xffffffffu, qmax);
        if (lane == 0 && qmax) atomicMax(&S.maxq[f], qmax);
    }
    if (__any_sync(0xffffffffu, fail) && lane == 0) atomicOr(&S.flags, 2u);
    __syncthreads();  // B
    if (S.flags & 2u) {
        write_raw<F>(a, b, n_b, t);
        return;
    }

    // ---- 3. segments, key and record layout (uniform)
    uint32_t o[F], wf[F], kshift[F], bits[F], keybits = 0, W = 0;
    {
        uint32_t g[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            bits[f] = bit_width(S.maxq[f]);
            g[f] = f < P ? min((uint32_t)a.G, bits[f]) : 0u;
            o[f] = f < P ? bits[f] - g[f] : 0u;
            wf[f] = f < P ? o[f] : bits[f];
        }
        uint32_t ks = 0;
#pragma unroll
        for (int f = F - 1; f >= 0; --f) {
            kshift[f] = ks;
            ks += g[f];
            W += wf[f];
        }
        keybits = ks;
    }
    const bool fast = W <= kFastRecordBits;
    // records as four words r0 (least significant) .. r3; each field's code is
    // appended below the record so far, so field 0 ends most significant
    uint32_t key[4], r0[4], r1[4], r2[4], r3[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        uint32_t k = 0;
#pragma unroll
        for (int f = 0; f < P; ++f) k |= (q[f][r] >> o[f]) << kshift[f];
        key[r] = k;
        r0[r] = r1[r] = r2[r] = r3[r] = 0u;
    }
    if (W <= 64u) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const uint32_t code = f < P ? (q[f][r] & ((1u << o[f]) - 1u)) : q[f][r];
                hi = __funnelshift_l(lo, hi, wf[f]);
                lo = (lo << wf[f]) | code;
            }
            r0[r] = lo;
            r1[r] = hi;
        }
    } else if (fast) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const uint32_t code = f < P ? (q[f][r] & ((1u << o[f]) - 1u)) : q[f][r];
                a3 = __funnelshift_l(a2, a3, wf[f]);
                a2 = __funnelshift_l(a1, a2, wf[f]);
                a1 = __funnelshift_l(a0, a1, wf[f]);
                a0 = (a0 << wf[f]) | code;
            }
            r0[r] = a0;
            r1[r] = a1;
            r2[r] = a2;
            r3[r] = a3;
        }
    }

    // ---- 4. stable counting sort: warp-local ranks in storage order
    uint16_t* myhist = hist + w * kMaxBins;
    uint32_t rank[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t peers = __match_any_sync(0xffffffffu, valid[r] ? key[r] : 0xffffffffu);
        uint32_t before = 0u;
        if (valid[r]) before = myhist[key[r]];
        __syncwarp();
        if (valid[r] && lane == 31 - __clz(peers)) myhist[key[r]] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rank[r] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();  // C

    // ---- 4b. scan over (bin, warp): sorted positions and the run-length code
    const int nbins = 1 << keybits;
    const int b0 = 2 * t;
    uint32_t c0 = 0, c1 = 0;
    uint32_t pre[kWarps];  // (prefix of bin b0) | (prefix of bin b0+1) << 16
    if (b0 < nbins) {
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t pair = *reinterpret_cast<const uint32_t*>(hist + ww * kMaxBins + b0);
            pre[ww] = c0 | (c1 << 16);
            c0 += pair & 0xffffu;
            c1 += pair >> 16;
        }
    }
    const uint32_t tot = c0 + c1;
    const uint32_t nz = (c0 ? 1u : 0u) + (c1 ? 1u : 0u);
    const uint32_t incl_tot = warp_incl_sum(tot);
    const uint32_t incl_nz = warp_incl_sum(nz);
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, max(c0, c1));
    if (lane == 31) {
        S.warp_tot[w] = incl_tot;
        S.warp_nz[w] = incl_nz;
    }
    if (lane == 0) atomicMax(&S.maxcnt, cmax);
    __syncthreads();  // D
    uint32_t base_tot = 0, base_nz = 0, U = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t vt = S.warp_tot[ww], vn = S.warp_nz[ww];
        if (ww < w) {
            base_tot += vt;
            base_nz += vn;
        }
        U += vn;
    }
    if (b0 < nbins) {
        const uint32_t start0 = base_tot + incl_tot - tot, start1 = start0 + c0;
        const uint32_t idx0 = base_nz + incl_nz - nz, idx1 = idx0 + (c0 ? 1u : 0u);
        const uint32_t base2 = start0 | (start1 << 16);  // neither half overflows: both < 1024
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww)
            *reinterpret_cast<uint32_t*>(hist + ww * kMaxBins + b0) = base2 + pre[ww];
        if (c0) {
            uniq[idx0] = (uint16_t)b0;
            cnt[idx0] = (uint16_t)c0;
        }
        if (c1) {
            uniq[idx1] = (uint16_t)(b0 + 1);
            cnt[idx1] = (uint16_t)c1;
        }
    }
    __syncthreads();  // E

    // ---- 4c. scatter to sorted order; deltas of the unique ids
    uint32_t dest[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) dest[r] = valid[r] ? myhist[key[r]] + rank[r] : 0u;
    {
        uint32_t dmax = 0;
        for (uint32_t k = t; k < U; k += kThreads) {
            const uint32_t d = (uint32_t)uniq[k] - (k ? (uint32_t)uniq[k - 1] : 0u);
            dmax = max(dmax, d);
        }
        dmax = __reduce_max_sync(0xffffffffu, dmax);
        if (lane == 0 && dmax) atomicMax(&S.maxdelta, dmax);
    }
    if (fast) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (valid[r]) recs[dest[r]] = make_uint4(r0[r], r1[r], r2[r], r3[r]);
    }
    if (a.perm) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (valid[r]) sperm[dest[r]] = (uint16_t)(128 * w + 32 * r + lane);
    }
    if (!fast) {
        __syncthreads();  // the histograms are read; the codes may overwrite them
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (!valid[r]) continue;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const uint32_t qq = q[f][r];
                codes[f * kBlock + dest[r]] = f < P ? (qq & ((1u << o[f]) - 1u)) : qq;
            }
        }
    }
    __syncthreads();  // F

    // ---- encoded size; raw when not smaller (keeps the bound size a bound)
    const uint32_t wd = bit_width(S.maxdelta), wc = bit_width(S.maxcnt);
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = ceil_words((uint32_t)n_b * W);
    const uint32_t enc = hdr + dwords + cwords + rwords;
    if (enc >= 1u + (uint32_t)F * (uint32_t)n_b) {
        write_raw<F>(a, b, n_b, t);
        return;
    }

    // ---- 5. block header and the three arrays (Section 4.3), assembled in the
    // zeroed staging words by thread-serial appenders, then copied out
    if (t == 0) stage[0] = (U << 1) | (wd << 12) | (wc << 17);
    if (t >= 1 && t <= F) {
        float m = 0.0f;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if (f == t - 1) m = mn[f];
        stage[t] = __float_as_uint(m);
    }
    if (t < ((F + 3) >> 2)) {
        uint32_t word = 0;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if ((f >> 2) == t) word |= bits[f] << (8 * (f & 3));
        stage[1 + F + t] = word;
    }
    {
        // deltas and counts: entries 2t, 2t+1
        const uint32_t k0 = 2u * (uint32_t)t;
        if (k0 < U && wd) {
            BitAppender ap(32u * hdr + k0 * wd);
            ap.put(stage, (uint32_t)uniq[k0] - (k0 ? (uint32_t)uniq[k0 - 1] : 0u), wd);
            if (k0 + 1 < U) ap.put(stage, (uint32_t)uniq[k0 + 1] - (uint32_t)uniq[k0], wd);
            ap.finish(stage);
        }
        if (k0 < U && wc) {
            BitAppender ap(32u * (hdr + dwords) + k0 * wc);
            ap.put(stage, (uint32_t)cnt[k0], wc);
            if (k0 + 1 < U) ap.put(stage, (uint32_t)cnt[k0 + 1], wc);
            ap.finish(stage);
        }
    }
    const uint32_t len = (uint32_t)n_b;
    const uint32_t rbase = hdr + dwords + cwords;
    if (fast) {
        // Thread t appends sorted records 4t..4t+3 (bits [4tW, 4tW + 4W)).
        const uint32_t j0 = 4u * (uint32_t)t;
        if (j0 < len && W) {
            BitAppender ap(32u * rbase + j0 * W);
            // widths of the record's four words
            const uint32_t w0 = min(W, 32u), w1 = min(W - w0, 32u), w2 = min(W - w0 - w1, 32u), w3 = W - w0 - w1 - w2;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint4 v = (j0 + e < len) ? recs[j0 + e] : make_uint4(0u, 0u, 0u, 0u);
                ap.put(stage, v.x, w0);
                if (w1) ap.put(stage, v.y, w1);
                if (w2) ap.put(stage, v.z, w2);
                if (w3) ap.put(stage, v.w, w3);
            }
            ap.finish(stage);
        }
    }
    __syncthreads();
    {
        // copy the staged words (all of them, or up to the records when the
        // records are wider than 64 bits); the slot is 16-byte aligned
        const uint32_t nstage = fast ? enc : rbase;
        const uint4* s4 = reinterpret_cast<const uint4*>(stage);
        uint4* o4 = reinterpret_cast<uint4*>(out);
        for (uint32_t k = t; k < (nstage >> 2); k += kThreads) o4[k] = s4[k];
        for (uint32_t k = (nstage & ~3u) + t; k < nstage; k += kThreads) out[k] = stage[k];
    }
    if (!fast) {
        // records wider than 128 bits: gather field by field from the codes
        uint32_t* rout = out + rbase;
        uint32_t rshift[F];
        {
            uint32_t rs = 0;
#pragma unroll
            for (int f = F - 1; f >= 0; --f) {
                rshift[f] = rs;
                rs += wf[f];
            }
        }
        for (uint32_t k = t; k < rwords; k += kThreads) {
            const uint32_t lo = 32u * k;
            uint32_t j = div_small(lo, W);
            uint32_t acc = 0;
            for (; j < len && j * W < lo + 32u; ++j) {
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    if (wf[f] == 0u) continue;
                    const int s0 = (int)(j * W + rshift[f]) - (int)lo;
                    if (s0 >= 32 || s0 + (int)wf[f] <= 0) continue;
                    const uint32_t v = codes[f * kBlock + j];
                    acc |= s0 >= 0 ? (v << s0) : (v >> -s0);
                }
            }
            rout[k] = acc;
        }
    }
    if (a.perm)
        for (int j = t; j < n_b; j += kThreads) a.perm[first + j] = (uint32_t)first + sperm[j];
    if (t == 0) a.sizes[b] = enc;
}

// ------------------------------------------------------------------ fast path

// Fast-path shared memory: the 128-bit sorted records, the unique ids and
// counts, the sorted permutation, and the staging words of the encoded block,
// whose first 8 KB hold the per-warp histograms until the scatter is done.
constexpr uint32_t kFastHist = 0u;
constexpr uint32_t kFastUniq = kFastHist + kHistBytes;
constexpr uint32_t kFastStage = kFastUniq + kMaxBins * 2u + kMaxBins * 2u + kBlock * 2u;
static_assert(kFastStage % 16u == 0u && kStageWords % 4u == 0u, "the staging words are cleared 16 bytes at a time");

__host__ __device__ constexpr uint32_t qse_fast_smem_bytes() { return kFastStage + kStageWords * 4u; }

struct QseFastShared {
    uint32_t minkey[kMaxFields];
    uint32_t maxkey[kMaxFields];
    uint32_t flags;                 // bit 0: non-finite value, bit 1: a value needs a fallback candidate
    uint32_t maxcnt, maxdelta;
    uint32_t warp_tot[kWarps];      // per warp: count sum | non-empty bins << 16
    uint32_t warp_last[kWarps];
    uint32_t offset;                // fused compaction: the block's offset in the payload, or kNotPlaced
};

// ---- fused compaction (an alternative to Section 4.4's three steps):
// every block publishes its size as soon as it is known, then looks back
// over its predecessors' published sizes (a decoupled look-back over
// blocks).  A block that finds its exclusive prefix writes itself into the
// stream at once; the scan and copy kernels that follow then only fill the
// offset table and move the other blocks.  A block left to the general path
// has no size yet and breaks the chain, as does a predecessor that has not
// published within the wait bound: the blocks behind it go to their
// temporary slots as in the three-step form.
constexpr unsigned long long kBlkAgg = 1ull << 62;     // size published, prefix not known
constexpr unsigned long long kBlkIncl = 2ull << 62;    // inclusive prefix published
constexpr unsigned long long kBlkBroken = 3ull << 62;  // no prefix will follow
constexpr uint32_t kNotPlaced = 0xffffffffu;
constexpr long long kLookbackCycles = 1ll << 17;       // about 60 us


// Exclusive prefix of the sizes of blocks 0..b-1 (every lane of one warp),
// or kNotPlaced when the chain is broken: a predecessor left to the general
// path, or one that has not published within `limit` SM cycles (0:
// kLookbackCycles).  Giving up is not an error: the block then goes through
// its temporary slot and the copy kernel.
static __device__ __noinline__ uint32_t block_lookback(const unsigned long long* bstate, uint32_t b,
                                                       long long limit = 0) {
    if (limit <= 0) limit = kLookbackCycles;
    const int lane = threadIdx.x & 31;
    uint32_t excl = 0;
    for (int base = (int)b - 1;; base -= 32) {
        const int j = base - lane;
        unsigned long long st = kBlkIncl;  // before block 0: prefix 0
        if (j >= 0) {
            const long long t0 = clock64();
            for (;;) {
                st = ld_relaxed_u64(bstate + j);
                if (st >> 62) break;
                if (clock64() - t0 > limit) {
                    st = kBlkBroken;
                    break;
                }
                __nanosleep(32);
            }
        }
        const uint32_t flag = (uint32_t)(st >> 62);
        const uint32_t stop = __ballot_sync(0xffffffffu, flag >= 2u);
        if (stop) {  // the nearest predecessor with a prefix, or a break
            const int first = __ffs(stop) - 1;
            if (__shfl_sync(0xffffffffu, flag, first) == 3u) return kNotPlaced;
            return excl + __reduce_add_sync(0xffffffffu, lane <= first ? (uint32_t)st : 0u);
        }
        excl += __reduce_add_sync(0xffffffffu, (uint32_t)st);
    }
}

// A block stored raw (its words go to the temporary slot).  With fused
// compaction it publishes its size and then, so that the blocks behind it
// need not walk past it, its inclusive prefix (warp 0).
template <int F, int CM>
__device__ __forceinline__ void raw_block(const QseArgs& a, uint32_t b, int n_b, int t) {
    constexpr bool DIRECT = CM == kCmDirect;
    const uint32_t raw_words = 1u + (uint32_t)F * (uint32_t)n_b;
    if (DIRECT && t == 0) st_release_u64(a.bstate + b, (b == 0 ? kBlkIncl : kBlkAgg) | raw_words);
    write_raw<F>(a, b, n_b, t);
    if (DIRECT && b != 0 && (t >> 5) == 0) {
        const uint32_t off = block_lookback(a.bstate, b);
        if (t == 0) st_release_u64(a.bstate + b, off == kNotPlaced ? kBlkBroken : (kBlkIncl | (off + raw_words)));
    }
}

// Whether every first candidate of a field's block is certain to pass the
// verification |RN(x - RN(fma(q, s, min)))| <= ebchk, so that it need not be
// computed.  With Q the largest code (< 2^k) and M the largest |x| of the
// block, the rounding of d = RN(x - min), of t = RN(fma(d, 1/s, 1/2)) (t <
// 2^(k+1)), of 1/s and of the reconstruction add up to at most
// s 2^(k-23) + 3.0001 ulp(M) + 2 ulp(s) beyond the half step s/2 <= eb 63/64,
// and the check passes whenever the total stays below eb (1 - 2^-20).  For
// k <= 15 and ulp(M) <= eb/512 the total is at most 0.0136 eb + s/2, inside
// the 1/64 margin (about 13% to spare).
__device__ __forceinline__ bool first_candidate_exact(uint32_t bits, float mn, float mx, float eb) {
    const float M = fmaxf(fabsf(mn), fabsf(mx));
    const float ulp = fmaxf(__uint_as_float(__float_as_uint(M) & 0x7f800000u) * 1.1920928955078125e-7f,
                            1.40129846e-45f);  // 2^(exponent - 23), at least the smallest subnormal
    return bits <= 15u && __fmul_rn(ulp, 512.0f) <= eb;
}

// Quantise the thread's 4 values of field f (first candidate only), add the
// field's segId to the key and append its code to the record words.  With
// VERIFY the candidate is checked as the format requires and `pend` is set
// when one fails; without, the caller has shown that none can fail
// (first_candidate_exact).
template <int NW, bool VERIFY>
__device__ __forceinline__ void quantise_append(const float (&x)[4], const bool (&valid)[4], float mn,
                                                const FieldParams& p, bool pos, uint32_t o, uint32_t ks,
                                                uint32_t wf, uint32_t (&key)[4], uint32_t (&rw)[4][4],
                                                bool& pend) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float tt = __fmaf_rn(__fsub_rn(x[r], mn), p.inv, 0.5f);
        const float u = __fadd_rd(tt, 8388608.0f);  // 2^23 + floor(t), t < 2^23 here
        uint32_t q = __float_as_uint(u) - kMagic23;
        if (VERIFY) {
            const float xh = __fmaf_rn(__fsub_rn(u, 8388608.0f), p.s, mn);
            pend |= valid[r] && !(fabsf(__fsub_rn(x[r], xh)) <= p.ebchk);
        }
        q = valid[r] ? q : 0u;
        uint32_t code = q;
        if (pos) {
            key[r] |= (q >> o) << ks;
            code = q & ((1u << o) - 1u);
        }
        // append below the record so far (field 0 ends most significant)
        if (NW == 4) {
            rw[r][3] = __funnelshift_l(rw[r][2], rw[r][3], wf);
            rw[r][2] = __funnelshift_l(rw[r][1], rw[r][2], wf);
        }
        rw[r][1] = __funnelshift_l(rw[r][0], rw[r][1], wf);
        rw[r][0] = (rw[r][0] << wf) | code;
    }
}

// Block b of the array described by a; a block the fast path cannot take is
// appended to a.general_list as list_id.
// The code width of one field of a block from its extremes (step 2 of the
// fused kernel): q0 = floor(fma(x - min, 1/s, 1/2)) is monotone in x, so when
// every value keeps its first candidate the largest code is q0 of the block
// maximum.  big: that code reaches 2^23; exact: no first candidate of the
// field can fail its check (first_candidate_exact).
__device__ __forceinline__ void block_field_width(uint32_t kmin, uint32_t kmax, const FieldParams& p, uint32_t& bits,
                                                  bool& big, bool& exact) {
    const float m0 = from_order_key(kmin);
    const float m = m0 == 0.0f ? 0.0f : m0;  // a zero minimum is stored as +0
    const float mx = from_order_key(kmax);
    const float tq = __fmaf_rn(__fsub_rn(mx, m), p.inv, 0.5f);
    big = !(tq < 8388608.0f);
    bits = bit_width(__float_as_uint(__fadd_rd(tq, 8388608.0f)) - kMagic23);
    exact = first_candidate_exact(bits, m, mx, p.eb);
}

// A block's widths and flags, precomputed once per block after the range
// pass (gpz_block_info_kernel): the width of field f in bits 5f..5f+4, and:
constexpr int kInfoBig = 61;      // some field's largest code reaches 2^23
constexpr int kInfoExact = 62;    // no first candidate of the block can fail its check

// PRE: the range pass has already found each block's extremes (a.bext);
// otherwise the block finds them itself.
template <int F, bool FULL, class Idx, int CM = kCmTemp, bool PRE = false>
__device__ __forceinline__ void qse_block_fast(const QseArgs& a, uint8_t* dsm, QseFastShared& S, Idx idx) {
    constexpr int P = F < 3 ? F : 3;
    constexpr bool DIRECT = CM == kCmDirect;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int n_b = FULL ? kBlock : (int)(a.n - (uint64_t)idx.b() * kBlock);
    uint16_t* hist = reinterpret_cast<uint16_t*>(dsm + kFastHist);          // [8][512] per-warp histograms
    uint16_t* uniq = reinterpret_cast<uint16_t*>(dsm + kFastUniq);          // [512]
    uint16_t* cnt = uniq + kMaxBins;                                         // [512]
    uint16_t* sperm = cnt + kMaxBins;                                        // [1024]
    uint32_t* stage = reinterpret_cast<uint32_t*>(dsm + kFastStage);        // [kStageWords] the encoded block

    if (!PRE && t < F) {
        S.minkey[t] = 0xffffffffu;
        S.maxkey[t] = 0u;
    }
    if (t == 0) {
        S.flags = 0u;
        S.maxcnt = 0u;
        S.maxdelta = 0u;
    }
    {
        uint32_t* h32 = reinterpret_cast<uint32_t*>(hist + w * kMaxBins);
#pragma unroll
        for (int k = 0; k < kMaxBins / 64; ++k) h32[lane + 32 * k] = 0u;
        // the encoded block is assembled by OR into cleared words
        uint4* s4 = reinterpret_cast<uint4*>(stage);
        for (uint32_t k = t; k < kStageWords / 4u; k += kThreads) s4[k] = make_uint4(0u, 0u, 0u, 0u);
    }

    // ---- 1. load (coalesced, streaming); block minimum and maximum
    bool valid[4];
    float x[F][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) valid[r] = FULL || (128 * w + 32 * r + lane < n_b);
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const float* src = a.fields[f] + (uint64_t)idx.b() * kBlock + 128 * w + lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) x[f][r] = valid[r] ? __ldcs(src + 32 * r) : 0.0f;
    }
    uint32_t kmin[F], kmax[F];  // the block's extremes, as order keys
    unsigned long long info = 0ull;  // the block's widths and flags, when precomputed (a.binfo)
    if constexpr (PRE) {  // from the range pass; (0, 0) marks a non-finite value
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const uint2 e = __ldg(a.bext + (size_t)idx.b() * F + f);
            kmin[f] = e.x;
            kmax[f] = e.y;
        }
        if (a.binfo) info = __ldg(a.binfo + idx.b());
        __syncthreads();  // shared counters initialised (the loads are in flight)
        bool nonfinite = false;
#pragma unroll
        for (int f = 0; f < F; ++f) nonfinite |= kmin[f] == 0u;
        if (nonfinite) {  // uniform: every thread read the same extremes
            raw_block<F, CM>(a, idx.b(), n_b, t);
            return;
        }
    } else {
        __syncthreads();  // shared reduction slots initialised (the loads are in flight)
        float probe = 0.0f;  // becomes NaN if any value is NaN or infinite (x * 0)
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float lo = INFINITY, hi = -INFINITY;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (valid[r]) {
                    probe = __fmaf_rn(x[f][r], 0.0f, probe);
                    lo = fminf(lo, x[f][r]);
                    hi = fmaxf(hi, x[f][r]);
                }
            }
            const uint32_t lk = __reduce_min_sync(0xffffffffu, lo == INFINITY ? 0xffffffffu : order_key(lo));
            const uint32_t hk = __reduce_max_sync(0xffffffffu, hi == -INFINITY ? 0u : order_key(hi));
            if (lane == 0) {
                atomicMin(&S.minkey[f], lk);
                atomicMax(&S.maxkey[f], hk);
            }
        }
        if (__any_sync(0xffffffffu, probe != probe) && lane == 0) atomicOr(&S.flags, 1u);
        __syncthreads();  // A
        if (S.flags & 1u) {
            raw_block<F, CM>(a, idx.b(), n_b, t);
            return;
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            kmin[f] = S.minkey[f];
            kmax[f] = S.maxkey[f];
        }
    }

    // ---- 2. widths from the block maxima: q0 = floor(fma(x - min, 1/s, 1/2))
    // is monotone in x, so when every value keeps its first candidate the
    // largest code is q0 of the block maximum
    float mn[F];
    uint32_t bits[F], o[F], wf[F], kshift[F], W = 0, keybits = 0;
    bool big = false, exact = true;
    {
        uint32_t g[F];
        const bool have_info = PRE && a.binfo != nullptr;  // uniform
        if (have_info) {
            big = (info >> kInfoBig) & 1ull;
            exact = (info >> kInfoExact) & 1ull;
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const float m = from_order_key(kmin[f]);
            mn[f] = m == 0.0f ? 0.0f : m;  // a zero minimum is stored as +0
            if (have_info) {
                bits[f] = (uint32_t)(info >> (5 * f)) & 31u;
            } else {
                bool bg, ex;
                block_field_width(kmin[f], kmax[f], a.d_params ? a.d_params[f] : a.params[f], bits[f], bg, ex);
                big |= bg;
                exact = exact && ex;
            }
            g[f] = f < P ? min((uint32_t)a.G, bits[f]) : 0u;
            o[f] = f < P ? bits[f] - g[f] : 0u;
            wf[f] = f < P ? o[f] : bits[f];
        }
        uint32_t ks = 0;
#pragma unroll
        for (int f = F - 1; f >= 0; --f) {
            kshift[f] = ks;
            ks += g[f];
            W += wf[f];
        }
        keybits = ks;
    }
    if (big || W > kFastRecordBits) {
        // left to the general kernel (uniform decision)
        if (t == 0) {
            if (DIRECT) st_release_u64(a.bstate + idx.b(), kBlkBroken);
            a.general_list[atomicAdd(a.general_count, 1u)] = idx.id();
        }
        return;
    }

    // ---- 3. quantise, key and record in one pass
    uint32_t key[4] = {0u, 0u, 0u, 0u};
    uint32_t rw[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rw[r][0] = rw[r][1] = rw[r][2] = rw[r][3] = 0u;
    bool pend = false;
    if (exact) {  // uniform: no first candidate of the block can fail its check
        if (W <= 64u) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const FieldParams p = a.d_params ? a.d_params[f] : a.params[f];
                quantise_append<2, false>(x[f], valid, mn[f], p, f < P, o[f], kshift[f], wf[f], key, rw, pend);
            }
        } else {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const FieldParams p = a.d_params ? a.d_params[f] : a.params[f];
                quantise_append<4, false>(x[f], valid, mn[f], p, f < P, o[f], kshift[f], wf[f], key, rw, pend);
            }
        }
    } else {
        if (W <= 64u) {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const FieldParams p = a.d_params ? a.d_params[f] : a.params[f];
                quantise_append<2, true>(x[f], valid, mn[f], p, f < P, o[f], kshift[f], wf[f], key, rw, pend);
            }
        } else {
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const FieldParams p = a.d_params ? a.d_params[f] : a.params[f];
                quantise_append<4, true>(x[f], valid, mn[f], p, f < P, o[f], kshift[f], wf[f], key, rw, pend);
            }
        }
        if (__any_sync(0xffffffffu, pend) && lane == 0) atomicOr(&S.flags, 2u);
    }

    // ---- 4. stable counting sort: warp-local ranks in storage order
    uint16_t* myhist = hist + w * kMaxBins;
    uint32_t rank[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const uint32_t peers = __match_any_sync(0xffffffffu, valid[r] ? key[r] : 0xffffffffu);
        uint32_t before = 0u;
        if (valid[r]) before = myhist[key[r]];
        __syncwarp();
        if (valid[r] && lane == 31 - __clz(peers)) myhist[key[r]] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        rank[r] = before + __popc(peers & lanemask_lt());
    }
    __syncthreads();  // C
    if (S.flags & 2u) {
        if (t == 0) {
            if (DIRECT) st_release_u64(a.bstate + idx.b(), kBlkBroken);
            a.general_list[atomicAdd(a.general_count, 1u)] = idx.id();
        }
        return;
    }

    // ---- 4b. scan over (bin, warp): sorted positions and the run-length code
    const int nbins = 1 << keybits;
    const int b0 = 2 * t;
    uint32_t c0 = 0, c1 = 0;
    uint32_t pre[kWarps];  // (prefix of bin b0) | (prefix of bin b0+1) << 16
    if (b0 < nbins) {
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t pair = *reinterpret_cast<const uint32_t*>(hist + ww * kMaxBins + b0);
            pre[ww] = c0 | (c1 << 16);
            c0 += pair & 0xffffu;
            c1 += pair >> 16;
        }
    }
    const uint32_t tot = c0 + c1;
    const uint32_t nz = (c0 ? 1u : 0u) + (c1 ? 1u : 0u);
    // one scan of both: the counts sum to at most 1024 and the non-empty bins
    // to at most 512, so they share a word
    const uint32_t incl_tn = warp_incl_sum(tot | (nz << 16));
    const uint32_t incl_tot = incl_tn & 0xffffu, incl_nz = incl_tn >> 16;
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, max(c0, c1));
    // the last non-empty bin up to this thread's (0 when none: a first id's
    // delta is the id itself), for the deltas of the unique ids
    uint32_t last = c1 ? (uint32_t)b0 + 1u : (c0 ? (uint32_t)b0 : 0u);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) last = max(last, __shfl_up_sync(0xffffffffu, last, o));
    if (lane == 31) {
        S.warp_tot[w] = incl_tn;
        S.warp_last[w] = last;
    }
    if (lane == 0) atomicMax(&S.maxcnt, cmax);
    __syncthreads();  // D
    uint32_t base_tot = 0, base_nz = 0, U = 0, prev = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t vtn = S.warp_tot[ww], vl = S.warp_last[ww];
        if (ww < w) {
            base_tot += vtn & 0xffffu;
            base_nz += vtn >> 16;
            prev = max(prev, vl);
        }
        U += vtn >> 16;
    }
    {
        const uint32_t up = __shfl_up_sync(0xffffffffu, last, 1);
        if (lane > 0) prev = max(prev, up);  // the last non-empty bin before b0
    }
    uint32_t dmax = 0;
    if (b0 < nbins) {
        const uint32_t start0 = base_tot + incl_tot - tot, start1 = start0 + c0;
        const uint32_t idx0 = base_nz + incl_nz - nz, idx1 = idx0 + (c0 ? 1u : 0u);
        const uint32_t base2 = start0 | (start1 << 16);  // neither half overflows: both < 1024
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww)
            *reinterpret_cast<uint32_t*>(hist + ww * kMaxBins + b0) = base2 + pre[ww];
        if (c0) {
            uniq[idx0] = (uint16_t)b0;
            cnt[idx0] = (uint16_t)c0;
        }
        if (c1) {
            uniq[idx1] = (uint16_t)(b0 + 1);
            cnt[idx1] = (uint16_t)c1;
        }
        if (c0) dmax = (uint32_t)b0 - prev;
        if (c1) dmax = max(dmax, (uint32_t)b0 + 1u - (c0 ? (uint32_t)b0 : prev));
    }
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    if (lane == 0 && dmax) atomicMax(&S.maxdelta, dmax);
    __syncthreads();  // E

    // ---- encoded size; raw when not smaller (keeps the bound size a bound)
    const uint32_t wd = bit_width(S.maxdelta), wc = bit_width(S.maxcnt);
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = ceil_words((uint32_t)n_b * W);
    const uint32_t enc = hdr + dwords + cwords + rwords;
    if (enc >= 1u + (uint32_t)F * (uint32_t)n_b) {
        raw_block<F, CM>(a, idx.b(), n_b, t);
        return;
    }
    if (DIRECT && t == 0) st_release_u64(a.bstate + idx.b(), (idx.b() == 0 ? kBlkIncl : kBlkAgg) | enc);

    // ---- 5. block header and the three arrays (Section 4.3), assembled in the
    // staging words (cleared at the start) -- the deltas and counts by
    // thread-serial appenders, the records each at its sorted position --
    // then copied out
    if (t == 0) stage[0] = (U << 1) | (wd << 12) | (wc << 17);
    if (t >= 1 && t <= F) {
        float m = 0.0f;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if (f == t - 1) m = mn[f];
        stage[t] = __float_as_uint(m);
    }
    if (t < ((F + 3) >> 2)) {
        uint32_t word = 0;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if ((f >> 2) == t) word |= bits[f] << (8 * (f & 3));
        stage[1 + F + t] = word;
    }
    {
        const uint32_t k0 = 2u * (uint32_t)t;
        if (k0 < U && wd) {
            BitAppender ap(32u * hdr + k0 * wd);
            ap.put(stage, (uint32_t)uniq[k0] - (k0 ? (uint32_t)uniq[k0 - 1] : 0u), wd);
            if (k0 + 1 < U) ap.put(stage, (uint32_t)uniq[k0 + 1] - (uint32_t)uniq[k0], wd);
            ap.finish(stage);
        }
        if (k0 < U && wc) {
            BitAppender ap(32u * (hdr + dwords) + k0 * wc);
            ap.put(stage, (uint32_t)cnt[k0], wc);
            if (k0 + 1 < U) ap.put(stage, (uint32_t)cnt[k0 + 1], wc);
            ap.finish(stage);
        }
    }
    // the records: each thread ORs its own four at their sorted positions
    {
        const uint32_t rbase = 32u * (hdr + dwords + cwords);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (!valid[r]) continue;
            const uint32_t dest = myhist[key[r]] + rank[r];  // sorted position
            if (a.perm) sperm[dest] = (uint16_t)(128 * w + 32 * r + lane);
            if (W == 0u) continue;
            const uint32_t bp = rbase + dest * W, wi = bp >> 5, sh = bp & 31u, end = sh + W;
            // the record is W bits, least significant word first, zero above W
            atomicOr(stage + wi, rw[r][0] << sh);
            if (end > 32u) atomicOr(stage + wi + 1, __funnelshift_l(rw[r][0], rw[r][1], sh));
            if (end > 64u) atomicOr(stage + wi + 2, __funnelshift_l(rw[r][1], rw[r][2], sh));
            if (end > 96u) atomicOr(stage + wi + 3, __funnelshift_l(rw[r][2], rw[r][3], sh));
            if (end > 128u) atomicOr(stage + wi + 4, __funnelshift_l(rw[r][3], 0u, sh));
        }
    }
    fence_proxy_async_shared();  // the staging words may be read by a bulk copy (async proxy)
    __syncthreads();
    uint32_t off = kNotPlaced;
    if constexpr (DIRECT) {  // the block's offset from its predecessors' sizes
        if (w == 0) {
            const uint32_t b = idx.b();
            uint32_t o = b == 0 ? 0u : block_lookback(a.bstate, b);
            if (o != kNotPlaced && (uint64_t)o + enc > a.direct_capacity) o = kNotPlaced;
            if (lane == 0) {
                if (b != 0) st_release_u64(a.bstate + b, o == kNotPlaced ? kBlkBroken : (kBlkIncl | (o + enc)));
                S.offset = o;
            }
        }
        __syncthreads();
        off = S.offset;
    }
    {
        const uint32_t b = idx.b();
        if (off != kNotPlaced) {  // straight into the stream (word-aligned)
            uint32_t* out = a.direct + off;
            for (uint32_t k = t; k < enc; k += kThreads) out[k] = stage[k];
        } else if (t == 0) {
            // to the temporary slot (16-byte aligned, room for the rounding
            // words) by one bulk copy, which the CTA's shared memory outlives:
            // thread 0 waits until the copy has read the staging words
            bulk_s2g(a.temp + (size_t)b * a.slot_words, stage, ((enc + 3u) & ~3u) * 4u);
        }
        const uint64_t first = (uint64_t)b * kBlock;
        if (a.perm)
            for (int j = t; j < n_b; j += kThreads) a.perm[first + j] = (uint32_t)first + sperm[j];
        if (t == 0) a.sizes[b] = enc | (off != kNotPlaced ? kPlaced : 0u);
    }
}


}  // namespace gpz
