// gpz_qse_tile.cuh -- the per-block body of the shared-memory tile
// compression kernel (Sections 4.1-4.3), used by the single-array kernel
// (gpz_qse_tile.cu, which describes the design) and by the batched kernel
// (gpz_batch_compress.cu).  Idx gives the block within its array (b()) and
// its entry for the general list (id()).
#pragma once

#include "gpz_qse_block.cuh"

namespace gpz {

namespace {

__host__ __device__ constexpr uint32_t tile_region_bytes(int F) {
    const uint32_t tile = (uint32_t)F * kBlock * 4u, stage = kStageWords * 4u;
    return tile > stage ? tile : stage;
}

__host__ __device__ constexpr uint32_t tile_smem_bytes(int F) {
    return tile_region_bytes(F) + kHistBytes + kMaxBins * 2u /*uniq*/ + kMaxBins * 2u /*counts*/ +
           kBlock * 2u /*perm*/;
}

// One field's constants for the block, derived once by thread f.
struct TileField {
    float mn, inv, s, ebchk;  // block minimum; step constants of the field
    uint32_t o, ks, wf, bits; // segOffset bits, key shift, record bits, code width
};

struct TileShared {
    uint64_t bar;                       // mbarrier of the tile's bulk copies
    uint32_t kmin[kMaxFields], kmax[kMaxFields];  // the block's extremes (absolute bound)
    TileField fc[kMaxFields];
    // bit 0: a non-finite value; bit 1: a value needs a fallback candidate;
    // bit 2: a code reaches 2^23 (general path); bit 3: some field's first
    // candidates need their check
    uint32_t flags;
    uint32_t maxcnt, maxdelta;
    uint32_t warp_tot[kWarps], warp_last[kWarps];
};

constexpr uint32_t kTfNonFinite = 1u, kTfFallback = 2u, kTfBig = 4u, kTfVerify = 8u;

// Field f's parameters from the argument block (uniform selection: the
// by-value parameters are not indexed dynamically).
template <int F>
__device__ __forceinline__ FieldParams field_params(const QseArgs& a, int f) {
    if (a.d_params) return a.d_params[f];
    FieldParams p = a.params[0];
#pragma unroll
    for (int k = 1; k < F; ++k)
        if (k == f) p = a.params[k];
    return p;
}

// Field t's constants for the block from its extremes (order keys), by
// thread t: q0 = floor(fma(x - min, 1/s, 1/2)) is monotone in x, so when
// every value keeps its first candidate the largest code is q0 of the block
// maximum.  P is the number of position fields.
template <int P>
__device__ __forceinline__ void field_constants(uint32_t kmin, uint32_t kmax, const FieldParams& p, int G, int t,
                                                TileShared& S) {
    uint32_t bits;
    bool big, exact;
    block_field_width(kmin, kmax, p, bits, big, exact);
    const float m0 = from_order_key(kmin);
    TileField c;
    c.mn = m0 == 0.0f ? 0.0f : m0;  // a zero minimum is stored as +0
    c.inv = p.inv;
    c.s = p.s;
    c.ebchk = p.ebchk;
    c.bits = bits;
    const uint32_t g = t < P ? min((uint32_t)G, bits) : 0u;
    c.o = t < P ? bits - g : 0u;
    c.wf = t < P ? c.o : bits;
    c.ks = g;  // this field's segId bits for now; the key shifts follow in every thread
    S.fc[t] = c;
    if (big) atomicOr(&S.flags, kTfBig);
    if (!exact) atomicOr(&S.flags, kTfVerify);
}

}  // namespace

// AOS: the input is interleaved records (a.interleaved); the tile then holds
// the block's records as they are in memory, value (f, i) at i * F + f.
template <int F, bool FULL, bool PRE, class Idx, bool AOS = false>
__device__ __forceinline__ void qse_block_tile(const QseArgs& a, uint8_t* dsm, TileShared& S, Idx idx) {
    constexpr int P = F < 3 ? F : 3;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t b = idx.b();  // the block within its array
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = FULL ? kBlock : (int)(a.n - first);
    float* tile = reinterpret_cast<float*>(dsm);                             // [F][1024] input ([1024][F] if AOS)
    // position of value (f, i) of the block in the tile
    auto at = [](int f, int i) { return AOS ? i * F + f : f * kBlock + i; };
    uint32_t* stage = reinterpret_cast<uint32_t*>(dsm);                      // the encoded block, later
    uint16_t* hist = reinterpret_cast<uint16_t*>(dsm + tile_region_bytes(F)); // [8][512] per-warp histograms
    uint16_t* uniq = hist + kWarps * kMaxBins;                               // [512]
    uint16_t* cnt = uniq + kMaxBins;                                         // [512]
    uint16_t* sperm = cnt + kMaxBins;                                        // [1024]

    // ---- 1. the tile: one bulk copy per field (thread 0); the ragged tail
    // of a last block by plain loads; the block's extremes
    // values moved in 16-byte units: per field, or of the whole run of records
    const uint32_t nvec = AOS ? ((uint32_t)(F * n_b) & ~3u) : ((uint32_t)n_b & ~3u);
    if (t == 0) {
        mbar_init(&S.bar, 1);
        mbar_arrive_expect_tx(&S.bar, (AOS ? 1u : (uint32_t)F) * nvec * 4u);
        if (nvec) {
            if (AOS) {
                bulk_g2s(tile, a.fields[0] + first * F, nvec * 4u, &S.bar);
            } else {
#pragma unroll
                for (int f = 0; f < F; ++f) bulk_g2s(tile + f * kBlock, a.fields[f] + first, nvec * 4u, &S.bar);
            }
        }
        S.flags = 0u;
        S.maxcnt = 0u;
        S.maxdelta = 0u;
    }
    if (AOS) {
        if (!FULL && t < 4) {
            const int k = (int)nvec + t;
            if (k < F * n_b) tile[k] = __ldcs(a.fields[0] + first * F + k);
        }
    } else if (!FULL && t < 4 * F) {
        const int f = t >> 2, i = (int)nvec + (t & 3);
        if (i < n_b) tile[f * kBlock + i] = __ldcs(a.fields[f] + first + i);
    }
    {
        uint32_t* h32 = reinterpret_cast<uint32_t*>(hist + w * kMaxBins);
#pragma unroll
        for (int k = 0; k < kMaxBins / 64; ++k) h32[lane + 32 * k] = 0u;
    }
    __syncwarp();  // S.flags cleared (thread 0) before threads 0..F-1 of warp 0 set bits in it
    if (t < F) {
        if (PRE) {  // from the range pass; (0, 0) marks a non-finite value
            const uint2 e = __ldg(a.bext + (size_t)b * F + t);
            const FieldParams p = field_params<F>(a, t);  // loaded with the extremes: one round trip
            if (e.x == 0u)
                atomicOr(&S.flags, kTfNonFinite);
            else
                field_constants<P>(e.x, e.y, p, a.G, t, S);
        } else {
            S.kmin[t] = 0xffffffffu;
            S.kmax[t] = 0u;
        }
    }
    bool valid[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) valid[r] = FULL || (128 * w + 32 * r + lane < n_b);
    __syncthreads();  // 1: the mbarrier, the counters and the extremes

    if constexpr (!PRE) {  // the block's extremes from the tile
        if (!mbar_wait_bounded(&S.bar, 0, a.status)) return;
        float probe = 0.0f;  // becomes NaN if any value is NaN or infinite (x * 0)
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float lo = INFINITY, hi = -INFINITY;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (valid[r]) {
                    const float x = tile[at(f, 128 * w + 32 * r + lane)];
                    probe = __fmaf_rn(x, 0.0f, probe);
                    lo = fminf(lo, x);
                    hi = fmaxf(hi, x);
                }
            }
            const uint32_t lk = __reduce_min_sync(0xffffffffu, lo == INFINITY ? 0xffffffffu : order_key(lo));
            const uint32_t hk = __reduce_max_sync(0xffffffffu, hi == -INFINITY ? 0u : order_key(hi));
            if (lane == 0) {
                atomicMin(&S.kmin[f], lk);
                atomicMax(&S.kmax[f], hk);
            }
        }
        if (__any_sync(0xffffffffu, probe != probe) && lane == 0) atomicOr(&S.flags, kTfNonFinite);
        __syncthreads();  // 1b: the extremes
    }

    // ---- 2. field constants (thread f) from the tile's extremes
    // (with a relative bound this was done before barrier 1)
    if (t < F && !PRE && !(S.flags & kTfNonFinite))
        field_constants<P>(S.kmin[t], S.kmax[t], field_params<F>(a, t), a.G, t, S);
    if constexpr (!PRE) __syncthreads();  // 2: the field constants
    uint32_t flags = S.flags;
    if (flags & kTfNonFinite) {
        if (PRE && !mbar_wait_bounded(&S.bar, 0, a.status)) return;  // no copy may outlive the CTA
        raw_block<F, kCmTemp>(a, b, n_b, t);
        return;
    }
    // key shifts (fields after f below it) and the record width
    uint32_t W = 0, keybits = 0;
#pragma unroll
    for (int f = F - 1; f >= 0; --f) {
        keybits += f < P ? S.fc[f].ks : 0u;
        W += S.fc[f].wf;
    }
    if ((flags & kTfBig) || W > kFastRecordBits) {
        if (PRE) mbar_wait_bounded(&S.bar, 0, a.status);
        if (t == 0) a.general_list[atomicAdd(a.general_count, 1u)] = idx.id();
        return;
    }

    // ---- 3. quantise from the tile, key and record in one pass
    if (PRE && !mbar_wait_bounded(&S.bar, 0, a.status)) return;
    uint32_t key[4] = {0u, 0u, 0u, 0u};
    uint32_t rw[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rw[r][0] = rw[r][1] = rw[r][2] = rw[r][3] = 0u;
    bool pend = false;
    {
        // key shift of position field f: the segId bits of the position fields after it
        uint32_t kshift[P];
        {
            uint32_t ks = 0;
#pragma unroll
            for (int f = P - 1; f >= 0; --f) {
                kshift[f] = ks;
                ks += S.fc[f].ks;
            }
        }
        const bool verify = (flags & kTfVerify) != 0u, wide = W > 64u;  // uniform
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const TileField c = S.fc[f];
            FieldParams p;
            p.eb = 0.0f;
            p.s = c.s;
            p.inv = c.inv;
            p.ebchk = c.ebchk;
            float x[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) x[r] = tile[at(f, 128 * w + 32 * r + lane)];
            const uint32_t ks = f < P ? kshift[f < P ? f : 0] : 0u;
            if (!verify) {
                if (!wide)
                    quantise_append<2, false>(x, valid, c.mn, p, f < P, c.o, ks, c.wf, key, rw, pend);
                else
                    quantise_append<4, false>(x, valid, c.mn, p, f < P, c.o, ks, c.wf, key, rw, pend);
            } else {
                if (!wide)
                    quantise_append<2, true>(x, valid, c.mn, p, f < P, c.o, ks, c.wf, key, rw, pend);
                else
                    quantise_append<4, true>(x, valid, c.mn, p, f < P, c.o, ks, c.wf, key, rw, pend);
            }
        }
        if (verify && __any_sync(0xffffffffu, pend) && lane == 0) atomicOr(&S.flags, kTfFallback);
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
    __syncthreads();  // C: every value quantised (the tile is dead) and ranked
    if (S.flags & kTfFallback) {
        if (t == 0) a.general_list[atomicAdd(a.general_count, 1u)] = idx.id();
        return;
    }
    {
        // the staging words, assembled by OR, overlay the tile: clear them
        uint4* s4 = reinterpret_cast<uint4*>(stage);
        for (uint32_t k = t; k < kStageWords / 4u; k += kThreads) s4[k] = make_uint4(0u, 0u, 0u, 0u);
    }

    // ---- 4b. scan over (bin, warp): sorted positions and the run-length code
    const int nbins = 1 << keybits;
    const int b0 = 2 * t;
    uint32_t c0 = 0, c1 = 0;  // counts of bins b0 and b0 + 1 over the warps
    if (b0 < nbins) {
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t pair = *reinterpret_cast<const uint32_t*>(hist + ww * kMaxBins + b0);
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
        // each warp's sorted start of the two bins: the start plus the counts
        // of the warps before it (re-read rather than held across the barrier)
        uint32_t run = start0 | (start1 << 16);  // neither half overflows: both < 1024
#pragma unroll
        for (int ww = 0; ww < kWarps; ++ww) {
            uint32_t* cell = reinterpret_cast<uint32_t*>(hist + ww * kMaxBins + b0);
            const uint32_t pair = *cell;
            *cell = run;
            run += pair;
        }
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
        raw_block<F, kCmTemp>(a, b, n_b, t);
        return;
    }

    // ---- 5. block header and the three arrays (Section 4.3), assembled in the
    // cleared staging words -- each thread ORs in two deltas, two counts and
    // its four records at their positions -- then one bulk copy to the
    // temporary slot
    if (t == 0) stage[0] = (U << 1) | (wd << 12) | (wc << 17);
    if (t >= 1 && t <= F) stage[t] = __float_as_uint(S.fc[t - 1].mn);
    if (t < ((F + 3) >> 2)) {
        uint32_t word = 0;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if ((f >> 2) == t) word |= S.fc[f].bits << (8 * (f & 3));
        stage[1 + F + t] = word;
    }
    {
        // deltas and counts of unique ids 2t and 2t+1: at most 2 x 9 and
        // 2 x 11 bits, so each pair is ORed into at most two words
        const uint32_t k0 = 2u * (uint32_t)t;
        if (k0 < U) {
            const bool two = k0 + 1 < U;
            const uint32_t u0 = uniq[k0], u1 = two ? (uint32_t)uniq[k0 + 1] : u0;
            const uint32_t dv = (u0 - (k0 ? (uint32_t)uniq[k0 - 1] : 0u)) | ((u1 - u0) << wd);
            const uint32_t cv = (uint32_t)cnt[k0] | ((two ? (uint32_t)cnt[k0 + 1] : 0u) << wc);
            const uint32_t nd = (two ? 2u : 1u) * wd, nc = (two ? 2u : 1u) * wc;
            const uint32_t dp = 32u * hdr + k0 * wd, cp = 32u * (hdr + dwords) + k0 * wc;
            if (nd) {
                atomicOr(stage + (dp >> 5), dv << (dp & 31u));
                if ((dp & 31u) + nd > 32u) atomicOr(stage + (dp >> 5) + 1, dv >> (32u - (dp & 31u)));
            }
            if (nc) {
                atomicOr(stage + (cp >> 5), cv << (cp & 31u));
                if ((cp & 31u) + nc > 32u) atomicOr(stage + (cp >> 5) + 1, cv >> (32u - (cp & 31u)));
            }
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
    fence_proxy_async_shared();  // the staging words are read by a bulk copy (async proxy)
    __syncthreads();
    if (t == 0) bulk_s2g(a.temp + (size_t)b * a.slot_words, stage, ((enc + 3u) & ~3u) * 4u);
    if (a.perm)
        for (int j = t; j < n_b; j += kThreads) a.perm[first + j] = (uint32_t)first + sperm[j];
    if (t == 0) a.sizes[b] = enc;
}

}  // namespace gpz
