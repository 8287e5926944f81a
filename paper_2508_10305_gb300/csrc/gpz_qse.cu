// gpz_qse.cu -- the fused per-block compression kernel (stages 1-3 of GPZ:
// quantisation, sorting, encoding; Sections 4.1-4.3 and Table 1's "Q.S.E."
// kernel) and the global range pass of the relative error bound.
//
// One warp owns one block of 1024 particles (Section 4: one warp per block),
// kQseWarps warps per CTA.  Per warp:
//   1. the block's F field tiles (4 KB each) are staged into shared memory
//      with one bulk copy per field (cp.async.bulk + mbarrier);
//   2. per field: exact fp32 minimum (Section 4.1), quantisation
//      q = floor(fma(x - min, 1/s, 1/2)) with the fp32 verification and
//      candidate fallback of the stream format, widths;
//   3. segId / segOffset by shift and mask (Section 5.1), the linearised
//      segId (key) and the per-particle record, in registers;
//   4. stable counting sort by key (Section 4.2): ranks in storage order from
//      __match_any_sync groups, a shared histogram, an exclusive scan;
//      the non-empty histogram bins are exactly the run-length code
//      (unique ids and counts, Section 4.3), so sort and run-length coding
//      share one pass;
//   5. fixed-length coding (Section 4.3): each lane packs 32 consecutive
//      values serially into a 64-bit accumulator; packed words are staged
//      in shared memory and written out coalesced;
//   6. the block's words go to its fixed temporary slot (step 1 of the
//      three-step compaction, Section 4.4) with its word count.
#include "gpz_internal.cuh"

namespace gpz {

// ------------------------------------------------------------------ range pass (relative bound)

__global__ void __launch_bounds__(kRangeThreads) gpz_range_kernel(RangeArgs a) {
    __shared__ float2 red[kRangeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int f = 0; f < a.F; ++f) {
        const float* x = a.fields[f];
        float lo = INFINITY, hi = -INFINITY;
        if (a.vec_ok) {
            const float4* x4 = reinterpret_cast<const float4*>(x);
            const uint64_t n4 = a.n >> 2;
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < n4; i += (uint64_t)gridDim.x * blockDim.x) {
                float4 v = __ldcs(x4 + i);
                lo = fminf(fminf(lo, v.x), fminf(v.y, fminf(v.z, v.w)));
                hi = fmaxf(fmaxf(hi, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
            }
            for (uint64_t i = (n4 << 2) + (uint64_t)blockIdx.x * blockDim.x + tid; i < a.n;
                 i += (uint64_t)gridDim.x * blockDim.x) {
                float v = x[i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        } else {
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
                float v = x[i];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        }
        lo = warp_min_f32(lo);
        hi = warp_max_f32(hi);
        if (lane == 0) red[warp] = make_float2(lo, hi);
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kRangeThreads / 32; ++w) {
                lo = fminf(lo, red[w].x);
                hi = fmaxf(hi, red[w].y);
            }
            a.partials[(size_t)blockIdx.x * a.F + f] = make_float2(lo, hi);
        }
        __syncthreads();
    }
    // The last CTA to finish folds the partials and finalises the constants.
    __shared__ bool last;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(a.done_counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid < a.F) {
        const int f = tid;
        float lo = INFINITY, hi = -INFINITY;
        for (unsigned c = 0; c < gridDim.x; ++c) {
            float2 p = __ldcg(a.partials + (size_t)c * a.F + f);
            lo = fminf(lo, p.x);
            hi = fmaxf(hi, p.y);
        }
        double rel = a.rel[0];
#pragma unroll
        for (int k = 1; k < kMaxFields; ++k)
            if (k == f) rel = a.rel[k];
        // eb = rel * (max - min) when that range is a finite positive number,
        // else eb = rel; step = eb * 63/32; reciprocal; verification threshold.
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
        a.d_params[f] = p;
    }
}

cudaError_t launch_range(const RangeArgs& a, int grid, cudaStream_t s) {
    gpz_range_kernel<<<grid, kRangeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ fused Q.S.E. kernel

// Per-warp scalars shared by the lanes (warp-uniform values).
struct WarpMeta {
    FieldParams p[kMaxFields];
    const float* ptr[kMaxFields];
    float mn[kMaxFields];
    uint32_t bits[kMaxFields];
    uint32_t w[kMaxFields];       // record width of the field: o (positions) or bits (extra fields)
    uint32_t o[kMaxFields];       // segOffset bits of a position axis
    uint32_t kshift[kMaxFields];  // left shift of the axis' segId within the key
    uint32_t rshift[kMaxFields];  // bit offset of the field inside the record
};

// Verification of one candidate code (the decompressor's reconstruction).
__device__ __forceinline__ bool code_ok(float x, uint32_t q, const FieldParams& p, float mn) {
    const float xh = __fmaf_rn(__uint2float_rn(q), p.s, mn);
    return fabsf(__fsub_rn(x, xh)) <= p.ebchk;
}

__device__ __noinline__ bool adjust_code(float x, uint32_t* q, FieldParams p, float mn) {
    if (*q > 0u && code_ok(x, *q - 1u, p, mn)) {
        *q -= 1u;
        return true;
    }
    if (code_ok(x, *q + 1u, p, mn)) {
        *q += 1u;
        return true;
    }
    return false;
}

// Write the packed words staged in `stage` (rows of kRow) to out: row L's
// words [c0, c0 + len) belong at out[L * row_words + c0 + ...]; words at or
// beyond `total` are not written.
__device__ __forceinline__ void flush_rows(const uint32_t* stage, uint32_t* out, int nrows, uint32_t row_words,
                                           uint32_t c0, uint32_t len, uint32_t total, int lane) {
    __syncwarp();
    if ((uint32_t)lane < len) {
        for (int L = 0; L < nrows; ++L) {
            const uint32_t idx = (uint32_t)L * row_words + c0 + lane;
            if (idx < total) out[idx] = stage[L * kRow + lane];
        }
    }
    __syncwarp();
}

// Fixed-length code of `len` u32 values held in padded rows of `src`, width
// w (0..31); lane L packs values [32L, 32L+32).  Returns the word count.
__device__ uint32_t pack_u32(const uint32_t* src, int len, uint32_t w, uint32_t* stage, uint32_t* out, int lane) {
    const uint32_t total = ceil_words((uint32_t)len * w);
    if (total == 0) return 0;
    const int nrows = (len + 31) >> 5;
    unsigned long long acc = 0;
    uint32_t nb = 0, k = 0;
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
        const int j = 32 * lane + t;
        const uint32_t v = j < len ? src[lane * kRow + t] : 0u;
        acc |= (unsigned long long)v << nb;
        nb += w;
        if (nb >= 32u) {
            stage[lane * kRow + k] = (uint32_t)acc;
            acc >>= 32;
            nb -= 32u;
            ++k;
        }
    }
    flush_rows(stage, out, nrows, w, 0, w, total, lane);
    return total;
}

// Fixed-length code of n_b records of width W <= 64, records held as u64 in
// padded rows of `rec`.  A lane's 32 records make W words; every 32 emitted
// words are flushed.
__device__ uint32_t pack_records64(const unsigned long long* rec, int n_b, uint32_t W, uint32_t* stage,
                                   uint32_t* out, int lane) {
    const uint32_t total = ceil_words((uint32_t)n_b * W);
    if (total == 0) return 0;
    const int nrows = (n_b + 31) >> 5;
    const uint32_t wlo = W < 32u ? W : 32u;
    const uint32_t whi = W - wlo;
    const uint32_t mlo = wlo == 32u ? 0xffffffffu : ((1u << wlo) - 1u);
    unsigned long long acc = 0;
    uint32_t nb = 0, k = 0;
    for (int t = 0; t < 32; ++t) {
        const int j = 32 * lane + t;
        const unsigned long long r = j < n_b ? rec[lane * kRow + t] : 0ull;
        acc |= (unsigned long long)((uint32_t)r & mlo) << nb;
        nb += wlo;
        if (nb >= 32u) {
            stage[lane * kRow + (k & 31u)] = (uint32_t)acc;
            acc >>= 32;
            nb -= 32u;
            ++k;
            if ((k & 31u) == 0u) flush_rows(stage, out, nrows, W, k - 32u, 32u, total, lane);
        }
        if (whi) {
            acc |= (unsigned long long)(uint32_t)(r >> 32) << nb;
            nb += whi;
            if (nb >= 32u) {
                stage[lane * kRow + (k & 31u)] = (uint32_t)acc;
                acc >>= 32;
                nb -= 32u;
                ++k;
                if ((k & 31u) == 0u) flush_rows(stage, out, nrows, W, k - 32u, 32u, total, lane);
            }
        }
    }
    if (k & 31u) flush_rows(stage, out, nrows, W, k & ~31u, k & 31u, total, lane);
    return total;
}

// General record packer (W > 64): codes are read field by field from the
// quantised tile through the block permutation.
__device__ uint32_t pack_records_wide(const uint32_t* tile, const uint32_t* perm_rows, const WarpMeta* m, int F,
                                     int P, int n_b, uint32_t W, uint32_t* stage, uint32_t* out, int lane) {
    const uint32_t total = ceil_words((uint32_t)n_b * W);
    const int nrows = (n_b + 31) >> 5;
    unsigned long long acc = 0;
    uint32_t nb = 0, k = 0;
    for (int t = 0; t < 32; ++t) {
        const int j = 32 * lane + t;
        const bool valid = j < n_b;
        const uint32_t i = valid ? perm_rows[lane * kRow + t] : 0u;
        for (int f = F - 1; f >= 0; --f) {
            const uint32_t wf = m->w[f];
            uint32_t code = valid ? tile[f * kBlock + i] : 0u;
            if (f < P) code &= (wf == 0u ? 0u : (0xffffffffu >> (32u - wf)));
            acc |= (unsigned long long)code << nb;
            nb += wf;
            if (nb >= 32u) {
                stage[lane * kRow + (k & 31u)] = (uint32_t)acc;
                acc >>= 32;
                nb -= 32u;
                ++k;
                if ((k & 31u) == 0u) flush_rows(stage, out, nrows, W, k - 32u, 32u, total, lane);
            }
        }
    }
    if (k & 31u) flush_rows(stage, out, nrows, W, k & ~31u, k & 31u, total, lane);
    return total;
}

__device__ void write_raw_block(const QseArgs& a, const WarpMeta* m, uint64_t first, int n_b, uint32_t* out,
                                int lane) {
    if (lane == 0) out[0] = 1u;
    for (int f = 0; f < a.F; ++f) {
        const float* src = m->ptr[f] + first;
        for (int i = lane; i < n_b; i += 32) out[1 + f * n_b + i] = __float_as_uint(__ldg(src + i));
    }
    if (a.perm) {
        for (int i = lane; i < n_b; i += 32) a.perm[first + i] = (uint32_t)(first + i);
    }
    if (lane == 0) a.sizes[(uint32_t)(first / kBlock)] = 1u + (uint32_t)a.F * (uint32_t)n_b;
}

uint32_t qse_warp_bytes(int F, uint32_t* tile_bytes) {
    uint32_t tb = (uint32_t)F * kBlock * 4u;
    const uint32_t rec_bytes = kPadWords * 8u;  // 1056 u64 records
    if (tb < rec_bytes) tb = rec_bytes;
    tb = (tb + 127u) & ~127u;
    if (tile_bytes) *tile_bytes = tb;
    uint32_t bytes = tb + 2u * kPadWords * 4u + kMaxBins * 4u + (uint32_t)sizeof(WarpMeta) + 16u;
    return (bytes + 127u) & ~127u;
}

__global__ void __launch_bounds__(32 * kQseWarps) gpz_qse_kernel(QseArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= a.nblocks) return;

    uint8_t* base = smem + (size_t)warp * a.warp_bytes;
    uint32_t* tile = reinterpret_cast<uint32_t*>(base);
    unsigned long long* rec_rows = reinterpret_cast<unsigned long long*>(base);
    uint32_t* scr = reinterpret_cast<uint32_t*>(base + a.tile_bytes);
    uint32_t* stage = scr + kPadWords;
    uint32_t* hist = stage + kPadWords;
    WarpMeta* m = reinterpret_cast<WarpMeta*>(hist + kMaxBins);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(m) + sizeof(WarpMeta));

    const int F = a.F;
    const int P = F < 3 ? F : 3;
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = (int)((a.n - first) < (uint64_t)kBlock ? (a.n - first) : (uint64_t)kBlock);

    // Per-field constants and pointers into the warp's meta block.
#pragma unroll
    for (int k = 0; k < kMaxFields; ++k) {
        if (lane == k && k < F) {
            m->p[k] = a.d_params ? a.d_params[k] : a.params[k];
            m->ptr[k] = a.fields[k];
        }
    }
    __syncwarp();

    // ---- 1. stage the field tiles
    const bool bulk = a.bulk_ok && n_b == kBlock;
    if (bulk) {
        if (lane == 0) {
            mbar_init(mbar, 1);
            mbar_expect_tx(mbar, (uint32_t)F * kBlock * 4u);
            for (int f = 0; f < F; ++f) bulk_g2s(tile + f * kBlock, m->ptr[f] + first, kBlock * 4u, mbar);
        }
    } else {
        for (int f = 0; f < F; ++f) {
            const float* src = m->ptr[f] + first;
            for (int i = lane; i < n_b; i += 32) tile[f * kBlock + i] = __float_as_uint(__ldg(src + i));
        }
    }
#pragma unroll
    for (int k = 0; k < kMaxBins / 32; ++k) hist[lane + 32 * k] = 0u;
    __syncwarp();
    if (bulk) {
        if (!mbar_wait_bounded(mbar, 0, a.status)) {
            // The copy never completed (status holds GPZ_ERR_TIMEOUT): wait
            // once more, bounded, for the copies in flight; leave an empty
            // block so that the later stages stay inside their buffers.
            mbar_wait_bounded(mbar, 0, a.status);
            if (lane == 0) a.sizes[b] = 0u;
            return;
        }
    }
    __syncwarp();

    uint32_t* out = a.temp + (size_t)b * a.slot_words;

    // ---- 2. block minimum per field; non-finite values force raw storage
    bool nonfinite = false;
    for (int f = 0; f < F; ++f) {
        const uint32_t* tf = tile + f * kBlock;
        float mn = INFINITY;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = 32 * r + lane;
            if (i < n_b) {
                const float x = __uint_as_float(tf[i]);
                nonfinite |= !(fabsf(x) <= 3.402823466e38f);
                mn = fminf(mn, x);
            }
        }
        mn = warp_min_f32(mn);
        if (mn == 0.0f) mn = 0.0f;  // a zero minimum is stored as +0
        if (lane == 0) m->mn[f] = mn;
    }
    if (__any_sync(0xffffffffu, nonfinite)) {
        write_raw_block(a, m, first, n_b, out, lane);
        return;
    }
    __syncwarp();

    // ---- 2b. quantisation with verification; widths
    bool fail = false;
    for (int f = 0; f < F; ++f) {
        uint32_t* tf = tile + f * kBlock;
        const FieldParams p = m->p[f];
        const float mn = m->mn[f];
        uint32_t qmax = 0u;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = 32 * r + lane;
            if (i < n_b) {
                const float x = __uint_as_float(tf[i]);
                const float t = __fmaf_rn(__fsub_rn(x, mn), p.inv, 0.5f);
                uint32_t q = 0u;
                if (t < 2147483648.0f) {
                    q = __float2uint_rd(t);
                    if (!code_ok(x, q, p, mn)) fail |= !adjust_code(x, &q, p, mn);
                } else {
                    fail = true;
                }
                tf[i] = q;
                qmax = max(qmax, q);
            }
        }
        qmax = warp_max_u32(qmax);
        if (lane == 0) m->bits[f] = bit_width(qmax);
    }
    if (__any_sync(0xffffffffu, fail)) {
        write_raw_block(a, m, first, n_b, out, lane);
        return;
    }
    __syncwarp();

    // ---- 3. segment split (shift and mask), key layout, record layout
    uint32_t keybits = 0, W = 0;
    {
        uint32_t g[kMaxFields], w[kMaxFields];
#pragma unroll
        for (int f = 0; f < kMaxFields; ++f) {
            const uint32_t bf = f < F ? m->bits[f] : 0u;
            g[f] = f < P ? min((uint32_t)a.G, bf) : 0u;
            w[f] = f < P ? bf - g[f] : bf;
            keybits += g[f];
            W += w[f];
        }
        if (lane == 0) {
            uint32_t ks = 0, rs = 0;
#pragma unroll
            for (int f = kMaxFields - 1; f >= 0; --f) {
                if (f < F) {
                    m->w[f] = w[f];
                    m->o[f] = f < P ? w[f] : 0u;
                    m->kshift[f] = ks;
                    m->rshift[f] = rs;
                    ks += g[f];
                    rs += w[f];
                }
            }
        }
    }
    __syncwarp();

    const bool fast = W <= 64u;
    uint32_t kr[32];              // key | rank << 16
    unsigned long long rec[32];   // record (fast path)
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        kr[r] = 0u;
        rec[r] = 0ull;
    }
    for (int f = 0; f < F; ++f) {
        const uint32_t* tf = tile + f * kBlock;
        const uint32_t o = m->o[f], ks = m->kshift[f], rs = m->rshift[f];
        const bool pos = f < P;
        const bool in_rec = fast && m->w[f] != 0u;  // a zero-width field adds no bits (and rs may be 64)
        const uint32_t omask = o == 0u ? 0u : (0xffffffffu >> (32u - o));
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int i = 32 * r + lane;
            const uint32_t q = i < n_b ? tf[i] : 0u;
            if (pos) kr[r] |= (q >> o) << ks;
            if (in_rec) rec[r] |= (unsigned long long)(pos ? (q & omask) : q) << rs;
        }
    }

    // ---- 4. stable counting sort: ranks in storage order
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = 32 * r + lane;
        const bool valid = i < n_b;
        const uint32_t key = kr[r];
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? key : 0xffffffffu);
        uint32_t before = 0u;
        if (valid) before = hist[key];
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) hist[key] = before + __popc(peers);
        __syncwarp();
        kr[r] = key | ((before + __popc(peers & lanemask_lt())) << 16);
    }

    // ---- 4b. scan of the histogram = run-length code (unique ids, counts)
    const int nbins = 1 << keybits;
    uint32_t* dlt = scr;            // deltas, padded rows 0..15
    uint32_t* cnt = scr + 16 * kRow; // counts, padded rows 16..31
    uint32_t U, wd, wc;
    {
        const int b0 = 16 * lane;
        uint32_t c[16];
        uint32_t sum = 0, nz = 0, cmax = 0;
        int last_nz = -1;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            c[k] = (b0 + k < nbins) ? hist[b0 + k] : 0u;
            sum += c[k];
            nz += c[k] ? 1u : 0u;
            cmax = max(cmax, c[k]);
            if (c[k]) last_nz = b0 + k;
        }
        const uint32_t sum_incl = warp_incl_sum(sum);
        const uint32_t nz_incl = warp_incl_sum(nz);
        int prev_nz = __shfl_up_sync(0xffffffffu, warp_incl_max(last_nz), 1);
        if (lane == 0) prev_nz = -1;
        uint32_t start = sum_incl - sum, idx = nz_incl - nz, dmax = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (b0 + k < nbins) hist[b0 + k] = start;  // exclusive start of the bin
            start += c[k];
            if (c[k]) {
                const uint32_t d = (uint32_t)(b0 + k) - (prev_nz < 0 ? 0u : (uint32_t)prev_nz);
                dlt[pad_idx((int)idx)] = d;
                cnt[pad_idx((int)idx)] = c[k];
                dmax = max(dmax, d);
                prev_nz = b0 + k;
                ++idx;
            }
        }
        U = __shfl_sync(0xffffffffu, nz_incl, 31);
        wd = bit_width(warp_max_u32(dmax));
        wc = bit_width(warp_max_u32(cmax));
    }
    __syncwarp();

    // ---- encoded size; raw when not smaller (keeps the bound size a bound)
    const uint32_t hdr = 1u + (uint32_t)F + (uint32_t)((F + 3) >> 2);
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = ceil_words((uint32_t)n_b * W);
    const uint32_t enc = hdr + dwords + cwords + rwords;
    if (enc >= 1u + (uint32_t)F * (uint32_t)n_b) {
        write_raw_block(a, m, first, n_b, out, lane);
        return;
    }

    // ---- 5. block header and the three arrays
    if (lane == 0) out[0] = (U << 1) | (wd << 12) | (wc << 17);
    if (lane >= 1 && lane <= F) out[lane] = __float_as_uint(m->mn[lane - 1]);
    if (lane < ((F + 3) >> 2)) {
        uint32_t word = 0;
        for (int k = 0; k < 4; ++k) {
            const int f = 4 * lane + k;
            if (f < F) word |= m->bits[f] << (8 * k);
        }
        out[1 + F + lane] = word;
    }
    pack_u32(dlt, (int)U, wd, stage, out + hdr, lane);
    pack_u32(cnt, (int)U, wc, stage, out + hdr + dwords, lane);

    // ---- 4c. scatter to sorted order: records (fast path) and the permutation
    const bool need_perm = a.perm != nullptr || !fast;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int i = 32 * r + lane;
        if (i < n_b) {
            const uint32_t key = kr[r] & 0xffffu;
            const int dest = (int)(hist[key] + (kr[r] >> 16));
            if (fast) rec_rows[pad_idx(dest)] = rec[r];
            if (need_perm) scr[pad_idx(dest)] = (uint32_t)i;
        }
    }
    __syncwarp();

    if (fast)
        pack_records64(rec_rows, n_b, W, stage, out + hdr + dwords + cwords, lane);
    else
        pack_records_wide(tile, scr, m, F, P, n_b, W, stage, out + hdr + dwords + cwords, lane);

    if (a.perm) {
        for (int r = 0; r < 32; ++r) {
            const int j = 32 * r + lane;
            if (j < n_b) a.perm[first + j] = (uint32_t)first + scr[r * kRow + lane];
        }
    }
    if (lane == 0) a.sizes[b] = enc;
}

// Warps per CTA: shared memory per warp limits residency, so pick the CTA
// width that keeps the most warps resident per SM (228 KB, 1 KB reserved per
// CTA).
int qse_warps_per_cta(uint32_t warp_bytes) {
    const uint32_t sm_bytes = 228u * 1024u;
    int best = 1, best_warps = 0;
    for (int w = 1; w <= kQseWarps; ++w) {
        const uint32_t cta = (uint32_t)w * warp_bytes + 1024u;
        if ((uint32_t)w * warp_bytes > 227u * 1024u) break;
        const int ctas = (int)(sm_bytes / cta);
        const int warps = (ctas > 32 ? 32 : ctas) * w;
        if (warps > best_warps) {
            best_warps = warps;
            best = w;
        }
    }
    return best;
}

cudaError_t launch_qse(const QseArgs& a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    const int wpc = qse_warps_per_cta(a.warp_bytes);
    const size_t smem = (size_t)a.warp_bytes * wpc;
    cudaError_t e = cudaFuncSetAttribute(gpz_qse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (a.nblocks + wpc - 1) / wpc;
    gpz_qse_kernel<<<grid, 32 * wpc, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpz
