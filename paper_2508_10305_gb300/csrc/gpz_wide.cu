// gpz_wide.cu -- 64-bit intermediates (Section 5.2, shared memory usage: GPZ
// keeps 32-bit intermediate values unless the value range or the precision
// needs 64-bit ones).  fp64 fields are quantised in fp64 to codes below 2^53
// and coded with the four stages of the 32-bit form (Sections 4.1-4.4); the
// stream is version 2:
//   header      16 words as version 1, word 1 = 2;
//   extension   4F words: per field eb and s as doubles, low word first;
//   table       nblocks + 1 word offsets, as version 1;
//   raw block   1, then the F x n_b fp64 values (two words each), field-major;
//   encoded     mode word (U, w_delta, w_count as version 1), the F block
//               minima as doubles (2F words), the code widths (bytes <= 53),
//               the deltas, the counts and the records (field 0 most
//               significant, up to 8 x 53 bits).
// Constants: s = RN64(eb * 63/32), inv = RN64(1/s), ebchk = eb less two ulps
// toward zero; a value's code is the first of q, q - 1, q + 1 (q =
// floor(fma(x - min, inv, 0.5))) whose reconstruction fma(q, s, min) is within
// ebchk, computed as one rounded difference -- which bounds the exact
// difference by eb.  A block with a non-finite value, a code that would reach
// 2^53 or no passing candidate is stored raw, as is a block whose encoding is
// not smaller.
//
// Kernels: a range pass (relative bounds), one CTA per block for the stages
// (the codes sorted into shared memory, each thread's four sorted records
// appended into staging words), the scan and copy of the 32-bit form, and one
// CTA per block to decode (the record words staged in shared memory).
#include <cmath>
#include <cstring>

#include "gpz.h"
#include "gpz_host.hpp"
#include "gpz_internal.cuh"

using namespace gpz;
using namespace gpz::host;

namespace gpz {

constexpr int kWideThreads = 256;
constexpr int kWideWarps = kWideThreads / 32;
constexpr uint32_t kWideMaxBits = 53;
constexpr unsigned long long kWideLimit = 1ull << 53;  // codes stay below 2^53
constexpr double kWideLimitD = 9007199254740992.0;     // 2^53
constexpr uint32_t kWideDcWords = 144u + 176u;         // deltas (<= 9 bits) and counts (<= 11 bits) of <= 512 runs

struct WideParams {
    double eb, s, inv, ebchk;
};

struct WideRangeArgs {
    const double* fields[kMaxFields];
    uint64_t n;
    int F;
    unsigned long long* res;  // [F][2]: max of ~key (the minimum), max of key, over the non-NaN values; zeroed
};

struct WideQseArgs {
    const double* fields[kMaxFields];
    uint64_t n;
    int F, G;
    WideParams params[kMaxFields];
    uint32_t* temp;  // [nblocks][slot_words]
    uint32_t slot_words;
    uint32_t* sizes;  // [nblocks]
    uint32_t* perm;   // [n] or nullptr
};

struct WideDecArgs {
    const uint32_t* stream;
    uint64_t total_words;
    double* out[kMaxFields];
    uint64_t n;
    int F;
    uint32_t nblocks;
    uint32_t* status;
};

__device__ __forceinline__ unsigned long long wide_key(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double wide_from_key(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Maximum over the warp (every lane calls it): the largest high word, then
// the largest low word among the lanes that hold it (two redux operations).
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ uint32_t bit_width64(unsigned long long v) { return 64u - (uint32_t)__clzll((long long)v); }

__device__ __forceinline__ unsigned long long mask64(uint32_t w) { return w >= 64u ? ~0ull : ((1ull << w) - 1ull); }

// |d| <= c for a non-NaN d and c >= 0, on the bit patterns (integer pipe).
__device__ __forceinline__ bool abs_le(double d, double c) {
    return ((unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull) <=
           (unsigned long long)__double_as_longlong(c);
}

// (double)q for q < 2^53 (exact), assembled on the integer pipe: exponent
// from the leading bit, the bits below it as the fraction.
__device__ __forceinline__ double code_to_double(unsigned long long q) {
    const int e = 63 - __clzll((long long)q);  // -1 for q = 0
    const unsigned long long frac = (q << ((52 - e) & 63)) & 0xfffffffffffffull;
    const unsigned long long bits = ((unsigned long long)(1023 + e) << 52) | frac;
    return q ? __longlong_as_double((long long)bits) : 0.0;
}

// floor(t) for 0 <= t < 2^53, on the integer pipe: the significand shifted
// right by the fraction bits the exponent leaves below the binary point.
__device__ __forceinline__ unsigned long long code_floor(double t) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(t);
    const int e = (int)(u >> 52) - 1023;  // t >= 0
    const unsigned long long m = (u & 0xfffffffffffffull) | 0x10000000000000ull;
    return e < 0 ? 0ull : (e >= 52 ? m : (m >> (52 - e)));
}

// The decompressor's reconstruction of code q, checked against the bound
// (x is finite, so x - x^ is never NaN).
__device__ __forceinline__ bool wide_ok(double x, unsigned long long q, const WideParams& p, double mn) {
    const double xh = __fma_rn(code_to_double(q), p.s, mn);
    return abs_le(__dsub_rn(x, xh), p.ebchk);
}

// When the first candidate needs no check.  With u = 2^-53, D = x - min >= 0,
// r = D / s and the three roundings of t = fma(RN(D), RN(1/s), 1/2):
// |q - r| <= 1/2 + e, e <= 3.01 u r + u/2; the reconstruction
// X = q s + min rounds to x^ with |x^ - X| <= u |X|, and the check's
// difference rounds once more.  So |RN(x - x^)| <= (s (1/2 + e) + u |X|)(1 + u).
// With s <= eb (63/32)(1 + u), r <= 2^40 (then e < 3.7e-4) and
// |X| <= max|x| + s <= eb (2^45 + 2) (then u |X| / eb < 0.0040), this is
// below 0.990 eb, under the threshold eb (1 - 2^-51) -- the 1/64 margin of
// the step absorbs the rounding.  eb >= 2^-1000 keeps every quantity normal
// (a subnormal difference is exact; a subnormal x^ errs by 2^-1075 at most).
__device__ __forceinline__ bool first_candidate_exact(double bmin, double bmax, const WideParams& p) {
    return p.eb >= 0x1p-1000 && __dsub_ru(bmax, bmin) <= p.s * 0x1p40 &&
           fmax(fabs(bmin), fabs(bmax)) <= p.eb * 0x1p45;
}

// Candidates q, q - 1, q + 1 (codes below 2^53); false when none passes.
__device__ __forceinline__ bool wide_quantise(double x, const WideParams& p, double mn, unsigned long long& q) {
    const double t = __fma_rn(__dsub_rn(x, mn), p.inv, 0.5);
    if (!(t < kWideLimitD)) return false;
    const unsigned long long q0 = code_floor(t);
    if (wide_ok(x, q0, p, mn)) {
        q = q0;
        return true;
    }
    if (q0 > 0ull && wide_ok(x, q0 - 1ull, p, mn)) {
        q = q0 - 1ull;
        return true;
    }
    if (q0 + 1ull < kWideLimit && wide_ok(x, q0 + 1ull, p, mn)) {
        q = q0 + 1ull;
        return true;
    }
    return false;
}

// ---------------------------------------------------------------- range pass

__global__ void __launch_bounds__(kWideThreads) gpz_wide_range_kernel(WideRangeArgs a) {
    const uint64_t stride = (uint64_t)gridDim.x * kWideThreads;
    const int lane = threadIdx.x & 31;
    for (int f = 0; f < a.F; ++f) {
        unsigned long long nmin = 0ull, kmax = 0ull;  // nmin = max of ~key
        for (uint64_t i = (uint64_t)blockIdx.x * kWideThreads + threadIdx.x; i < a.n; i += stride) {
            const double v = __ldcs(a.fields[f] + i);
            if (v == v) {
                const unsigned long long k = wide_key(v);
                nmin = max(nmin, ~k);
                kmax = max(kmax, k);
            }
        }
        nmin = warp_max_u64(nmin);
        kmax = warp_max_u64(kmax);
        if (lane == 0) {
            if (nmin) atomicMax(a.res + 2 * f, nmin);
            if (kmax) atomicMax(a.res + 2 * f + 1, kmax);
        }
    }
}

// ---------------------------------------------------------------- stages 1-3 per block

struct WideShared {
    unsigned long long nminkey[kMaxFields];  // max of ~key: the block minimum
    unsigned long long maxkey[kMaxFields];   // the block maximum
    unsigned long long maxq[kMaxFields];
    uint32_t flags, maxcnt, maxdelta;
    uint32_t warp_tot[kWideWarps], warp_nz[kWideWarps];
};

template <int F>
constexpr uint32_t wide_smem_bytes() {
    return 8u * F * kBlock + kWideWarps * kMaxBins * 2u + kMaxBins * 4u + kBlock * 2u + kWideDcWords * 4u;
}

// Appends the low w (<= 32) bits of v at increasing bit positions of zeroed
// shared words (a word shared with a neighbour's range is merged atomically).
struct WideAppender {
    unsigned long long acc;
    uint32_t nb, wi;
    __device__ __forceinline__ explicit WideAppender(uint32_t bitpos) : acc(0ull), nb(bitpos & 31u), wi(bitpos >> 5) {}
    __device__ __forceinline__ void put(uint32_t* sw, uint32_t v, uint32_t w) {
        acc |= (unsigned long long)v << nb;
        nb += w;
        if (nb >= 32u) {
            atomicOr(sw + wi, (uint32_t)acc);
            acc >>= 32;
            nb -= 32u;
            ++wi;
        }
    }
    __device__ __forceinline__ void finish(uint32_t* sw) {
        if (nb) atomicOr(sw + wi, (uint32_t)acc);
    }
};

template <int F>
__device__ __forceinline__ void wide_write_raw(const WideQseArgs& a, uint32_t b, int n_b, int t) {
    const uint64_t first = (uint64_t)b * kBlock;
    uint32_t* out = a.temp + (size_t)b * a.slot_words;
    if (t == 0) out[0] = 1u;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.fields[f] + first);
        for (int i = t; i < n_b; i += kWideThreads) {
            const unsigned long long u = __ldg(src + i);
            const uint32_t k = 1u + 2u * ((uint32_t)f * (uint32_t)n_b + (uint32_t)i);
            out[k] = (uint32_t)u;
            out[k + 1] = (uint32_t)(u >> 32);
        }
    }
    if (a.perm)
        for (int i = t; i < n_b; i += kWideThreads) a.perm[first + i] = (uint32_t)(first + i);
    if (t == 0) a.sizes[b] = 1u + 2u * (uint32_t)F * (uint32_t)n_b;
}

template <int F>
__global__ void __launch_bounds__(kWideThreads, F <= 6 ? 3 : 2) gpz_wide_qse_kernel(WideQseArgs a) {
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ WideShared S;
    constexpr int P = F < 3 ? F : 3;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t b = blockIdx.x;
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = (int)min((uint64_t)kBlock, a.n - first);
    unsigned long long* codes = reinterpret_cast<unsigned long long*>(dsm);  // [F][1024], sorted order
    uint16_t* hist = reinterpret_cast<uint16_t*>(dsm + 8u * F * kBlock);    // [8][512] per-warp counts
    uint16_t* uniq = hist + kWideWarps * kMaxBins;                           // [512]
    uint16_t* cnt = uniq + kMaxBins;                                         // [512]
    uint16_t* sperm = cnt + kMaxBins;                                        // [1024]
    uint32_t* dc = reinterpret_cast<uint32_t*>(sperm + kBlock);              // [kWideDcWords]
    uint32_t* out = a.temp + (size_t)b * a.slot_words;

    if (t < F) {
        S.nminkey[t] = 0ull;
        S.maxkey[t] = 0ull;
        S.maxq[t] = 0ull;
    }
    if (t == 0) {
        S.flags = 0u;
        S.maxcnt = 0u;
        S.maxdelta = 0u;
    }
    for (int k = t; k < kWideWarps * kMaxBins / 2; k += kWideThreads) reinterpret_cast<uint32_t*>(hist)[k] = 0u;
    for (int k = t; k < (int)kWideDcWords; k += kWideThreads) dc[k] = 0u;

    // ---- 1. load, non-finite values, block minima (order keys)
    bool valid[4];
    double x[F][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) valid[r] = 128 * w + 32 * r + lane < n_b;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const double* src = a.fields[f] + first + 128 * w + lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) x[f][r] = valid[r] ? __ldcs(src + 32 * r) : 0.0;
    }
    __syncthreads();  // shared slots initialised
    bool nonfinite = false;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        unsigned long long nk = 0ull, xk = 0ull;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (valid[r]) {
                const unsigned long long u = (unsigned long long)__double_as_longlong(x[f][r]);
                nonfinite |= ((u >> 52) & 0x7ffu) == 0x7ffu;  // infinite or NaN
                const unsigned long long k = wide_key(x[f][r]);
                nk = max(nk, ~k);
                xk = max(xk, k);
            }
        }
        nk = warp_max_u64(nk);
        xk = warp_max_u64(xk);
        if (lane == 0 && nk) {
            atomicMax(&S.nminkey[f], nk);
            atomicMax(&S.maxkey[f], xk);
        }
    }
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr(&S.flags, 1u);
    __syncthreads();
    if (S.flags & 1u) {
        wide_write_raw<F>(a, b, n_b, t);
        return;
    }
    // fields whose first candidates pass for certain (flag bit 2 + f)
    if (t < F) {
        double lo = 0.0, hi = 0.0;
        WideParams pf = a.params[0];
#pragma unroll
        for (int f = 0; f < F; ++f)
            if (f == t) {
                lo = wide_from_key(~S.nminkey[f]);
                hi = wide_from_key(S.maxkey[f]);
                pf = a.params[f];
            }
        if (first_candidate_exact(lo, hi, pf)) atomicOr(&S.flags, 4u << t);
    }
    __syncthreads();
    const uint32_t exact = S.flags >> 2;

    // ---- 2. codes with verification
    double mn[F];
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const double m = wide_from_key(~S.nminkey[f]);
        mn[f] = m == 0.0 ? 0.0 : m;  // a zero minimum is stored as +0
    }
    unsigned long long q[F][4];
    bool fail = false;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        unsigned long long qm = 0ull;
        if ((exact >> f) & 1u) {  // uniform over the block
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                q[f][r] = valid[r] ? code_floor(__fma_rn(__dsub_rn(x[f][r], mn[f]), a.params[f].inv, 0.5)) : 0ull;
                qm = max(qm, q[f][r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                q[f][r] = 0ull;
                if (valid[r]) {
                    fail |= !wide_quantise(x[f][r], a.params[f], mn[f], q[f][r]);
                    qm = max(qm, q[f][r]);
                }
            }
        }
        qm = warp_max_u64(qm);
        if (lane == 0 && qm) atomicMax(&S.maxq[f], qm);
    }
    if (__any_sync(0xffffffffu, fail) && lane == 0) atomicOr(&S.flags, 2u);
    __syncthreads();
    if (S.flags & 2u) {
        wide_write_raw<F>(a, b, n_b, t);
        return;
    }

    // ---- 3. widths, segments, key (Section 4.1)
    uint32_t bits[F], o[F], kshift[F], keybits = 0, W = 0;
    {
        uint32_t g[F], wf[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            bits[f] = bit_width64(S.maxq[f]);
            g[f] = f < P ? min((uint32_t)a.G, bits[f]) : 0u;
            o[f] = f < P ? bits[f] - g[f] : 0u;
            wf[f] = f < P ? o[f] : bits[f];
        }
#pragma unroll
        for (int f = F - 1; f >= 0; --f) {
            kshift[f] = keybits;
            keybits += g[f];
            W += wf[f];
        }
    }
    uint32_t key[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        uint32_t k = 0;
#pragma unroll
        for (int f = 0; f < P; ++f) k |= (uint32_t)(q[f][r] >> o[f]) << kshift[f];
        key[r] = k;
    }

    // ---- 4. stable counting sort by key (Section 4.2): warp-local ranks in storage order
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
    __syncthreads();

    // scan over (bin, warp): every bin's first sorted slot per warp, the runs
    const int nbins = 1 << keybits;
    const int b0 = 2 * t;
    uint32_t c0 = 0, c1 = 0;
    uint32_t pre[kWideWarps];
    if (b0 < nbins) {
#pragma unroll
        for (int ww = 0; ww < kWideWarps; ++ww) {
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
    __syncthreads();
    uint32_t base_tot = 0, base_nz = 0, U = 0;
#pragma unroll
    for (int ww = 0; ww < kWideWarps; ++ww) {
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
        const uint32_t base2 = start0 | (start1 << 16);
#pragma unroll
        for (int ww = 0; ww < kWideWarps; ++ww)
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
    __syncthreads();

    // scatter the codes to sorted order; the largest delta of the unique ids
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (!valid[r]) continue;
        const uint32_t dest = myhist[key[r]] + rank[r];
#pragma unroll
        for (int f = 0; f < F; ++f)
            codes[f * kBlock + dest] = f < P ? (q[f][r] & mask64(o[f])) : q[f][r];
        sperm[dest] = (uint16_t)(128 * w + 32 * r + lane);
    }
    {
        uint32_t dmax = 0;
        for (uint32_t k = t; k < U; k += kWideThreads)
            dmax = max(dmax, (uint32_t)uniq[k] - (k ? (uint32_t)uniq[k - 1] : 0u));
        dmax = __reduce_max_sync(0xffffffffu, dmax);
        if (lane == 0 && dmax) atomicMax(&S.maxdelta, dmax);
    }
    __syncthreads();

    // ---- 5. sizes; raw when the encoding is not smaller
    const uint32_t wd = bit_width(S.maxdelta), wc = bit_width(S.maxcnt);
    const uint32_t hdr = 1u + 2u * (uint32_t)F + (uint32_t)((F + 3) >> 2);
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = ceil_words((uint32_t)n_b * W);
    const uint32_t enc = hdr + dwords + cwords + rwords;
    if (enc >= 1u + 2u * (uint32_t)F * (uint32_t)n_b) {
        wide_write_raw<F>(a, b, n_b, t);
        return;
    }

    // ---- 6. block header, deltas and counts (Section 4.3)
    if (t == 0) out[0] = (U << 1) | (wd << 12) | (wc << 17);
    if (t < 2 * F) {
        double m = 0.0;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if (f == (t >> 1)) m = mn[f];
        const unsigned long long u = (unsigned long long)__double_as_longlong(m);
        out[1 + t] = (t & 1) ? (uint32_t)(u >> 32) : (uint32_t)u;
    }
    if (t < ((F + 3) >> 2)) {
        uint32_t word = 0;
#pragma unroll
        for (int f = 0; f < F; ++f)
            if ((f >> 2) == t) word |= bits[f] << (8 * (f & 3));
        out[1 + 2 * F + t] = word;
    }
    {
        const uint32_t k0 = 2u * (uint32_t)t;
        if (k0 < U && wd) {
            WideAppender ap(k0 * wd);
            ap.put(dc, (uint32_t)uniq[k0] - (k0 ? (uint32_t)uniq[k0 - 1] : 0u), wd);
            if (k0 + 1 < U) ap.put(dc, (uint32_t)uniq[k0 + 1] - (uint32_t)uniq[k0], wd);
            ap.finish(dc);
        }
        if (k0 < U && wc) {
            WideAppender ap(32u * dwords + k0 * wc);
            ap.put(dc, (uint32_t)cnt[k0], wc);
            if (k0 + 1 < U) ap.put(dc, (uint32_t)cnt[k0 + 1], wc);
            ap.finish(dc);
        }
    }
    __syncthreads();
    for (uint32_t k = t; k < dwords + cwords; k += kWideThreads) out[hdr + k] = dc[k];

    // ---- 7. record words: record j at stream bits [jW, jW + W) of the
    // record array, field F-1 least significant
    uint32_t wfv[F], rshift[F];
    {
        uint32_t rs = 0;
#pragma unroll
        for (int f = F - 1; f >= 0; --f) {
            wfv[f] = f < P ? o[f] : bits[f];
            rshift[f] = rs;
            rs += wfv[f];
        }
    }
    uint32_t* rout = out + hdr + dwords + cwords;
    if (W >= 8u) {
        // Thread t appends sorted records 4t..4t+3 (bits [4tW, 4tW + 4W), at
        // least 32 of them) into staging words that reuse the codes' space.
        // It writes the words inside its range itself; its first word (shared
        // with the left neighbour) and its unfinished last word (shared with
        // the right one) go to an exchange area in the histograms' space and
        // are merged after a barrier.  Every staging word is written once.
        const int j0 = 4 * t;
        const bool act = j0 < n_b;
        const int nrec = act ? min(4, n_b - j0) : 0;
        unsigned long long c[4][F];
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int f = 0; f < F; ++f) c[e][f] = e < nrec ? codes[f * kBlock + j0 + e] : 0ull;
        __syncthreads();  // every code read: their space becomes the staging words
        uint32_t* stage = reinterpret_cast<uint32_t*>(codes);  // 2048 F words >= ceil(1024 x 53 F / 32)
        uint32_t* xl = reinterpret_cast<uint32_t*>(hist);      // first word, when finished here
        uint32_t* xls = xl + kWideThreads;                      // ... and whether it was
        uint32_t* xr = xls + kWideThreads;                      // unfinished last word
        uint32_t* xri = xr + kWideThreads;                      // ... and its index (or none)
        constexpr uint32_t kNone = 0xffffffffu;
        const uint32_t start = (uint32_t)j0 * W;
        const uint32_t w0 = start >> 5;
        uint32_t nb = start & 31u, wi = w0, first_done = 0u;
        unsigned long long acc = 0ull;
        auto put = [&](uint32_t v, uint32_t w) {  // w <= 32, nb < 32 on entry
            acc |= (unsigned long long)v << nb;
            nb += w;
            if (nb >= 32u) {
                const uint32_t word = (uint32_t)acc;
                if (wi == w0) {
                    xl[t] = word;
                    first_done = 1u;
                } else {
                    stage[wi] = word;
                }
                acc >>= 32;
                nb -= 32u;
                ++wi;
            }
        };
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e >= nrec) break;
#pragma unroll
            for (int f = F - 1; f >= 0; --f) {
                const uint32_t w = wfv[f];
                const unsigned long long v = c[e][f];
                if (w > 32u) {
                    put((uint32_t)v, 32u);
                    put((uint32_t)(v >> 32), w - 32u);
                } else if (w) {
                    put((uint32_t)v, w);
                }
            }
        }
        xls[t] = first_done;
        xri[t] = (act && nb) ? wi : kNone;
        xr[t] = (uint32_t)acc;
        __syncthreads();
        if (act) {
            uint32_t val = first_done ? xl[t] : 0u;
            if (t > 0 && xri[t - 1] == w0) val |= xr[t - 1];
            const uint32_t last = xri[t];
            if (last == w0) val |= xr[t];
            stage[w0] = val;
            const bool next_act = j0 + 4 < n_b;
            if (last != kNone && last != w0 && !next_act) stage[last] = xr[t];  // no right neighbour takes it
        }
        __syncthreads();
        for (uint32_t k = t; k < rwords; k += kWideThreads) rout[k] = stage[k];
    } else {
        // short records: word k gathered from the codes of the records it overlaps
        for (uint32_t k = t; k < rwords; k += kWideThreads) {
            const uint32_t lo = 32u * k;
            uint32_t acc = 0;
            for (uint32_t j = lo / W; j < (uint32_t)n_b && j * W < lo + 32u; ++j) {
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    if (wfv[f] == 0u) continue;
                    const int s0 = (int)(j * W + rshift[f]) - (int)lo;
                    if (s0 >= 32 || s0 + (int)wfv[f] <= 0) continue;
                    const unsigned long long v = codes[f * kBlock + j];
                    acc |= s0 >= 0 ? (uint32_t)(v << s0) : (uint32_t)(v >> -s0);
                }
            }
            rout[k] = acc;
        }
    }
    if (a.perm)
        for (int j = t; j < n_b; j += kWideThreads) a.perm[first + j] = (uint32_t)first + sperm[j];
    if (t == 0) a.sizes[b] = enc;
}

// ---------------------------------------------------------------- decompression

struct WideDecShared {
    double mn[kMaxFields], s[kMaxFields];
    uint32_t g[kMaxFields], o[kMaxFields], wf[kMaxFields], kshift[kMaxFields], rshift[kMaxFields];
    uint16_t uniq[kMaxBins];
    uint32_t mask[32], warp_uc[kWideWarps];
    uint32_t ok, raw, bad, U, wd, wc, W, keybits, off, nw;
};

// w (<= 32) bits at bit position pos of A[0..len); 0 when w = 0.
__device__ __forceinline__ uint32_t wide_get(const uint32_t* A, uint32_t len, uint32_t pos, uint32_t w) {
    if (w == 0u) return 0u;
    const uint32_t wi = pos >> 5, sh = pos & 31u;
    const uint32_t lo = wi < len ? __ldg(A + wi) : 0u;
    const uint32_t hi = (sh + w > 32u && wi + 1u < len) ? __ldg(A + wi + 1u) : 0u;
    return __funnelshift_r(lo, hi, sh) & (w >= 32u ? 0xffffffffu : ((1u << w) - 1u));
}

// w (<= 53) bits at bit position pos of the staged record words; the two
// words after the array keep the reads in bounds (bits read past the array
// lie above the field and are masked off).
__device__ __forceinline__ unsigned long long wide_get64_s(const uint32_t* A, uint32_t pos, uint32_t w) {
    if (w == 0u) return 0ull;  // (a zero-width field may sit at the very end of the array)
    const uint32_t wi = pos >> 5, sh = pos & 31u;
    const unsigned long long lo = (unsigned long long)A[wi] | ((unsigned long long)A[wi + 1] << 32);
    const unsigned long long hi = A[wi + 2];
    const unsigned long long v = sh ? ((lo >> sh) | (hi << (64u - sh))) : lo;
    return v & mask64(w);
}

// Staged record words of one block: at most ceil(1024 x 53 F / 32), plus two.
template <int F>
constexpr uint32_t wide_dec_smem_bytes() {
    return 4u * ((kBlock * kWideMaxBits * (uint32_t)F + 31u) / 32u + 2u);
}

template <int F>
__global__ void __launch_bounds__(kWideThreads) gpz_wide_decode_kernel(WideDecArgs a) {
    __shared__ WideDecShared S;
    extern __shared__ __align__(16) uint32_t srec[];  // the block's record words
    constexpr int P = F < 3 ? F : 3;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const uint32_t* Sw = a.stream;
    const uint32_t b = blockIdx.x;
    const uint64_t first = (uint64_t)b * kBlock;
    const int n_b = (int)min((uint64_t)kBlock, a.n - first);
    const uint64_t table_start = kHeaderWords + 4ull * F;
    const uint64_t payload_start = table_start + a.nblocks + 1;
    const uint32_t hdr = 1u + 2u * (uint32_t)F + (uint32_t)((F + 3) >> 2);
    if (t < 32) S.mask[t] = 0u;
    if (t == 0) S.bad = 0u;

    // ---- 1. warp 0: the stream header, the block's place, its header
    if (w == 0) {
        const uint32_t hv = lane < kHeaderWords ? __ldg(Sw + lane) : 0u;  // the host checked total_words >= 16
        const bool header_fits = payload_start <= a.total_words;
        const uint32_t payload_words = __shfl_sync(0xffffffffu, hv, 9);
        uint32_t off = 0, end = 0;
        if (header_fits) {
            off = __ldg(Sw + table_start + b);
            end = __ldg(Sw + table_start + b + 1);
        }
        const bool inside =
            header_fits && payload_start + payload_words <= a.total_words && off <= end && end <= payload_words;
        bool ok = true;
        switch (lane) {
            case 0: ok = hv == kMagic; break;
            case 1: ok = hv == 2u; break;
            case 2: ok = hv == (uint32_t)F; break;
            case 3: ok = hv <= (uint32_t)kMaxSegBits; break;
            case 4: ok = hv == (uint32_t)kBlock; break;
            case 5: ok = hv <= 1u; break;
            case 6: ok = hv == (uint32_t)(a.n & 0xffffffffull); break;
            case 7: ok = hv == (uint32_t)(a.n >> 32); break;
            case 8: ok = hv == a.nblocks; break;
            case 9: break;
            default: ok = lane >= kHeaderWords || hv == 0u; break;
        }
        const uint32_t G = __shfl_sync(0xffffffffu, hv, 3);
        ok = __all_sync(0xffffffffu, ok) && inside && !(b == 0 && off != 0) &&
             !(b + 1 == a.nblocks && end != payload_words) && end != off;
        const uint32_t nw = end - off;
        const uint32_t* blk = Sw + payload_start + off;
        const uint32_t bw = (ok && (uint32_t)lane < min(hdr, nw)) ? __ldg(blk + lane) : 0u;
        const uint32_t mode = __shfl_sync(0xffffffffu, bw, 0);
        const bool raw = ok && (mode & 1u);
        if (raw) ok = mode == 1u && nw == 1u + 2u * (uint32_t)F * (uint32_t)n_b;
        const bool fl = lane < F;
        const uint32_t mlo = __shfl_sync(0xffffffffu, bw, (1 + 2 * lane) & 31);
        const uint32_t mhi = __shfl_sync(0xffffffffu, bw, (2 + 2 * lane) & 31);
        const uint32_t wword = __shfl_sync(0xffffffffu, bw, (1 + 2 * F + (lane >> 2)) & 31);
        const uint32_t bits = fl ? (wword >> (8 * (lane & 3))) & 0xffu : 0u;
        const uint32_t bf = bits <= kWideMaxBits ? bits : 0u;
        const uint32_t g = lane < P ? min(G, bf) : 0u;
        const uint32_t wf = fl ? (lane < P ? bf - g : bf) : 0u;
        uint32_t U = 0, wd = 0, wc = 0, W = 0, keybits = 0;
        if (ok && !raw) {
            U = (mode >> 1) & 0x7ffu;
            wd = (mode >> 12) & 31u;
            wc = (mode >> 17) & 31u;
            ok = (mode >> 22) == 0u && nw >= hdr && !__any_sync(0xffffffffu, fl && bits > kWideMaxBits);
            const uint32_t lastw = __shfl_sync(0xffffffffu, bw, (hdr - 1) & 31);
            if ((F & 3) != 0) ok = ok && (lastw >> (8 * (F & 3))) == 0u;
            keybits = __reduce_add_sync(0xffffffffu, g);
            W = __reduce_add_sync(0xffffffffu, wf);
            ok = ok && U >= 1u && U <= (uint32_t)n_b && U <= (1u << keybits) && wd <= keybits && wc <= 11u &&
                 (uint64_t)nw == (uint64_t)hdr + ceil_words(U * wd) + ceil_words(U * wc) +
                                      ((uint64_t)n_b * W + 31u) / 32u;
        }
        if (fl) {
            S.mn[lane] = __longlong_as_double((long long)(((unsigned long long)mhi << 32) | mlo));
            S.s[lane] = header_fits ? __longlong_as_double((long long)(((unsigned long long)__ldg(
                                                                             Sw + kHeaderWords + 4 * lane + 3)
                                                                         << 32) |
                                                                        __ldg(Sw + kHeaderWords + 4 * lane + 2)))
                                    : 0.0;
            S.g[lane] = g;
            S.o[lane] = lane < P ? bf - g : 0u;
            S.wf[lane] = wf;
        }
        __syncwarp();
        if (fl) {
            uint32_t ks = 0, rs = 0;
            for (int f = F - 1; f > lane; --f) {
                ks += S.g[f];
                rs += S.wf[f];
            }
            S.kshift[lane] = ks;
            S.rshift[lane] = rs;
        }
        if (lane == 0) {
            S.ok = ok;
            S.raw = raw;
            S.U = U;
            S.wd = wd;
            S.wc = wc;
            S.W = W;
            S.keybits = keybits;
            S.off = off;
            S.nw = nw;
        }
    }
    __syncthreads();
    if (!S.ok) {
        if (t == 0) set_status(a.status, kStCorrupt);
        return;
    }
    const uint32_t* blk = Sw + payload_start + S.off;
    if (S.raw) {
#pragma unroll
        for (int f = 0; f < F; ++f)
            for (int i = t; i < n_b; i += kWideThreads) {
                const uint32_t k = 1u + 2u * ((uint32_t)f * (uint32_t)n_b + (uint32_t)i);
                const unsigned long long u = ((unsigned long long)__ldg(blk + k + 1) << 32) | __ldg(blk + k);
                a.out[f][first + i] = __longlong_as_double((long long)u);
            }
        return;
    }

    // ---- 2. unique ids and run starts (Section 4.3, undone); the record
    // words are copied to shared memory meanwhile (visible after the barriers)
    const uint32_t U = S.U, wd = S.wd, wc = S.wc, W = S.W, keybits = S.keybits;
    const uint32_t dwords = ceil_words(U * wd), cwords = ceil_words(U * wc);
    const uint32_t rwords = S.nw - hdr - dwords - cwords;  // <= ceil(n_b W / 32) by the size check
    const uint32_t idlimit = 1u << keybits;
    {
        const uint32_t* R = blk + hdr + dwords + cwords;
        for (uint32_t k = t; k < rwords; k += kWideThreads) srec[k] = __ldg(R + k);
    }
    {
        const uint32_t* D = blk + hdr;
        const uint32_t* Cc = D + dwords;
        const uint32_t k0 = 2u * t, k1 = k0 + 1u;
        const bool v0 = k0 < U, v1 = k1 < U;
        uint32_t d0 = v0 ? wide_get(D, dwords, k0 * wd, wd) : 0u, d1 = v1 ? wide_get(D, dwords, k1 * wd, wd) : 0u;
        uint32_t c0 = v0 ? wide_get(Cc, cwords, k0 * wc, wc) : 0u, c1 = v1 ? wide_get(Cc, cwords, k1 * wc, wc) : 0u;
        bool bad = (v0 && (d0 >= idlimit || c0 == 0u || c0 > (uint32_t)n_b || (k0 > 0 && d0 == 0u))) ||
                   (v1 && (d1 >= idlimit || c1 == 0u || c1 > (uint32_t)n_b || d1 == 0u));
        if (bad) d0 = d1 = c0 = c1 = 0u;
        const uint32_t su = d0 + d1, sc = c0 + c1;
        const uint32_t iuc = warp_incl_sum(su | (sc << 15));  // ids < 2^15 and counts <= 2^16 per warp
        const uint32_t iu = iuc & 0x7fffu, ic = iuc >> 15;
        if (lane == 31) S.warp_uc[w] = iuc;
        __syncthreads();
        uint32_t bu = 0, bc = 0, total = 0;
#pragma unroll
        for (int ww = 0; ww < kWideWarps; ++ww) {
            const uint32_t uc = S.warp_uc[ww];
            if (ww < w) {
                bu += uc & 0x7fffu;
                bc += uc >> 15;
            }
            total += uc >> 15;
        }
        const uint32_t u0 = bu + iu - su + d0, u1 = u0 + d1;
        const uint32_t s0 = bc + ic - sc, s1 = s0 + c0;
        if (v0) {
            if (u0 >= idlimit || s0 >= (uint32_t)n_b) {
                bad = true;
            } else {
                S.uniq[k0] = (uint16_t)u0;
                atomicOr(&S.mask[s0 >> 5], 1u << (s0 & 31u));
            }
        }
        if (v1) {
            if (u1 >= idlimit || s1 >= (uint32_t)n_b) {
                bad = true;
            } else {
                S.uniq[k1] = (uint16_t)u1;
                atomicOr(&S.mask[s1 >> 5], 1u << (s1 & 31u));
            }
        }
        if (t == 0 && total != (uint32_t)n_b) bad = true;
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&S.bad, 1u);
    }
    __syncthreads();
    if (S.bad) {
        if (t == 0) set_status(a.status, kStCorrupt);
        return;
    }
    // every warp scans the 32 mask words itself: lane i holds word i and the
    // run starts before it
    const uint32_t mword = S.mask[lane];
    const uint32_t mpc = __popc(mword);
    const uint32_t mpre = warp_incl_sum(mpc) - mpc;

    // ---- 3. positions 4t..4t+3: run, key, record fields, q = segId * 2^o + segOffset
    // thread t's four positions lie in mask word t/8 (every lane shuffles)
    const int src = (t >> 3) & 31;
    const uint32_t mrow = __shfl_sync(0xffffffffu, mword, src), prow = __shfl_sync(0xffffffffu, mpre, src);
    const int j0 = 4 * t;
    if (j0 >= n_b) return;
    const int left = n_b - j0;
    uint32_t key[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t bit = (uint32_t)(j0 + e) & 31u;
        int run = (int)(prow + __popc(mrow & ((2u << bit) - 1u))) - 1;
        run = run < 0 ? 0 : (run >= (int)U ? (int)U - 1 : run);
        key[e] = S.uniq[run];
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const uint32_t wf = S.wf[f], rs = S.rshift[f], ks = S.kshift[f], gm = (1u << S.g[f]) - 1u, of = S.o[f];
        const double sf = S.s[f], mf = S.mn[f];
        double v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t j = (uint32_t)min(j0 + e, n_b - 1);  // positions past the block repeat the last
            unsigned long long qv = wide_get64_s(srec, j * W + rs, wf);
            if (f < P) qv |= (unsigned long long)((key[e] >> ks) & gm) << of;
            v[e] = __fma_rn(code_to_double(qv), sf, mf);  // qv < 2^53
        }
        double* dst = a.out[f] + first + j0;
        if (left >= 4 && (reinterpret_cast<uintptr_t>(a.out[f]) & 15u) == 0) {
            reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
            reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e < left) dst[e] = v[e];
        }
    }
}

// ---------------------------------------------------------------- launches

template <int F>
cudaError_t launch_wide_qse_f(const WideQseArgs& a, uint32_t nblocks, cudaStream_t s) {
    constexpr uint32_t smem = wide_smem_bytes<F>();
    // set at every launch (the attributes belong to the current device), with
    // the largest shared-memory carveout so that three CTAs fit per SM
    cudaError_t e = cudaFuncSetAttribute(gpz_wide_qse_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gpz_wide_qse_kernel<F>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    gpz_wide_qse_kernel<F><<<nblocks, kWideThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int F>
cudaError_t launch_wide_dec_f(const WideDecArgs& a, cudaStream_t s) {
    constexpr uint32_t smem = wide_dec_smem_bytes<F>();
    cudaError_t e = cudaFuncSetAttribute(gpz_wide_decode_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gpz_wide_decode_kernel<F>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    gpz_wide_decode_kernel<F><<<a.nblocks, kWideThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wide_qse(const WideQseArgs& a, uint32_t nblocks, cudaStream_t s) {
    switch (a.F) {
        case 1: return launch_wide_qse_f<1>(a, nblocks, s);
        case 2: return launch_wide_qse_f<2>(a, nblocks, s);
        case 3: return launch_wide_qse_f<3>(a, nblocks, s);
        case 4: return launch_wide_qse_f<4>(a, nblocks, s);
        case 5: return launch_wide_qse_f<5>(a, nblocks, s);
        case 6: return launch_wide_qse_f<6>(a, nblocks, s);
        case 7: return launch_wide_qse_f<7>(a, nblocks, s);
        case 8: return launch_wide_qse_f<8>(a, nblocks, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_wide_decode(const WideDecArgs& a, cudaStream_t s) {
    switch (a.F) {
        case 1: return launch_wide_dec_f<1>(a, s);
        case 2: return launch_wide_dec_f<2>(a, s);
        case 3: return launch_wide_dec_f<3>(a, s);
        case 4: return launch_wide_dec_f<4>(a, s);
        case 5: return launch_wide_dec_f<5>(a, s);
        case 6: return launch_wide_dec_f<6>(a, s);
        case 7: return launch_wide_dec_f<7>(a, s);
        case 8: return launch_wide_dec_f<8>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gpz

// ---------------------------------------------------------------- host side

namespace {

constexpr uint64_t kWideAlign = 256;
constexpr uint64_t kWideCtrlBytes = 256;  // words: 0 status, 1 scan tile counter, 4-5 out size
constexpr uint64_t kWideResBytes = 256;   // range pass: [8][2] order keys

uint32_t wide_slot_words(int F) { return (uint32_t)align_up(1ull + 2ull * (uint64_t)F * kBlock, 4); }

struct WideLayout {
    uint64_t ctrl, res, states, sizes, temp, total, zero_bytes;
};

WideLayout wide_layout(uint64_t n, int F) {
    WideLayout L{};
    const uint64_t nb = nblocks_of(n);
    uint64_t o = 0;
    L.ctrl = o;
    o += kWideCtrlBytes;
    L.res = o;
    o += kWideResBytes;
    L.states = o;
    o += align_up((nb + 1 + kScanTile - 1) / kScanTile * 8ull, kWideAlign);
    L.zero_bytes = o;  // ctrl, range results and scan states are cleared per call
    L.sizes = o;
    o += align_up(nb * 4ull, kWideAlign);
    L.temp = o;
    o += align_up(nb * wide_slot_words(F) * 4ull, kWideAlign);
    L.total = o;
    return L;
}

// The constants of one field (each one IEEE double operation).
WideParams wide_params(double eb) {
    WideParams p;
    p.eb = eb;
    const volatile double s = eb * 1.96875;
    p.s = s;
    const volatile double inv = 1.0 / p.s;
    p.inv = inv;
    p.ebchk = std::nextafter(std::nextafter(eb, 0.0), 0.0);
    return p;
}

double wide_from_key_host(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
}

gpz_status wide_read_status(uint32_t* status, cudaStream_t s) {
    uint32_t st = 0;
    if (cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return GPZ_ERR_CUDA;
    return (gpz_status)st;
}

bool wide_fields_ok(const double* const* d_fields, uint64_t n, int F) {
    if (n == 0) return true;
    if (!d_fields) return false;
    for (int f = 0; f < F; ++f)
        if (!d_fields[f] || !aligned(d_fields[f], 8)) return false;
    return true;
}

}  // namespace

namespace gpz {
namespace host {

uint64_t wide_workspace_size(uint64_t n, int F) {
    if (F < 1 || F > kMaxFields) return 0;
    return wide_layout(n, F).total;
}

// Stages, scan and copy of the 64-bit form with absolute bounds eb[f]; the
// header's mode word is `mode` (the caller's bound mode).
gpz_status wide_compress(const double* const* d_fields, uint64_t n, int F, int G, int mode, const double* eb,
                         void* d_out, uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size,
                         uint32_t* d_perm, void* d_ws, uint64_t ws_size, cudaStream_t s) {
    const uint64_t nb = nblocks_of(n);
    if (nb + 2ull * (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    if (out_capacity < gpz_bound_size_wide(n, F)) return GPZ_ERR_CAPACITY;
    const WideLayout L = wide_layout(n, F);
    if (ws_size < L.total) return GPZ_ERR_CAPACITY;
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.ctrl);
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return GPZ_ERR_CUDA;
    Recorder rec(s);
    rec.begin(3);
    WideQseArgs qa{};
    for (int f = 0; f < F; ++f) {
        qa.fields[f] = n ? d_fields[f] : nullptr;
        qa.params[f] = wide_params(eb[f]);
    }
    qa.n = n;
    qa.F = F;
    qa.G = G;
    qa.temp = reinterpret_cast<uint32_t*>(ws + L.temp);
    qa.slot_words = wide_slot_words(F);
    qa.sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
    qa.perm = d_perm;
    if (nb > 0) {
        if (launch_wide_qse(qa, (uint32_t)nb, s) != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("wide_qse");
    }
    const uint32_t table_start = (uint32_t)(kHeaderWords + 4 * F);
    uint32_t* stream_words = static_cast<uint32_t*>(d_out);
    ScanArgs sa{};
    sa.sizes = qa.sizes;
    sa.nblocks = (uint32_t)nb;
    sa.n = n;
    sa.F = 2 * F;  // a raw block holds 1 + 2F n_b words
    sa.table = stream_words + table_start;
    sa.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
    sa.tile_counter = status + 1;
    sa.status = status;
    if (launch_scan(sa, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("scan");
    CompactArgs ca{};
    ca.temp = qa.temp;
    ca.slot_words = qa.slot_words;
    ca.sizes = qa.sizes;
    ca.table = sa.table;
    ca.stream = stream_words;
    ca.payload_start = (uint32_t)(table_start + nb + 1);
    ca.nblocks = (uint32_t)nb;
    ca.n = n;
    ca.F = F;
    ca.G = G;
    ca.mode = mode;
    ca.d_out_size = d_out_size ? reinterpret_cast<unsigned long long*>(d_out_size)
                               : reinterpret_cast<unsigned long long*>(ws + L.ctrl + 16);
    ca.version = 2;
    ca.ext_words = 4u * (uint32_t)F;
    for (int f = 0; f < F; ++f) {
        unsigned long long e, st;
        std::memcpy(&e, &qa.params[f].eb, 8);
        std::memcpy(&st, &qa.params[f].s, 8);
        ca.ext[4 * f] = (uint32_t)e;
        ca.ext[4 * f + 1] = (uint32_t)(e >> 32);
        ca.ext[4 * f + 2] = (uint32_t)st;
        ca.ext[4 * f + 3] = (uint32_t)(st >> 32);
    }
    if (launch_compact(ca, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("compact");
    if (h_out_size) {
        if (cudaMemcpyAsync(h_out_size, ca.d_out_size, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return GPZ_ERR_CUDA;
        return wide_read_status(status, s);
    }
    return GPZ_OK;
}

}  // namespace host
}  // namespace gpz

extern "C" {

uint64_t gpz_bound_size_wide(uint64_t n, int F) {
    if (F < 1 || F > kMaxFields) return 0;
    const uint64_t nb = nblocks_of(n);
    return 4ull * (kHeaderWords + 4ull * F + (nb + 1) + nb + 2ull * (uint64_t)F * n);
}

uint64_t gpz_compress_wide_workspace_size(uint64_t n, int F) { return wide_workspace_size(n, F); }

gpz_status gpz_compress_wide(const double* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                             uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                             void* d_ws, uint64_t ws_size, double* h_eb_used, void* stream) {
    if (!p || !d_out || !aligned(d_out, 4) || !d_ws || !aligned(d_ws, kWideAlign)) return GPZ_ERR_INVALID_ARG;
    const int F = p->n_fields;
    if (F < 1 || F > kMaxFields || p->seg_bits < 0 || p->seg_bits > kMaxSegBits ||
        (p->mode != GPZ_EB_ABS && p->mode != GPZ_EB_REL))
        return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F; ++f)
        if (!(p->eb[f] > 0.0) || !std::isfinite(p->eb[f])) return GPZ_ERR_INVALID_ARG;
    if (!wide_fields_ok(d_fields, n, F) || (d_perm && !aligned(d_perm, 4))) return GPZ_ERR_INVALID_ARG;
    const WideLayout L = wide_layout(n, F);
    if (ws_size < L.total) return GPZ_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    double eb[kMaxFields];
    for (int f = 0; f < F; ++f) eb[f] = p->eb[f];
    if (p->mode == GPZ_EB_REL && n > 0) {
        // the fp64 range of the non-NaN values (one synchronisation)
        uint8_t* ws = static_cast<uint8_t*>(d_ws);
        unsigned long long* res = reinterpret_cast<unsigned long long*>(ws + L.res);
        if (cudaMemsetAsync(res, 0, kWideResBytes, s) != cudaSuccess) return GPZ_ERR_CUDA;
        WideRangeArgs ra{};
        for (int f = 0; f < F; ++f) ra.fields[f] = d_fields[f];
        ra.n = n;
        ra.F = F;
        ra.res = res;
        const uint64_t want = (n + kWideThreads - 1) / kWideThreads;
        const unsigned grid = (unsigned)(want < 152ull * 8ull ? want : 152ull * 8ull);
        Recorder rec(s);
        rec.begin(1);
        gpz_wide_range_kernel<<<grid, kWideThreads, 0, s>>>(ra);
        if (cudaGetLastError() != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("wide_range");
        unsigned long long got[2 * kMaxFields];
        if (cudaMemcpyAsync(got, res, 16ull * F, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GPZ_ERR_CUDA;
        for (int f = 0; f < F; ++f) {
            if (got[2 * f] == 0ull) continue;  // every value NaN: the bound stays rel
            const volatile double range = wide_from_key_host(got[2 * f + 1]) - wide_from_key_host(~got[2 * f]);
            if (range > 0.0 && std::isfinite(range)) {
                const volatile double t = p->eb[f] * range;
                if (t > 0.0 && std::isfinite(t)) eb[f] = t;
            }
        }
    }
    if (h_eb_used)
        for (int f = 0; f < F; ++f) h_eb_used[f] = eb[f];
    return wide_compress(d_fields, n, F, p->seg_bits, p->mode, eb, d_out, out_capacity, d_out_size, h_out_size,
                         d_perm, d_ws, ws_size, s);
}

gpz_status gpz_decompress_wide(const void* d_in, uint64_t in_size, double* const* d_fields, int F, uint64_t n,
                               void* d_ws, uint64_t ws_size, void* stream) {
    if (!d_in || !aligned(d_in, 4) || F < 1 || F > kMaxFields || !d_ws || !aligned(d_ws, 16))
        return GPZ_ERR_INVALID_ARG;
    if (ws_size < gpz_decompress_workspace_size()) return GPZ_ERR_CAPACITY;
    if (!wide_fields_ok(const_cast<const double* const*>(d_fields), n, F)) return GPZ_ERR_INVALID_ARG;
    if (in_size % 4 != 0 || in_size < 4ull * kHeaderWords) return GPZ_ERR_CORRUPT;
    const uint64_t nb = nblocks_of(n);
    if (nb + 2ull * (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* status = static_cast<uint32_t*>(d_ws);
    if (cudaMemsetAsync(status, 0, 4, s) != cudaSuccess) return GPZ_ERR_CUDA;
    if (nb == 0) return GPZ_OK;
    WideDecArgs da{};
    da.stream = static_cast<const uint32_t*>(d_in);
    da.total_words = in_size / 4;
    for (int f = 0; f < F; ++f) da.out[f] = d_fields[f];
    da.n = n;
    da.F = F;
    da.nblocks = (uint32_t)nb;
    da.status = status;
    Recorder rec(s);
    rec.begin(1);
    if (launch_wide_decode(da, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("wide_decompress");
    return GPZ_OK;
}

}  // extern "C"
