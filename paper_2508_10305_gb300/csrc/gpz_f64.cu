// gpz_f64.cu -- fp64 input and output (Section 5.1: the paper down-casts fp64
// input to fp32 when that suffices for the error bound; otherwise the 64-bit
// form of gpz_wide.cu, Section 5.2).  Compression rounds every value to fp32 on the GPU and
// compresses the fp32 values with each field's bound reduced by the largest
// rounding error over its finite values, eb' = eb - max |x - RN32(x)|, so
// that every decompressed value lies within eb of its fp64 input.  One
// prepass kernel writes the fp32 copy (in the workspace) and finds, per
// field, the fp64 extremes of the non-NaN values and the largest rounding
// error; the host reads those (the call synchronises once), forms eb' (a
// relative bound is taken over the fp64 range) and calls gpz_compress with
// absolute bounds on the copy -- or, when some eb' is not positive, calls the
// 64-bit form with the bounds eb.  Decompression of a version-1 stream runs
// the block decoder storing fp64 (each value widened exactly from its fp32
// reconstruction); a version-2 stream goes to gpz_decompress_wide.
#include <cmath>
#include <cstring>

#include "gpz.h"
#include "gpz_host.hpp"
#include "gpz_internal.cuh"

using namespace gpz;
using namespace gpz::host;

namespace gpz {

constexpr int kF64Threads = 256;

// Order key of a double: unsigned order equals numeric order (NaN excluded).
__device__ __forceinline__ unsigned long long order_key64(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// res[3f] = order key of the field's minimum, res[3f+1] of its maximum (over
// the non-NaN values), res[3f+2] = bits of the largest |x - RN32(x)| over
// the finite values (non-negative, so its bits order as the value).
// res must start as {~0, 0, 0} per field.
__global__ void __launch_bounds__(kF64Threads) gpz_f64_prepass_kernel(F64Args a) {
    __shared__ unsigned long long s_res[kF64Threads / 32][3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * kF64Threads;
    for (int f = 0; f < a.F; ++f) {
        const double* x = a.in[f];
        float* y = a.out32[f];
        unsigned long long kmin = ~0ull, kmax = 0ull, dmax = 0ull;
        auto round1 = [&](double v) -> float {
            const unsigned long long u = (unsigned long long)__double_as_longlong(v);
            const int e = (int)((u >> 52) & 0x7ffu);
            const int e32 = e - 1023 + 127;
            if (e32 >= 1 && e32 <= 254) {
                // fp32-normal magnitude: round to nearest even on the bits, and
                // the rounding error |v - r| = |rem - (up ? 2^29 : 0)| * 2^(e-1075)
                // (exact in double) as its bit pattern, with integer operations
                const unsigned long long m = u & 0xfffffffffffffull;
                const uint32_t m24 = (uint32_t)(m >> 29), rem = (uint32_t)(m & 0x1fffffffu);
                const bool up = rem > 0x10000000u || (rem == 0x10000000u && (m24 & 1u));
                const uint32_t rb = (((uint32_t)(u >> 63)) << 31) | (((uint32_t)e32 << 23) + m24 + (up ? 1u : 0u));
                const uint32_t res = up ? 0x20000000u - rem : rem;  // < 2^29
                unsigned long long d = 0ull;
                if (res) {
                    const int p = 31 - __clz(res);  // position of the leading bit
                    d = ((unsigned long long)(e - 52 + p) << 52) |
                        (((unsigned long long)res << (52 - p)) & 0xfffffffffffffull);
                }
                if (((rb >> 23) & 0xffu) == 0xffu) d = 0x7ff0000000000000ull;  // rounded past the fp32 range: |v - r| is infinite
                dmax = max(dmax, d);
                const unsigned long long k = order_key64(v);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
                return __uint_as_float(rb);  // a carry into exponent 255 is the correct +-Inf
            }
            const float r = __double2float_rn(v);  // zero, fp32-subnormal, beyond fp32, infinite or NaN
            if (v == v) {  // not NaN
                const unsigned long long k = order_key64(v);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
                if (fabs(v) <= 1.7976931348623157e308) {  // finite: the rounding error is exact in double
                    const double d = fabs(v - (double)r);
                    dmax = max(dmax, (unsigned long long)__double_as_longlong(d));
                }
            }
            return r;
        };
        auto visit = [&](double v, uint64_t i) { y[i] = round1(v); };
        if ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
            // pairs of values: 16-byte loads (four in flight per thread), 8-byte stores
            const double2* x2 = reinterpret_cast<const double2*>(x);
            float2* y2 = reinterpret_cast<float2*>(y);  // y is 16-byte aligned
            const uint64_t npairs = a.n / 2;
            uint64_t q = (uint64_t)blockIdx.x * kF64Threads + tid;
            for (; q + 3 * stride < npairs; q += 4 * stride) {
                const double2 v0 = __ldcs(x2 + q), v1 = __ldcs(x2 + q + stride), v2 = __ldcs(x2 + q + 2 * stride),
                              v3 = __ldcs(x2 + q + 3 * stride);
                y2[q] = make_float2(round1(v0.x), round1(v0.y));
                y2[q + stride] = make_float2(round1(v1.x), round1(v1.y));
                y2[q + 2 * stride] = make_float2(round1(v2.x), round1(v2.y));
                y2[q + 3 * stride] = make_float2(round1(v3.x), round1(v3.y));
            }
            for (; q < npairs; q += stride) {
                const double2 v = __ldcs(x2 + q);
                y2[q] = make_float2(round1(v.x), round1(v.y));
            }
            if ((a.n & 1ull) && blockIdx.x == 0 && tid == 0) visit(__ldcs(x + a.n - 1), a.n - 1);  // odd last value
        } else {
            uint64_t i = (uint64_t)blockIdx.x * kF64Threads + tid;
            for (; i + 3 * stride < a.n; i += 4 * stride) {  // four loads in flight per thread
                const double v0 = __ldcs(x + i), v1 = __ldcs(x + i + stride), v2 = __ldcs(x + i + 2 * stride),
                             v3 = __ldcs(x + i + 3 * stride);
                visit(v0, i);
                visit(v1, i + stride);
                visit(v2, i + 2 * stride);
                visit(v3, i + 3 * stride);
            }
            for (; i < a.n; i += stride) visit(__ldcs(x + i), i);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
            dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        }
        if (lane == 0) {
            s_res[warp][0] = kmin;
            s_res[warp][1] = kmax;
            s_res[warp][2] = dmax;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kF64Threads / 32; ++w) {
                kmin = min(kmin, s_res[w][0]);
                kmax = max(kmax, s_res[w][1]);
                dmax = max(dmax, s_res[w][2]);
            }
            atomicMin(a.res + 3 * f, kmin);
            atomicMax(a.res + 3 * f + 1, kmax);
            atomicMax(a.res + 3 * f + 2, dmax);
        }
        __syncthreads();
    }
}

}  // namespace gpz

namespace {

constexpr uint64_t kF64Align = 256;
constexpr uint64_t kResBytes = 256;  // 3 x 8 fields x 8 bytes

uint64_t f32_ld(uint64_t n) { return align_up(n, 4); }
uint64_t f32_bytes(uint64_t n, int F) { return align_up(4ull * f32_ld(n) * (uint64_t)F, kF64Align); }
unsigned f64_grid(uint64_t n) {
    const uint64_t want = (n + kF64Threads - 1) / kF64Threads;
    const uint64_t cap = 152ull * 8ull;
    return (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
}

double from_key64(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
}

}  // namespace

extern "C" {

uint64_t gpz_compress_f64_workspace_size(uint64_t n, int n_fields) {
    const uint64_t c = gpz_compress_workspace_size(n, n_fields);
    if (c == 0) return 0;
    const uint64_t narrow = align_up(c, kF64Align) + kResBytes + f32_bytes(n, n_fields);
    const uint64_t wide = wide_workspace_size(n, n_fields);  // the 64-bit form, when fp32 cannot hold the bound
    return narrow > wide ? narrow : wide;
}

uint64_t gpz_decompress_f64_workspace_size(uint64_t n, int n_fields) {
    (void)n;
    if (n_fields < 1 || n_fields > kMaxFields) return 0;
    return align_up(gpz_decompress_workspace_size(), kF64Align);  // the status word
}

gpz_status gpz_compress_f64(const double* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                            uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                            void* d_ws, uint64_t ws_size, double* h_eb_used, void* stream) {
    if (!p || p->n_fields < 1 || p->n_fields > kMaxFields || (p->mode != GPZ_EB_ABS && p->mode != GPZ_EB_REL))
        return GPZ_ERR_INVALID_ARG;
    const int F = p->n_fields;
    for (int f = 0; f < F; ++f)
        if (!(p->eb[f] > 0.0) || !std::isfinite(p->eb[f])) return GPZ_ERR_INVALID_ARG;
    if (n > 0) {
        if (!d_fields) return GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F; ++f)
            if (!d_fields[f] || (reinterpret_cast<uintptr_t>(d_fields[f]) & 7u)) return GPZ_ERR_INVALID_ARG;
    }
    const uint64_t need = gpz_compress_f64_workspace_size(n, F);
    if (need == 0) return GPZ_ERR_INVALID_ARG;
    if (!d_ws || ws_size < need) return d_ws ? GPZ_ERR_CAPACITY : GPZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_ws) % kF64Align) return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    const uint64_t cws = align_up(gpz_compress_workspace_size(n, F), kF64Align);
    unsigned long long* res = reinterpret_cast<unsigned long long*>(ws + cws);
    float* y = reinterpret_cast<float*>(ws + cws + kResBytes);
    const uint64_t ld = f32_ld(n);

    // the prepass: the fp32 copy, the fp64 extremes and the largest rounding error
    unsigned long long init[3 * kMaxFields];
    for (int f = 0; f < F; ++f) {
        init[3 * f] = ~0ull;
        init[3 * f + 1] = 0ull;
        init[3 * f + 2] = 0ull;
    }
    if (cudaMemcpyAsync(res, init, 24ull * F, cudaMemcpyHostToDevice, s) != cudaSuccess) return GPZ_ERR_CUDA;
    F64Args fa{};
    fa.F = F;
    fa.n = n;
    fa.res = res;
    for (int f = 0; f < F; ++f) {
        fa.in[f] = n ? d_fields[f] : nullptr;
        fa.out32[f] = y + (uint64_t)f * ld;
    }
    if (n > 0) {
        Recorder rec(s);
        rec.begin(1);
        gpz_f64_prepass_kernel<<<f64_grid(n), kF64Threads, 0, s>>>(fa);
        if (cudaGetLastError() != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("f64");
    }
    unsigned long long got[3 * kMaxFields];
    if (cudaMemcpyAsync(got, res, 24ull * F, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GPZ_ERR_CUDA;

    // the reduced absolute bounds (each step one IEEE double operation)
    double ebp[kMaxFields], ebf[kMaxFields];
    bool narrow = true;
    for (int f = 0; f < F; ++f) {
        double e = p->eb[f];
        const bool any = got[3 * f] != ~0ull;  // some value is not NaN
        if (p->mode == GPZ_EB_REL && any) {
            const volatile double range = from_key64(got[3 * f + 1]) - from_key64(got[3 * f]);
            if (range > 0.0 && std::isfinite(range)) {
                const volatile double t = p->eb[f] * range;
                if (t > 0.0 && std::isfinite(t)) e = t;
            }
        }
        double delta;
        std::memcpy(&delta, &got[3 * f + 2], 8);
        const volatile double reduced = e - delta;
        ebf[f] = e;
        ebp[f] = reduced;
        if (!(reduced > 0.0) || !std::isfinite(reduced)) narrow = false;
    }
    if (!narrow) {
        // fp32 cannot hold some field's bound: 64-bit intermediates with the bounds eb_f
        if (h_eb_used)
            for (int f = 0; f < F; ++f) h_eb_used[f] = ebf[f];
        return wide_compress(d_fields, n, F, p->seg_bits, p->mode, ebf, d_out, out_capacity, d_out_size, h_out_size,
                             d_perm, d_ws, ws_size, s);
    }
    if (h_eb_used)
        for (int f = 0; f < F; ++f) h_eb_used[f] = ebp[f];
    gpz_params q{};
    q.mode = GPZ_EB_ABS;
    q.n_fields = F;
    q.seg_bits = p->seg_bits;
    q.flags = p->flags;
    for (int f = 0; f < F; ++f) q.eb[f] = ebp[f];
    const float* fields[kMaxFields];
    for (int f = 0; f < F; ++f) fields[f] = y + (uint64_t)f * ld;
    // the compression workspace sits at the start, so gpz_sync_status(d_ws) reads its status
    return gpz_compress(fields, n, &q, d_out, out_capacity, d_out_size, h_out_size, d_perm, ws, cws, stream);
}

gpz_status gpz_decompress_f64(const void* d_in, uint64_t in_size, double* const* d_fields, int n_fields, uint64_t n,
                              void* d_ws, uint64_t ws_size, void* stream) {
    if (n_fields < 1 || n_fields > kMaxFields) return GPZ_ERR_INVALID_ARG;
    const int F = n_fields;
    if (n > 0) {
        if (!d_fields) return GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F; ++f)
            if (!d_fields[f] || (reinterpret_cast<uintptr_t>(d_fields[f]) & 7u)) return GPZ_ERR_INVALID_ARG;
    }
    const uint64_t need = gpz_decompress_f64_workspace_size(n, F);
    if (!d_ws || ws_size < need) return d_ws ? GPZ_ERR_CAPACITY : GPZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_ws) % kF64Align) return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_in && in_size >= 8 && aligned(d_in, 4)) {
        // the stream's version word: version 2 is the 64-bit form
        uint32_t head[2] = {0u, 0u};
        if (cudaMemcpyAsync(head, d_in, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GPZ_ERR_CUDA;
        if (head[1] == 2u) return gpz_decompress_wide(d_in, in_size, d_fields, F, n, d_ws, ws_size, stream);
    }
    // version 1: the block decoder stores fp64 directly (each value the fp32
    // reconstruction, widened exactly); the workspace holds the status word
    if (!d_in || !aligned(d_in, 4)) return GPZ_ERR_INVALID_ARG;
    if (in_size % 4 != 0 || in_size < 4ull * kHeaderWords) return GPZ_ERR_CORRUPT;
    const uint64_t nb = (n + kBlock - 1) / kBlock;
    if (nb + (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    uint32_t* status = static_cast<uint32_t*>(d_ws);
    if (cudaMemsetAsync(status, 0, 4, s) != cudaSuccess) return GPZ_ERR_CUDA;
    if (nb == 0) return GPZ_OK;
    DecArgs da{};
    da.stream = static_cast<const uint32_t*>(d_in);
    da.total_words = in_size / 4;
    for (int f = 0; f < F; ++f) da.out[f] = reinterpret_cast<float*>(d_fields[f]);  // double arrays
    da.n = n;
    da.F = F;
    da.nblocks = (uint32_t)nb;
    da.status = status;
    Recorder rec(s);
    rec.begin(1);
    if (launch_decompress64(da, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("decompress");
    return GPZ_OK;
}

}  // extern "C"
