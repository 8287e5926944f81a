// gpz_api.cu -- host side of libgpz: the C ABI declared in include/gpz.h.
// Validates arguments, lays out the workspace, finalises the per-field
// constants and enqueues the kernels on the caller's stream:
//   compress:   [range (relative bound)] -> Q.S.E. (shared-memory tile kernel,
//               or, for fields not 16-byte aligned, block widths + register
//               kernel) -> look-back scan -> copy
//   decompress: decode
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "gpz.h"
#include "gpz_host.hpp"
#include "gpz_internal.cuh"

using namespace gpz;
using namespace gpz::host;

namespace gpz {
namespace host {
StageTimer g_timer;
std::atomic<uint64_t> g_launches{0};

// The library's workspace pools, one per device, created at first use.  The
// release threshold keeps freed memory in the pool, so that a call after the
// first maps no new pages; gpz_release_pooled_memory hands it back.
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t pool_of_current(cudaMemPool_t* out, bool create) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pools[dev] && create) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = pool_of_current(&pool, true);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}
}  // namespace host
}  // namespace gpz

namespace {

constexpr uint64_t kAlign = 256;
constexpr int kRangeGridMax = 152 * 8;  // range-pass CTAs: 8 per SM of a GB300 (full occupancy)
constexpr uint64_t kCtrlBytes = 256;    // words: 0 status, 1 scan tile counter, 2 range counter,
                                        // 3 general-list count, 4-5 out size, 8 blocks left to the
                                        // copy kernel (fused compaction)
constexpr uint64_t kParamBytes = 256;   // FieldParams[8]
constexpr unsigned kKnownFlags = GPZ_FLAG_FUSED_COMPACTION;

uint32_t slot_words_of(int F) { return (uint32_t)align_up(1ull + (uint64_t)F * kBlock, 4); }

uint64_t ntiles_of(uint64_t nblocks) { return (nblocks + 1 + kScanTile - 1) / kScanTile; }

struct WsLayout {
    uint64_t ctrl, params, states, bstates, partials, bext, binfo, sizes, list, temp, total, zero_bytes;
};

WsLayout layout_of(uint64_t n, int F) {
    WsLayout L{};
    const uint64_t nb = nblocks_of(n);
    uint64_t o = 0;
    L.ctrl = o;
    o += kCtrlBytes;
    L.params = o;
    o += kParamBytes;
    L.states = o;
    o += align_up(ntiles_of(nb) * 8, kAlign);
    L.bstates = o;  // per-block look-back states of the fused compaction
    o += align_up(nb * 8, kAlign);
    L.zero_bytes = o;  // ctrl + params + both look-back state arrays are cleared per call
    L.partials = o;
    o += align_up((uint64_t)kRangeGridMax * F * sizeof(float2), kAlign);
    L.bext = o;  // each block's extremes from the range pass (relative bound)
    o += align_up(nb * F * 8ull, kAlign);
    L.binfo = o;  // each block's widths and flags, derived from them
    o += align_up(nb * 8ull, kAlign);
    L.sizes = o;
    o += align_up(nb * 4, kAlign);
    L.list = o;
    o += align_up(nb * 4, kAlign);
    L.temp = o;
    o += align_up(nb * slot_words_of(F) * 4ull, kAlign);
    L.total = o;
    return L;
}

gpz_status read_status(void* d_ws, cudaStream_t s, bool clear) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return GPZ_ERR_CUDA;
    uint32_t st = 0;
    if (cudaMemcpy(&st, d_ws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return GPZ_ERR_CUDA;
    if (clear && st != 0 && cudaMemset(d_ws, 0, 4) != cudaSuccess) return GPZ_ERR_CUDA;
    return (gpz_status)st;
}

}  // namespace

extern "C" {

uint64_t gpz_bound_size(uint64_t n, int F) {
    if (F < 1 || F > kMaxFields) return 0;
    const uint64_t nb = nblocks_of(n);
    return 4ull * (kHeaderWords + 2ull * F + (nb + 1) + nb + (uint64_t)F * n);
}

uint64_t gpz_compress_workspace_size(uint64_t n, int F) {
    if (F < 1 || F > kMaxFields) return 0;
    return layout_of(n, F).total;
}

uint64_t gpz_decompress_workspace_size(void) { return kCtrlBytes; }

const char* gpz_status_str(gpz_status s) {
    switch (s) {
        case GPZ_OK: return "ok";
        case GPZ_ERR_INVALID_ARG: return "invalid argument";
        case GPZ_ERR_CAPACITY: return "buffer too small";
        case GPZ_ERR_CORRUPT: return "corrupt stream";
        case GPZ_ERR_CUDA: return "CUDA error";
        case GPZ_ERR_OOM: return "out of device memory";
        case GPZ_ERR_TIMEOUT: return "device wait timed out";
        case GPZ_ERR_UNSUPPORTED: return "unsupported size";
    }
    return "unknown status";
}

void gpz_set_stage_timing(void* stream, int enable) {
    std::lock_guard<std::mutex> g(g_timer.mu);
    g_timer.enabled = enable != 0;
    g_timer.stream = (cudaStream_t)stream;
}

int gpz_stage_times(const char** names, float* total_ms, int* launches, int max) {
    std::lock_guard<std::mutex> g(g_timer.mu);
    int k = 0;
    if (g_timer.nspans > 0) {
        const int lastev = g_timer.spans[g_timer.nspans - 1].b;
        if (cudaEventSynchronize(g_timer.ev[lastev]) == cudaSuccess) {
            for (int i = 0; i < g_timer.nspans; ++i) {
                const auto& sp = g_timer.spans[i];
                float t = 0.0f;
                if (cudaEventElapsedTime(&t, g_timer.ev[sp.a], g_timer.ev[sp.b]) != cudaSuccess) continue;
                int j = 0;
                while (j < k && std::strcmp(names[j], sp.name) != 0) ++j;
                if (j == k) {
                    if (k == max) continue;
                    names[k] = sp.name;
                    total_ms[k] = 0.0f;
                    launches[k] = 0;
                    ++k;
                }
                total_ms[j] += t;
                launches[j] += 1;
            }
        }
    }
    g_timer.used = 0;
    g_timer.nspans = 0;
    return k;
}

uint64_t gpz_launch_count(int reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

gpz_status gpz_sync_status(void* d_ws, void* stream) {
    if (!d_ws) return GPZ_ERR_INVALID_ARG;
    return read_status(d_ws, (cudaStream_t)stream, true);
}

gpz_status gpz_inspect(const void* h_header, uint64_t len, uint64_t* n, int* n_fields, int* seg_bits,
                       int* mode) {
    if (!h_header || len < 4ull * kHeaderWords) return GPZ_ERR_INVALID_ARG;
    uint32_t w[kHeaderWords];
    std::memcpy(w, h_header, sizeof(w));
    if (w[0] != kMagic || w[1] != kVersion || w[2] < 1 || w[2] > (uint32_t)kMaxFields ||
        w[3] > (uint32_t)kMaxSegBits || w[4] != (uint32_t)kBlock || w[5] > 1)
        return GPZ_ERR_CORRUPT;
    const uint64_t nn = (uint64_t)w[6] | ((uint64_t)w[7] << 32);
    if (w[8] != nblocks_of(nn)) return GPZ_ERR_CORRUPT;
    if (n) *n = nn;
    if (n_fields) *n_fields = (int)w[2];
    if (seg_bits) *seg_bits = (int)w[3];
    if (mode) *mode = (int)w[5];
    return GPZ_OK;
}

}  // extern "C"

namespace gpz {
namespace host {

RangeTargets compress_range_targets(uint64_t n, int F) {
    const WsLayout L = layout_of(n, F);
    RangeTargets r;
    r.ctrl = L.ctrl;
    r.params = L.params;
    r.partials = L.partials;
    r.bext = L.bext;
    return r;
}

// gpz_compress; with range_done the range pass's outputs (the block
// extremes, the CTAs' partial extremes folded into the constants) are
// already in the workspace, written on this stream by a kernel that read the
// fields anyway, and are neither cleared nor recomputed.
gpz_status compress_impl(const float* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                         uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                         void* d_ws, uint64_t ws_size, void* stream, bool range_done,
                         const float* interleaved) {
    if (!p || !d_out || !aligned(d_out, 4)) return GPZ_ERR_INVALID_ARG;
    const int F = p->n_fields;
    if (F < 1 || F > kMaxFields || p->seg_bits < 0 || p->seg_bits > kMaxSegBits ||
        (p->mode != GPZ_EB_ABS && p->mode != GPZ_EB_REL))
        return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F; ++f)
        if (!(p->eb[f] > 0.0) || !std::isfinite(p->eb[f])) return GPZ_ERR_INVALID_ARG;
    if ((p->flags & ~kKnownFlags) != 0u) return GPZ_ERR_INVALID_ARG;
    if (n > 0) {
        if (!d_fields) return GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F; ++f)
            if (!d_fields[f] || !aligned(d_fields[f], 4)) return GPZ_ERR_INVALID_ARG;
    }
    if (d_perm && !aligned(d_perm, 4)) return GPZ_ERR_INVALID_ARG;
    const uint64_t nb = nblocks_of(n);
    if (nb + (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    if (out_capacity < gpz_bound_size(n, F)) return GPZ_ERR_CAPACITY;
    const WsLayout L = layout_of(n, F);
    cudaStream_t s = (cudaStream_t)stream;
    bool own_ws = false;
    if (d_ws) {
        if (ws_size < L.total) return GPZ_ERR_CAPACITY;
        if (!aligned(d_ws, kAlign)) return GPZ_ERR_INVALID_ARG;
    } else {
        if (dev_malloc_async(&d_ws, L.total, s) != cudaSuccess) return GPZ_ERR_OOM;
        own_ws = true;
    }
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.ctrl);
    uint32_t* tile_counter = status + 1;
    uint32_t* range_counter = status + 2;
    unsigned long long* ws_out_size = reinterpret_cast<unsigned long long*>(ws + L.ctrl + 16);
    FieldParams* d_params = reinterpret_cast<FieldParams*>(ws + L.params);

    gpz_status rc = GPZ_OK;
    Recorder rec(s);
    range_done = range_done && p->mode == GPZ_EB_REL && d_ws != nullptr && !own_ws;
    do {
        if (range_done) {  // keep the constants: clear the control words and the look-back states only
            if ((rc = cuda_status(cudaMemsetAsync(ws + L.ctrl, 0, kCtrlBytes, s))) != GPZ_OK) break;
            if ((rc = cuda_status(cudaMemsetAsync(ws + L.states, 0, L.zero_bytes - L.states, s))) != GPZ_OK) break;
        } else if ((rc = cuda_status(cudaMemsetAsync(ws, 0, L.zero_bytes, s))) != GPZ_OK) {
            break;
        }
        rec.begin();
        FieldParams hp[kMaxFields] = {};
        const bool rel = p->mode == GPZ_EB_REL;
        if (!rel)
            for (int f = 0; f < F; ++f) hp[f] = finalise(p->eb[f]);
        bool vec_ok = true;
        for (int f = 0; f < F && n > 0; ++f) vec_ok = vec_ok && aligned(d_fields[f], 16);
        if (interleaved) vec_ok = aligned(interleaved, 16);
        const bool fused = (p->flags & GPZ_FLAG_FUSED_COMPACTION) != 0u;
        // the shared-memory tile kernel takes 16-byte aligned fields and derives
        // each block's widths itself; the register kernel reads them from the
        // block-info pass (relative bound)
        const bool tile = vec_ok && !fused;
        if (interleaved && (!tile || (rel && !range_done))) {  // the caller's side of the contract
            rc = GPZ_ERR_INVALID_ARG;
            break;
        }

        if (rel) {
            RangeArgs ra{};
            for (int f = 0; f < F; ++f) {
                ra.fields[f] = n ? d_fields[f] : nullptr;
                ra.rel[f] = p->eb[f];
            }
            ra.n = n;
            ra.F = F;
            ra.vec_ok = vec_ok ? 1 : 0;
            ra.partials = reinterpret_cast<float2*>(ws + L.partials);
            ra.done_counter = range_counter;
            ra.d_params = d_params;
            ra.bext = reinterpret_cast<uint2*>(ws + L.bext);
            uint64_t want = (nb * F + kRangeThreads / 32 - 1) / (kRangeThreads / 32);  // a warp per (block, field)
            const int grid = (int)(want < 1 ? 1 : (want > (uint64_t)kRangeGridMax ? kRangeGridMax : want));
            if (!range_done) {
                if ((rc = cuda_status(launch_range(ra, grid, s))) != GPZ_OK) break;
                rec.mark("range");
            }
            if (nb > 0 && !tile) {
                if ((rc = cuda_status(launch_block_info(ra.bext, d_params, (uint32_t)nb, F,
                                                        reinterpret_cast<unsigned long long*>(ws + L.binfo), s))) !=
                    GPZ_OK)
                    break;
                rec.mark("info");
            }
        }

        QseArgs qa{};
        for (int f = 0; f < F; ++f) {
            qa.fields[f] = n ? d_fields[f] : nullptr;
            qa.params[f] = hp[f];
        }
        qa.n = n;
        qa.nblocks = (uint32_t)nb;
        qa.F = F;
        qa.G = p->seg_bits;
        qa.bulk_ok = vec_ok ? 1 : 0;
        qa.interleaved = interleaved ? 1 : 0;
        qa.d_params = rel ? d_params : nullptr;
        qa.bext = rel ? reinterpret_cast<const uint2*>(ws + L.bext) : nullptr;
        qa.binfo = rel && !tile ? reinterpret_cast<const unsigned long long*>(ws + L.binfo) : nullptr;
        qa.temp = reinterpret_cast<uint32_t*>(ws + L.temp);
        qa.slot_words = slot_words_of(F);
        qa.sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
        qa.perm = d_perm;
        qa.status = status;
        qa.general_list = reinterpret_cast<uint32_t*>(ws + L.list);
        qa.general_count = status + 3;
        const uint32_t table_start = (uint32_t)(kHeaderWords + 2 * F);
        if (fused) {
            const uint64_t payload_start = table_start + nb + 1;
            qa.direct = static_cast<uint32_t*>(d_out) + payload_start;
            qa.direct_capacity = out_capacity / 4 - payload_start;  // out_capacity >= the bound
            qa.bstate = reinterpret_cast<unsigned long long*>(ws + L.bstates);
            qa.deferred_count = status + 8;
        }
        if (nb > 0) {
            const cudaError_t e = fused ? launch_qse_direct(qa, s) : tile ? launch_qse_tile(qa, s) : launch_qse(qa, s);
            if ((rc = cuda_status(e)) != GPZ_OK) break;
            rec.mark("qse");
            ++g_launches;  // launch_qse enqueues two kernels: the fast path and the general list
        }

        uint32_t* stream_words = static_cast<uint32_t*>(d_out);
        ScanArgs sa{};
        sa.sizes = qa.sizes;
        sa.nblocks = (uint32_t)nb;
        sa.n = n;
        sa.F = F;
        sa.table = stream_words + table_start;
        sa.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
        sa.tile_counter = tile_counter;
        sa.status = status;
        if ((rc = cuda_status(launch_scan(sa, s))) != GPZ_OK) break;
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
        ca.G = p->seg_bits;
        ca.mode = p->mode;
        for (int f = 0; f < F; ++f) ca.params[f] = hp[f];
        ca.d_params = rel ? d_params : nullptr;
        ca.d_out_size = d_out_size ? reinterpret_cast<unsigned long long*>(d_out_size) : ws_out_size;
        ca.unplaced = fused ? status + 8 : nullptr;
        ca.version = kVersion;
        if ((rc = cuda_status(launch_compact(ca, s))) != GPZ_OK) break;
        rec.mark("compact");

        if (h_out_size || own_ws) {
            if (h_out_size) {
                if ((rc = cuda_status(cudaMemcpyAsync(h_out_size, ca.d_out_size, 8, cudaMemcpyDeviceToHost, s))) !=
                    GPZ_OK)
                    break;
            }
            rc = read_status(status, s, !own_ws);
        }
    } while (false);
    if (own_ws) {
        cudaFreeAsync(d_ws, s);
        if (rc == GPZ_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = GPZ_ERR_CUDA;
    }
    return rc;
}

}  // namespace host
}  // namespace gpz

extern "C" {

gpz_status gpz_compress(const float* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                        uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size, uint32_t* d_perm,
                        void* d_ws, uint64_t ws_size, void* stream) {
    return compress_impl(d_fields, n, p, d_out, out_capacity, d_out_size, h_out_size, d_perm, d_ws, ws_size, stream,
                         false);
}

gpz_status gpz_decompress(const void* d_in, uint64_t in_size, float* const* d_fields, int F, uint64_t n,
                          void* d_ws, uint64_t ws_size, void* stream) {
    return decompress_impl(d_in, in_size, d_fields, F, n, d_ws, ws_size, stream, nullptr);
}

}  // extern "C"

namespace gpz {
namespace host {

gpz_status decompress_impl(const void* d_in, uint64_t in_size, float* const* d_fields, int F, uint64_t n,
                           void* d_ws, uint64_t ws_size, void* stream, float* interleaved) {
    if (!d_in || !aligned(d_in, 4) || F < 1 || F > kMaxFields) return GPZ_ERR_INVALID_ARG;
    if (n > 0) {
        if (!d_fields) return GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F; ++f)
            if (!d_fields[f] || !aligned(d_fields[f], 4)) return GPZ_ERR_INVALID_ARG;
    }
    if (in_size % 4 != 0 || in_size < 4ull * kHeaderWords) return GPZ_ERR_CORRUPT;
    const uint64_t nb = nblocks_of(n);
    if (nb + (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    bool own_ws = false;
    if (d_ws) {
        if (ws_size < gpz_decompress_workspace_size()) return GPZ_ERR_CAPACITY;
        if (!aligned(d_ws, 16)) return GPZ_ERR_INVALID_ARG;
    } else {
        if (dev_malloc_async(&d_ws, gpz_decompress_workspace_size(), s) != cudaSuccess) return GPZ_ERR_OOM;
        own_ws = true;
    }
    uint32_t* status = static_cast<uint32_t*>(d_ws);
    gpz_status rc = GPZ_OK;
    Recorder rec(s);
    do {
        if ((rc = cuda_status(cudaMemsetAsync(status, 0, 4, s))) != GPZ_OK) break;
        rec.begin();
        DecArgs da{};
        da.stream = static_cast<const uint32_t*>(d_in);
        da.total_words = in_size / 4;
        for (int f = 0; f < F; ++f) da.out[f] = n ? d_fields[f] : nullptr;
        if (interleaved) da.out[0] = interleaved;  // d_fields[f] = interleaved + f
        da.interleaved = interleaved ? 1 : 0;
        da.n = n;
        da.F = F;
        da.nblocks = (uint32_t)nb;
        da.status = status;
        if (nb > 0) {
            if ((rc = cuda_status(launch_decompress(da, s))) != GPZ_OK) break;
            rec.mark("decompress");
        }
        if (own_ws) rc = read_status(status, s, false);
    } while (false);
    if (own_ws) {
        cudaFreeAsync(d_ws, s);
        if (rc == GPZ_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = GPZ_ERR_CUDA;
    }
    return rc;
}

}  // namespace host
}  // namespace gpz

extern "C" {

uint64_t gpz_pooled_bytes(void) {
    cudaMemPool_t pool = nullptr;
    if (gpz::host::pool_of_current(&pool, false) != cudaSuccess || !pool) return 0;
    uint64_t v = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) return 0;
    return v;
}

gpz_status gpz_release_pooled_memory(void) {
    cudaMemPool_t pool = nullptr;
    if (gpz::host::pool_of_current(&pool, false) != cudaSuccess) return GPZ_ERR_CUDA;
    if (!pool) return GPZ_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return GPZ_ERR_CUDA;
    return cuda_status(cudaMemPoolTrimTo(pool, 0));
}

}  // extern "C"
