// gpz_batch_api.cu -- host side of the batched entry points (include/gpz_batch.h):
// plan creation (validation, grouping by field count, the flattened work
// lists), the workspace layout, the enqueue of one run, CUDA-graph capture
// and replay, and the launch-shape tuner.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gpz.h"
#include "gpz_batch.h"
#include "gpz_batch.cuh"
#include "gpz_host.hpp"

using namespace gpz;
using namespace gpz::host;

namespace {

constexpr uint64_t kAlign = 256;
// block tickets[8], general counts[8] (at 8), scan tile counter (16), scan
// status (17), range-item tickets[8] (24): one word each, per group
constexpr uint64_t kCtrlBytes = 256;
constexpr uint32_t kMaxItems = 1u << 31;

struct Group {
    int F;
    uint32_t first, count;              // plan positions
    uint32_t range_first, range_items;
    uint32_t block_first, blocks;
    int max_ctas;                       // CTAs per SM that fit
};

struct Layout {
    uint64_t ctrl, rkeys, rdone, ready, status, states, zero_bytes;
    uint64_t rparams, offsets, sizes, list, out_sizes, temp, total;
};

uint64_t ntiles_of(uint64_t blocks) { return (blocks + 1 + kScanTile - 1) / kScanTile; }

}  // namespace

struct gpz_batch {
    int kind = 0;  // 0 compression, 1 decompression
    uint32_t count = 0;
    std::vector<BatchChunk> chunks;  // plan order: grouped by field count, stable
    std::vector<Group> groups;
    uint32_t total_blocks = 0;
    uint64_t temp_words = 0;
    bool any_rel = false;
    int sms = 0;
    gpz_batch_config cfg{};
    Layout L{};
    // device copy: chunks, range_end, block_end
    void* d_mem = nullptr;
    BatchChunk* d_chunks = nullptr;
    uint32_t* d_range_end = nullptr;
    uint32_t* d_block_end = nullptr;
    // captured graph
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_ws = nullptr;
    const void* g_out = nullptr;
    gpz_batch_config g_cfg{};
    uint32_t launches = 0;
};

namespace {

bool same_cfg(const gpz_batch_config& a, const gpz_batch_config& b) {
    return a.ctas_per_sm == b.ctas_per_sm && a.claim == b.claim && a.range_slice == b.range_slice &&
           a.compact_ctas == b.compact_ctas;
}

void drop_graph(gpz_batch* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    p->g_ws = p->g_out = nullptr;
}

// Range items of every relative-bound chunk for the plan's slice, the
// flattened prefixes, and their upload.  Returns false when the items do not
// fit the 31-bit ticket space.
bool lay_out_range(gpz_batch* p, std::vector<uint32_t>& range_end) {
    uint64_t r = 0;
    range_end.assign(p->count, 0);
    for (auto& g : p->groups) {
        g.range_first = (uint32_t)r;
        for (uint32_t k = 0; k < g.count; ++k) {
            BatchChunk& ch = p->chunks[g.first + k];
            ch.range_base = (uint32_t)r;
            ch.range_slices = 0;
            if (p->kind == 0 && ch.mode == GPZ_EB_REL) {
                const uint64_t s = std::max<uint64_t>(1, (ch.n + p->cfg.range_slice - 1) / p->cfg.range_slice);
                ch.range_slices = (uint32_t)std::min<uint64_t>(s, kMaxItems);
                r += (uint64_t)ch.F * s;
            }
            range_end[g.first + k] = (uint32_t)std::min<uint64_t>(r, kMaxItems);
        }
        g.range_items = (uint32_t)std::min<uint64_t>(r - g.range_first, kMaxItems);
        if ((uint64_t)g.range_items + g.blocks >= kMaxItems) return false;
    }
    return r < kMaxItems;
}

gpz_status upload(gpz_batch* p) {
    std::vector<uint32_t> range_end;
    if (!lay_out_range(p, range_end)) return GPZ_ERR_UNSUPPORTED;
    std::vector<uint32_t> block_end(p->count);
    for (uint32_t c = 0; c < p->count; ++c) block_end[c] = p->chunks[c].block_base + p->chunks[c].nblocks;
    if (cudaMemcpy(p->d_chunks, p->chunks.data(), sizeof(BatchChunk) * p->count, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(p->d_range_end, range_end.data(), 4ull * p->count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_block_end, block_end.data(), 4ull * p->count, cudaMemcpyHostToDevice) != cudaSuccess)
        return GPZ_ERR_CUDA;
    return GPZ_OK;
}

gpz_batch_config clamp_cfg(const gpz_batch* p, gpz_batch_config c) {
    int fit = 5;
    for (const auto& g : p->groups) fit = std::min(fit, g.max_ctas);
    if (fit < 1) fit = 1;
    if (c.ctas_per_sm == 0 || c.ctas_per_sm > (uint32_t)fit) c.ctas_per_sm = (uint32_t)fit;
    if (c.claim == 0) c.claim = 4;
    c.claim = std::min<uint32_t>(c.claim, 64);
    if (c.range_slice == 0) c.range_slice = 65536;
    c.range_slice = std::min<uint32_t>(std::max<uint32_t>(c.range_slice / 1024 * 1024, 1024), 1u << 24);
    if (c.compact_ctas == 0) c.compact_ctas = 16;
    c.compact_ctas = std::min<uint32_t>(c.compact_ctas, 32);
    return c;
}

// Common part of plan creation once the chunks are filled in (caller order).
gpz_status finish_plan(gpz_batch* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || p->sms < 1)
        return GPZ_ERR_CUDA;
    // group by field count, keeping the caller's order within a group
    std::stable_sort(p->chunks.begin(), p->chunks.end(),
                     [](const BatchChunk& a, const BatchChunk& b) { return a.F < b.F; });
    uint64_t blocks = 0, temp = 0;
    for (uint32_t c = 0; c < p->count; ++c) {
        BatchChunk& ch = p->chunks[c];
        if (p->groups.empty() || p->groups.back().F != ch.F) {
            Group g{};
            g.F = ch.F;
            g.first = c;
            g.block_first = (uint32_t)blocks;
            p->groups.push_back(g);
        }
        Group& g = p->groups.back();
        ++g.count;
        ch.block_base = (uint32_t)blocks;
        ch.temp_base = temp;
        blocks += ch.nblocks;
        g.blocks += ch.nblocks;
        if (p->kind == 0) temp += (uint64_t)ch.nblocks * batch_slot_words(ch.F);
        if (blocks >= kMaxItems) return GPZ_ERR_UNSUPPORTED;
    }
    p->total_blocks = (uint32_t)blocks;
    p->temp_words = temp;
    for (auto& g : p->groups) {
        g.max_ctas = p->kind == 0 ? batch_compress_max_ctas_per_sm(g.F) : batch_decompress_max_ctas_per_sm(g.F);
        if (g.max_ctas < 1) return GPZ_ERR_CUDA;
    }
    p->cfg = clamp_cfg(p, gpz_batch_config{});

    // workspace layout
    Layout& L = p->L;
    const uint64_t n = p->count;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = o;
        o += align_up(bytes, kAlign);
        return at;
    };
    L.ctrl = take(kCtrlBytes);
    L.status = take(4 * n);
    if (p->kind == 0) {
        L.rkeys = take(4ull * kMaxFields * 2 * n);
        L.rdone = take(4 * n);
        L.ready = take(4 * n);
        L.states = take(8 * ntiles_of(blocks));
        L.zero_bytes = o;
        L.rparams = take(sizeof(FieldParams) * kMaxFields * n);
        L.offsets = take(8 * (blocks + 1));
        L.sizes = take(4 * blocks);
        L.list = take(4 * blocks);
        L.out_sizes = take(8 * n);
        L.temp = take(4 * temp);
    } else {
        L.zero_bytes = o;
    }
    L.total = o;

    // device copy of the descriptors and the prefix arrays
    const uint64_t bytes = align_up(sizeof(BatchChunk) * n, kAlign) + 2 * align_up(4 * n, kAlign);
    if (cudaMalloc(&p->d_mem, bytes) != cudaSuccess) {
        p->d_mem = nullptr;
        return GPZ_ERR_OOM;
    }
    uint8_t* m = static_cast<uint8_t*>(p->d_mem);
    p->d_chunks = reinterpret_cast<BatchChunk*>(m);
    p->d_range_end = reinterpret_cast<uint32_t*>(m + align_up(sizeof(BatchChunk) * n, kAlign));
    p->d_block_end = reinterpret_cast<uint32_t*>(m + align_up(sizeof(BatchChunk) * n, kAlign) + align_up(4 * n, kAlign));
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
        p->cap = nullptr;
        return GPZ_ERR_CUDA;
    }
    const gpz_status st = upload(p);
    if (st != GPZ_OK) return st;
    // kernels per run: per group the fused kernel and the general one (or the
    // decoder) when the group has work, then the scan and the compaction
    p->launches = p->kind == 0 ? 2u : 0u;
    for (const auto& g : p->groups)
        if ((p->kind == 0 && (uint64_t)g.range_items + g.blocks > 0) || (p->kind == 1 && g.blocks > 0))
            p->launches += p->kind == 0 ? 2u : 1u;
    return GPZ_OK;
}

// Enqueue one run on stream s (also used inside graph capture).
gpz_status enqueue(gpz_batch* p, uint8_t* ws, uint64_t* d_out_sizes, cudaStream_t s, bool timed) {
    const Layout& L = p->L;
    const gpz_batch_config& cfg = p->cfg;
    uint32_t* ctrl = reinterpret_cast<uint32_t*>(ws + L.ctrl);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return GPZ_ERR_CUDA;
    Recorder rec(s);
    if (timed) rec.begin((int)p->launches);
    if (p->kind == 1) {
        for (size_t k = 0; k < p->groups.size(); ++k) {
            const Group& g = p->groups[k];
            if (g.blocks == 0) continue;  // nothing to decode
            BatchDecompressArgs a{};
            a.chunks = p->d_chunks;
            a.first = g.first;
            a.nchunks = g.count;
            a.block_end = p->d_block_end;
            a.block_first = g.block_first;
            a.total_blocks = g.blocks;
            a.claim = cfg.claim;
            a.ticket = ctrl + k;
            a.chunk_status = status;
            const uint32_t per_sm = std::min<uint32_t>(cfg.ctas_per_sm, (uint32_t)g.max_ctas);
            const uint64_t want = ((uint64_t)g.blocks + cfg.claim - 1) / cfg.claim;
            const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)per_sm * p->sms, want));
            if (launch_batch_decompress(a, g.F, grid, s) != cudaSuccess) return GPZ_ERR_CUDA;
            rec.mark("batch_decompress");
        }
        return GPZ_OK;
    }
    BatchCompressArgs a{};
    a.chunks = p->d_chunks;
    a.range_end = p->d_range_end;
    a.block_end = p->d_block_end;
    a.slice = cfg.range_slice;
    a.claim = cfg.claim;
    a.rkeys = reinterpret_cast<uint32_t*>(ws + L.rkeys);
    a.rdone = reinterpret_cast<uint32_t*>(ws + L.rdone);
    a.ready = reinterpret_cast<uint32_t*>(ws + L.ready);
    a.rparams = reinterpret_cast<FieldParams*>(ws + L.rparams);
    a.temp = reinterpret_cast<uint32_t*>(ws + L.temp);
    a.sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
    a.chunk_status = status;
    for (size_t k = 0; k < p->groups.size(); ++k) {
        const Group& g = p->groups[k];
        a.first = g.first;
        a.nchunks = g.count;
        a.range_first = g.range_first;
        a.range_items = g.range_items;
        a.block_first = g.block_first;
        a.total_blocks = g.blocks;
        a.ticket = ctrl + k;
        a.general_list = reinterpret_cast<uint32_t*>(ws + L.list) + g.block_first;
        a.general_count = ctrl + 8 + k;
        const uint32_t per_sm = std::min<uint32_t>(cfg.ctas_per_sm, (uint32_t)g.max_ctas);
        const uint64_t items = (uint64_t)g.range_items + g.blocks;
        if (items == 0) continue;  // only empty absolute-bound chunks: the compaction writes their headers
        const uint64_t want = (items + cfg.claim - 1) / cfg.claim;
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)per_sm * p->sms, want));
        if (launch_batch_compress(a, g.F, grid, s) != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("batch_qse");
        const int ggrid = (int)std::max<uint32_t>(1, std::min<uint32_t>(g.blocks, 2u * (uint32_t)p->sms));
        if (launch_batch_general(a, g.F, ggrid, s) != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("batch_general");
    }
    BatchScanArgs sa{};
    sa.sizes = a.sizes;
    sa.total_blocks = p->total_blocks;
    sa.offsets = reinterpret_cast<unsigned long long*>(ws + L.offsets);
    sa.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
    sa.tile_counter = ctrl + 16;
    sa.status = ctrl + 17;
    if (launch_batch_scan(sa, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("batch_scan");
    BatchCompactArgs ca{};
    ca.chunks = p->d_chunks;
    ca.nchunks = p->count;
    ca.block_end = p->d_block_end;
    ca.total_blocks = p->total_blocks;
    ca.temp = a.temp;
    ca.offsets = sa.offsets;
    ca.rparams = a.rparams;
    ca.ready = a.ready;
    ca.out_sizes = reinterpret_cast<unsigned long long*>(d_out_sizes ? (void*)d_out_sizes : (void*)(ws + L.out_sizes));
    ca.chunk_status = status;
    const uint64_t warps = (uint64_t)p->total_blocks + p->count;
    const uint64_t want = (warps + kCompactWarps - 1) / kCompactWarps;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)cfg.compact_ctas * p->sms, want));
    if (launch_batch_compact(ca, grid, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("batch_compact");
    return GPZ_OK;
}

gpz_status check_ws(const gpz_batch* p, const void* d_ws, uint64_t ws_size) {
    if (!d_ws || !aligned(d_ws, kAlign)) return GPZ_ERR_INVALID_ARG;
    if (ws_size < p->L.total) return GPZ_ERR_CAPACITY;
    return GPZ_OK;
}

}  // namespace

extern "C" {

gpz_status gpz_batch_create_compress(const gpz_compress_chunk* h, uint32_t count, gpz_batch** plan) {
    if (!plan) return GPZ_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!h || count == 0 || count >= kMaxItems) return GPZ_ERR_INVALID_ARG;
    gpz_batch* p = new gpz_batch();
    p->kind = 0;
    p->count = count;
    p->chunks.resize(count);
    for (uint32_t c = 0; c < count; ++c) {
        const gpz_compress_chunk& d = h[c];
        const gpz_params& q = d.params;
        const int F = q.n_fields;
        gpz_status bad = GPZ_OK;
        if (F < 1 || F > kMaxFields || q.seg_bits < 0 || q.seg_bits > kMaxSegBits ||
            (q.mode != GPZ_EB_ABS && q.mode != GPZ_EB_REL) || !d.out || !aligned(d.out, 4) ||
            (d.perm && !aligned(d.perm, 4)))
            bad = GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F && bad == GPZ_OK; ++f)
            if (!(q.eb[f] > 0.0) || !std::isfinite(q.eb[f])) bad = GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F && bad == GPZ_OK && d.n > 0; ++f)
            if (!d.fields[f] || !aligned(d.fields[f], 4)) bad = GPZ_ERR_INVALID_ARG;
        if (bad == GPZ_OK && nblocks_of(d.n) + (uint64_t)F * d.n >= (1ull << 32)) bad = GPZ_ERR_UNSUPPORTED;
        if (bad == GPZ_OK && d.out_capacity < gpz_bound_size(d.n, F)) bad = GPZ_ERR_CAPACITY;
        if (bad != GPZ_OK) {
            delete p;
            return bad;
        }
        BatchChunk& ch = p->chunks[c];
        std::memset(&ch, 0, sizeof(ch));
        bool vec = true;
        for (int f = 0; f < F; ++f) {
            ch.in[f] = d.n ? d.fields[f] : nullptr;
            vec = vec && (d.n == 0 || aligned(d.fields[f], 16));
            if (q.mode == GPZ_EB_REL)
                ch.rel[f] = q.eb[f];
            else
                ch.params[f] = finalise(q.eb[f]);
        }
        ch.dst = static_cast<uint32_t*>(d.out);
        ch.words = d.out_capacity / 4;
        ch.n = d.n;
        ch.perm = d.perm;
        ch.nblocks = (uint32_t)nblocks_of(d.n);
        ch.index = c;
        ch.F = F;
        ch.G = q.seg_bits;
        ch.mode = q.mode;
        ch.bulk_ok = vec ? 1 : 0;
        p->any_rel = p->any_rel || q.mode == GPZ_EB_REL;
    }
    const gpz_status st = finish_plan(p);
    if (st != GPZ_OK) {
        gpz_batch_destroy(p);
        return st;
    }
    *plan = p;
    return GPZ_OK;
}

gpz_status gpz_batch_create_decompress(const gpz_decompress_chunk* h, uint32_t count, gpz_batch** plan) {
    if (!plan) return GPZ_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!h || count == 0 || count >= kMaxItems) return GPZ_ERR_INVALID_ARG;
    gpz_batch* p = new gpz_batch();
    p->kind = 1;
    p->count = count;
    p->chunks.resize(count);
    for (uint32_t c = 0; c < count; ++c) {
        const gpz_decompress_chunk& d = h[c];
        const int F = d.n_fields;
        gpz_status bad = GPZ_OK;
        if (!d.in || !aligned(d.in, 4) || F < 1 || F > kMaxFields) bad = GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F && bad == GPZ_OK && d.n > 0; ++f)
            if (!d.fields[f] || !aligned(d.fields[f], 4)) bad = GPZ_ERR_INVALID_ARG;
        if (bad == GPZ_OK && (d.in_size % 4 != 0 || d.in_size < 4ull * kHeaderWords)) bad = GPZ_ERR_CORRUPT;
        if (bad == GPZ_OK && nblocks_of(d.n) + (uint64_t)F * d.n >= (1ull << 32)) bad = GPZ_ERR_UNSUPPORTED;
        if (bad != GPZ_OK) {
            delete p;
            return bad;
        }
        BatchChunk& ch = p->chunks[c];
        std::memset(&ch, 0, sizeof(ch));
        for (int f = 0; f < F; ++f) ch.out[f] = d.n ? d.fields[f] : nullptr;
        ch.src = static_cast<const uint32_t*>(d.in);
        ch.words = d.in_size / 4;
        ch.n = d.n;
        ch.nblocks = (uint32_t)nblocks_of(d.n);
        ch.index = c;
        ch.F = F;
    }
    const gpz_status st = finish_plan(p);
    if (st != GPZ_OK) {
        gpz_batch_destroy(p);
        return st;
    }
    *plan = p;
    return GPZ_OK;
}

void gpz_batch_destroy(gpz_batch* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    drop_graph(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->d_mem) cudaFree(p->d_mem);
    delete p;
}

uint64_t gpz_batch_workspace_size(const gpz_batch* p) { return p ? p->L.total : 0; }

uint32_t gpz_batch_launches(const gpz_batch* p) { return p ? p->launches : 0; }

gpz_status gpz_batch_get_config(const gpz_batch* p, gpz_batch_config* cfg) {
    if (!p || !cfg) return GPZ_ERR_INVALID_ARG;
    *cfg = p->cfg;
    return GPZ_OK;
}

gpz_status gpz_batch_set_config(gpz_batch* p, const gpz_batch_config* cfg) {
    if (!p || !cfg) return GPZ_ERR_INVALID_ARG;
    const gpz_batch_config c = clamp_cfg(p, *cfg);
    const bool reslice = c.range_slice != p->cfg.range_slice;
    p->cfg = c;
    drop_graph(p);
    if (reslice && p->any_rel) {
        if (cudaDeviceSynchronize() != cudaSuccess) return GPZ_ERR_CUDA;  // the descriptors may be in use
        return upload(p);
    }
    return GPZ_OK;
}

gpz_status gpz_batch_run(gpz_batch* p, void* d_ws, uint64_t ws_size, uint64_t* d_out_sizes, int use_graph,
                         void* stream) {
    if (!p) return GPZ_ERR_INVALID_ARG;
    gpz_status st = check_ws(p, d_ws, ws_size);
    if (st != GPZ_OK) return st;
    if (d_out_sizes && !aligned(d_out_sizes, 8)) return GPZ_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    if (!use_graph) return enqueue(p, ws, d_out_sizes, s, true);
    if (!p->exec || p->g_ws != d_ws || p->g_out != d_out_sizes || !same_cfg(p->g_cfg, p->cfg)) {
        drop_graph(p);
        // the launches draw on the counter when captured; a replay adds them below
        const uint64_t before = g_launches.load();
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GPZ_ERR_CUDA;
        st = enqueue(p, ws, d_out_sizes, p->cap, false);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
        g_launches.store(before);
        if (st != GPZ_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            return st != GPZ_OK ? st : GPZ_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&p->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            p->exec = nullptr;
            return GPZ_ERR_CUDA;
        }
        p->g_ws = d_ws;
        p->g_out = d_out_sizes;
        p->g_cfg = p->cfg;
    }
    Recorder rec(s);
    rec.begin(1);
    if (cudaGraphLaunch(p->exec, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark(p->kind == 0 ? "batch_graph_compress" : "batch_graph_decompress");
    g_launches += p->launches - 1;  // mark() counted one
    return GPZ_OK;
}

gpz_status gpz_batch_sync_status(const gpz_batch* p, const void* d_ws, uint32_t* h_status, void* stream) {
    if (!p || !d_ws) return GPZ_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GPZ_ERR_CUDA;
    const uint8_t* ws = static_cast<const uint8_t*>(d_ws);
    std::vector<uint32_t> st(p->count);
    uint32_t ctrl[32];
    if (cudaMemcpy(st.data(), ws + p->L.status, 4ull * p->count, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ctrl, ws + p->L.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GPZ_ERR_CUDA;
    gpz_status first = p->kind == 0 && ctrl[17] ? (gpz_status)ctrl[17] : GPZ_OK;
    for (uint32_t c = 0; c < p->count; ++c) {
        const uint32_t idx = p->chunks[c].index;
        uint32_t v = st[c];
        if (v == 0 && p->kind == 0 && ctrl[17]) v = ctrl[17];  // the scan's failure spoils every chunk
        if (h_status) h_status[idx] = v;
    }
    if (first == GPZ_OK) {
        // the first failing chunk in descriptor order
        uint32_t best = 0xffffffffu;
        for (uint32_t c = 0; c < p->count; ++c)
            if (st[c] != 0 && p->chunks[c].index < best) {
                best = p->chunks[c].index;
                first = (gpz_status)st[c];
            }
    }
    return first;
}

gpz_status gpz_batch_tune(gpz_batch* p, void* d_ws, uint64_t ws_size, uint64_t* d_out_sizes, int reps,
                          void* stream, gpz_batch_config* chosen, float* ms_per_run) {
    if (!p || reps < 1) return GPZ_ERR_INVALID_ARG;
    gpz_status st = check_ws(p, d_ws, ws_size);
    if (st != GPZ_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int fit = 5;
    for (const auto& g : p->groups) fit = std::min(fit, g.max_ctas);
    std::vector<gpz_batch_config> cand;
    const uint32_t claims[] = {1, 2, 4, 8};
    for (uint32_t ctas = (uint32_t)fit; ctas >= 1 && ctas + 2 > (uint32_t)fit; --ctas)
        for (uint32_t cl : claims) {
            if (p->kind == 0 && p->any_rel) {
                for (uint32_t sl : {16384u, 65536u, 262144u}) cand.push_back({ctas, cl, sl, 16});
            } else {
                cand.push_back({ctas, cl, 65536, 16});
            }
        }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GPZ_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GPZ_ERR_CUDA;
    }
    auto time_cfg = [&](const gpz_batch_config& c, float* out) -> gpz_status {
        gpz_status r = gpz_batch_set_config(p, &c);
        if (r != GPZ_OK) return r;
        if ((r = enqueue(p, static_cast<uint8_t*>(d_ws), d_out_sizes, s, false)) != GPZ_OK) return r;
        if (cudaEventRecord(e0, s) != cudaSuccess) return GPZ_ERR_CUDA;
        for (int k = 0; k < reps; ++k)
            if ((r = enqueue(p, static_cast<uint8_t*>(d_ws), d_out_sizes, s, false)) != GPZ_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return GPZ_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return GPZ_ERR_CUDA;
        *out = ms / (float)reps;
        return GPZ_OK;
    };
    gpz_batch_config best = p->cfg;
    float best_ms = 3.0e38f;
    for (const auto& c : cand) {
        float ms = 0.0f;
        if ((st = time_cfg(c, &ms)) != GPZ_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = p->cfg;
        }
    }
    if (st == GPZ_OK && p->kind == 0) {
        // then the compaction grid, with the rest fixed
        const gpz_batch_config base = best;
        for (uint32_t cc : {4u, 8u, 32u}) {
            gpz_batch_config c = base;
            c.compact_ctas = cc;
            float ms = 0.0f;
            if ((st = time_cfg(c, &ms)) != GPZ_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = p->cfg;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GPZ_OK) return st;
    st = gpz_batch_set_config(p, &best);
    if (st != GPZ_OK) return st;
    if (chosen) *chosen = best;
    if (ms_per_run) *ms_per_run = best_ms;
    return GPZ_OK;
}

}  // extern "C"
