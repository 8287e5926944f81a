// gpz_batch_core.cu -- host side of one batched run (see gpz_batch_core.hpp):
// descriptor checks, grouping by field count, the flattened work lists, the
// workspace layout and the enqueue of the kernels.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "gpz_batch_core.hpp"
#include "gpz_host.hpp"

namespace gpz {
namespace host {

namespace {

constexpr uint64_t kAlign = 256;
// general-list counts[8] (one per group), scan tile counter (16), scan status (17)
constexpr uint64_t kCtrlBytes = 256;
constexpr uint32_t kMaxItems = 1u << 31;

uint64_t ntiles_of(uint64_t blocks) { return (blocks + 1 + kScanTile - 1) / kScanTile; }

// The SM count, and the compression kernels' shared-memory attributes set
// once per device and field count.
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
bool g_prepared[kMaxDevices][kMaxFields + 1] = {};
int g_sms[kMaxDevices] = {};

gpz_status device_info(int kind, int F, int* sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GPZ_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (!g_sms[dev] && (cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                        g_sms[dev] < 1)) {
        g_sms[dev] = 0;
        return GPZ_ERR_CUDA;
    }
    if (kind == 0 && !g_prepared[dev][F]) {
        if (!batch_prepare_kernels(F)) return GPZ_ERR_CUDA;
        g_prepared[dev][F] = true;
    }
    *sms = g_sms[dev];
    return GPZ_OK;
}

gpz_batch_config clamp_cfg(gpz_batch_config cfg) {
    if (cfg.range_slice == 0) cfg.range_slice = 65536;
    cfg.range_slice = std::min<uint32_t>(std::max<uint32_t>(cfg.range_slice / 1024 * 1024, 1024), 1u << 24);
    if (cfg.compact_ctas == 0) cfg.compact_ctas = 16;
    cfg.compact_ctas = std::min<uint32_t>(cfg.compact_ctas, 32);
    if (cfg.general_ctas == 0) cfg.general_ctas = 2;
    cfg.general_ctas = std::min<uint32_t>(cfg.general_ctas, 4);
    if (cfg.qse_form != 2) cfg.qse_form = 1;
    return cfg;
}

// Range items of every relative-bound chunk for the current slice.  False
// when a launch's items would not fit a 31-bit grid.
bool lay_out_range(BatchCore& c) {
    uint64_t r = 0;
    c.range_end.assign(c.count(), 0);
    for (auto& g : c.groups) {
        g.range_first = (uint32_t)r;
        for (uint32_t k = 0; k < g.count; ++k) {
            BatchChunk& ch = c.chunks[g.first + k];
            ch.range_base = (uint32_t)r;
            ch.range_slices = 0;
            if (c.kind == 0 && ch.mode == GPZ_EB_REL) {
                const uint64_t s = std::max<uint64_t>(1, (ch.n + c.cfg.range_slice - 1) / c.cfg.range_slice);
                ch.range_slices = (uint32_t)std::min<uint64_t>(s, kMaxItems);
                r += (uint64_t)ch.F * s;
            }
            c.range_end[g.first + k] = (uint32_t)std::min<uint64_t>(r, kMaxItems);
        }
        g.range_items = (uint32_t)std::min<uint64_t>(r - g.range_first, kMaxItems);
        if ((uint64_t)g.range_items + g.blocks >= kMaxItems) return false;
    }
    return r < kMaxItems;
}

uint64_t desc_offset(const BatchCore& c, int part) {  // 0 chunks, 1 range_end
    return part == 0 ? 0 : align_up(sizeof(BatchChunk) * c.count(), kAlign);
}

}  // namespace

gpz_status core_add_compress(BatchCore& c, const gpz_compress_chunk& d) {
    const gpz_params& q = d.params;
    const int F = q.n_fields;
    if (F < 1 || F > kMaxFields || q.seg_bits < 0 || q.seg_bits > kMaxSegBits ||
        (q.mode != GPZ_EB_ABS && q.mode != GPZ_EB_REL) || !d.out || !aligned(d.out, 4) ||
        (d.perm && !aligned(d.perm, 4)))
        return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F; ++f)
        if (!(q.eb[f] > 0.0) || !std::isfinite(q.eb[f])) return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F && d.n > 0; ++f)
        if (!d.fields[f] || !aligned(d.fields[f], 4)) return GPZ_ERR_INVALID_ARG;
    if (nblocks_of(d.n) + (uint64_t)F * d.n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    if (d.out_capacity < gpz_bound_size(d.n, F)) return GPZ_ERR_CAPACITY;
    if (c.count() >= kMaxItems) return GPZ_ERR_UNSUPPORTED;
    BatchChunk ch;
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
    ch.index = c.count();
    ch.F = F;
    ch.G = q.seg_bits;
    ch.mode = q.mode;
    ch.bulk_ok = vec ? 1 : 0;
    c.kind = 0;
    c.any_rel = c.any_rel || q.mode == GPZ_EB_REL;
    c.chunks.push_back(ch);
    return GPZ_OK;
}

gpz_status core_add_decompress(BatchCore& c, const gpz_decompress_chunk& d) {
    const int F = d.n_fields;
    if (!d.in || !aligned(d.in, 4) || F < 1 || F > kMaxFields) return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F && d.n > 0; ++f)
        if (!d.fields[f] || !aligned(d.fields[f], 4)) return GPZ_ERR_INVALID_ARG;
    if (d.in_size % 4 != 0 || d.in_size < 4ull * kHeaderWords) return GPZ_ERR_CORRUPT;
    if (nblocks_of(d.n) + (uint64_t)F * d.n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    if (c.count() >= kMaxItems) return GPZ_ERR_UNSUPPORTED;
    BatchChunk ch;
    std::memset(&ch, 0, sizeof(ch));
    for (int f = 0; f < F; ++f) ch.out[f] = d.n ? d.fields[f] : nullptr;
    ch.src = static_cast<const uint32_t*>(d.in);
    ch.words = d.in_size / 4;
    ch.n = d.n;
    ch.nblocks = (uint32_t)nblocks_of(d.n);
    ch.index = c.count();
    ch.F = F;
    c.kind = 1;
    c.chunks.push_back(ch);
    return GPZ_OK;
}

gpz_status core_finish(BatchCore& c, const gpz_batch_config* cfg) {
    if (c.chunks.empty()) return GPZ_ERR_INVALID_ARG;
    // group by field count and (compression) bound mode, keeping the caller's
    // order within a group: relative-bound groups read each block's extremes
    // from their range items
    const bool bymode = c.kind == 0;
    std::stable_sort(c.chunks.begin(), c.chunks.end(), [bymode](const BatchChunk& a, const BatchChunk& b) {
        return a.F != b.F ? a.F < b.F : (bymode && a.mode < b.mode);
    });
    c.groups.clear();
    uint64_t blocks = 0, temp = 0;
    for (uint32_t k = 0; k < c.count(); ++k) {
        BatchChunk& ch = c.chunks[k];
        const int pre = bymode && ch.mode == GPZ_EB_REL;
        if (c.groups.empty() || c.groups.back().F != ch.F || c.groups.back().pre != pre) {
            BatchGroup g{};
            g.F = ch.F;
            g.pre = pre;
            g.bulk = 1;
            g.first = k;
            g.block_first = (uint32_t)blocks;
            c.groups.push_back(g);
        }
        BatchGroup& g = c.groups.back();
        ++g.count;
        g.bulk = g.bulk && ch.bulk_ok;
        ch.block_base = (uint32_t)blocks;
        ch.temp_base = temp;
        blocks += ch.nblocks;
        g.blocks += ch.nblocks;
        if (c.kind == 0) temp += (uint64_t)ch.nblocks * batch_slot_words(ch.F);
        if (blocks >= kMaxItems) return GPZ_ERR_UNSUPPORTED;
    }
    c.total_blocks = (uint32_t)blocks;
    c.temp_words = temp;
    for (auto& g : c.groups) {
        const gpz_status st = device_info(c.kind, g.F, &c.sms);
        if (st != GPZ_OK) return st;
    }
    c.cfg = clamp_cfg(cfg ? *cfg : gpz_batch_config{});
    if (!lay_out_range(c)) return GPZ_ERR_UNSUPPORTED;

    BatchLayout& L = c.L;
    const uint64_t n = c.count();
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        const uint64_t at = o;
        o += align_up(bytes, kAlign);
        return at;
    };
    L = BatchLayout{};
    L.ctrl = take(kCtrlBytes);
    L.status = take(4 * n);
    if (c.kind == 0) {
        L.rkeys = take(4ull * kMaxFields * 2 * n);
        L.rdone = take(4 * n);
        L.states = take(8 * ntiles_of(blocks));
        L.zero_bytes = o;
        L.map = take(4 * blocks);
        L.rparams = take(sizeof(FieldParams) * kMaxFields * n);
        L.bext = c.any_rel ? take(8ull * kMaxFields * blocks) : 0;
        L.offsets = take(8 * (blocks + 1));
        L.sizes = take(4 * blocks);
        L.list = take(4 * blocks);
        L.out_sizes = take(8 * n);
        L.temp = take(4 * temp);
    } else {
        L.zero_bytes = o;
        L.map = take(4 * blocks);
        L.loc = take(16 * blocks);
    }
    L.total = o;
    // kernels per run: the map when there are blocks; per group the range
    // items, the blocks and the general list (or the decoder) when it has
    // them; the scan and the compaction
    c.launches = (blocks > 0 ? 1u : 0u) + (c.kind == 0 ? 2u : 0u);
    for (const auto& g : c.groups)
        c.launches += c.kind == 0 ? (g.range_items > 0) + 2u * (g.blocks > 0) : (g.blocks > 0);
    return GPZ_OK;
}

gpz_status core_set_config(BatchCore& c, const gpz_batch_config& cfg, bool* redo) {
    const gpz_batch_config v = clamp_cfg(cfg);
    *redo = c.kind == 0 && c.any_rel && v.range_slice != c.cfg.range_slice;
    c.cfg = v;
    if (*redo && !lay_out_range(c)) return GPZ_ERR_UNSUPPORTED;
    return GPZ_OK;
}

uint64_t core_device_bytes(const BatchCore& c) { return desc_offset(c, 1) + align_up(4ull * c.count(), kAlign); }

void core_pack(const BatchCore& c, uint8_t* host) {
    std::memcpy(host + desc_offset(c, 0), c.chunks.data(), sizeof(BatchChunk) * c.count());
    std::memcpy(host + desc_offset(c, 1), c.range_end.data(), 4ull * c.count());
}

BatchDevice core_device_view(const BatchCore& c, uint8_t* device) {
    BatchDevice d;
    d.chunks = reinterpret_cast<BatchChunk*>(device + desc_offset(c, 0));
    d.range_end = reinterpret_cast<uint32_t*>(device + desc_offset(c, 1));
    return d;
}

gpz_status core_enqueue(const BatchCore& c, const BatchDevice& dev, uint8_t* ws, uint64_t* d_out_sizes,
                        cudaStream_t s, bool timed) {
    const BatchLayout& L = c.L;
    const gpz_batch_config& cfg = c.cfg;
    uint32_t* ctrl = reinterpret_cast<uint32_t*>(ws + L.ctrl);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
    uint32_t* map = reinterpret_cast<uint32_t*>(ws + L.map);
    if (cudaMemsetAsync(ws, 0, L.zero_bytes, s) != cudaSuccess) return GPZ_ERR_CUDA;
    Recorder rec(s);
    if (timed) rec.begin((int)c.launches);
    if (c.total_blocks > 0) {
        BatchMapArgs ma{};
        ma.chunks = dev.chunks;
        ma.nchunks = c.count();
        ma.block_map = map;
        ma.block_loc = c.kind == 1 ? reinterpret_cast<uint4*>(ws + L.loc) : nullptr;
        if (launch_batch_map(ma, s) != cudaSuccess) return GPZ_ERR_CUDA;
        rec.mark("batch_map");
    }
    if (c.kind == 1) {
        for (const BatchGroup& g : c.groups) {
            if (g.blocks == 0) continue;  // nothing to decode
            BatchDecompressArgs a{};
            a.chunks = dev.chunks;
            a.block_map = map;
            a.block_loc = reinterpret_cast<const uint4*>(ws + L.loc);
            a.block_first = g.block_first;
            a.total_blocks = g.blocks;
            a.chunk_status = status;
            if (launch_batch_decompress(a, g.F, s) != cudaSuccess) return GPZ_ERR_CUDA;
            rec.mark("batch_decompress");
        }
        return GPZ_OK;
    }
    BatchCompressArgs a{};
    a.chunks = dev.chunks;
    a.range_end = dev.range_end;
    a.block_map = map;
    a.slice = cfg.range_slice;
    a.rkeys = reinterpret_cast<uint32_t*>(ws + L.rkeys);
    a.rdone = reinterpret_cast<uint32_t*>(ws + L.rdone);
    a.rparams = reinterpret_cast<FieldParams*>(ws + L.rparams);
    a.bext = c.any_rel ? reinterpret_cast<uint2*>(ws + L.bext) : nullptr;
    a.temp = reinterpret_cast<uint32_t*>(ws + L.temp);
    a.sizes = reinterpret_cast<uint32_t*>(ws + L.sizes);
    a.chunk_status = status;
    for (size_t k = 0; k < c.groups.size(); ++k) {
        const BatchGroup& g = c.groups[k];
        a.first = g.first;
        a.nchunks = g.count;
        a.range_first = g.range_first;
        a.range_items = g.range_items;
        a.block_first = g.block_first;
        a.total_blocks = g.blocks;
        a.general_list = reinterpret_cast<uint32_t*>(ws + L.list) + g.block_first;
        a.general_count = ctrl + k;
        a.pre = g.pre && a.bext != nullptr;
        a.tile = g.bulk && cfg.qse_form == 1;
        if (g.range_items > 0) {
            if (launch_batch_range(a, s) != cudaSuccess) return GPZ_ERR_CUDA;
            rec.mark("batch_range");
        }
        if (g.blocks > 0) {
            if (launch_batch_compress(a, g.F, s) != cudaSuccess) return GPZ_ERR_CUDA;
            rec.mark("batch_qse");
            const int ggrid = (int)std::max<uint32_t>(1, std::min<uint32_t>(g.blocks, cfg.general_ctas * (uint32_t)c.sms));
            if (launch_batch_general(a, g.F, ggrid, s) != cudaSuccess) return GPZ_ERR_CUDA;
            rec.mark("batch_general");
        }
    }
    BatchScanArgs sa{};
    sa.sizes = a.sizes;
    sa.total_blocks = c.total_blocks;
    sa.offsets = reinterpret_cast<unsigned long long*>(ws + L.offsets);
    sa.tile_state = reinterpret_cast<unsigned long long*>(ws + L.states);
    sa.tile_counter = ctrl + 16;
    sa.status = ctrl + 17;
    if (launch_batch_scan(sa, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("batch_scan");
    BatchCompactArgs ca{};
    ca.chunks = dev.chunks;
    ca.nchunks = c.count();
    ca.block_map = map;
    ca.total_blocks = c.total_blocks;
    ca.temp = a.temp;
    ca.offsets = sa.offsets;
    ca.rparams = a.rparams;
    ca.out_sizes = reinterpret_cast<unsigned long long*>(d_out_sizes ? (void*)d_out_sizes : (void*)(ws + L.out_sizes));
    ca.chunk_status = status;
    const uint64_t warps = (uint64_t)c.total_blocks + c.count();
    const uint64_t want = (warps + kCompactWarps - 1) / kCompactWarps;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)cfg.compact_ctas * c.sms, want));
    if (launch_batch_compact(ca, grid, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark("batch_compact");
    return GPZ_OK;
}

}  // namespace host
}  // namespace gpz
