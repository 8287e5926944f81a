// gpz_batch_api.cu -- the batched entry points (include/gpz_batch.h): a plan
// is a BatchCore (gpz_batch_core.hpp) plus its own device copy of the
// descriptors, a CUDA graph of one run, and the launch-shape tuner.
#include <algorithm>
#include <vector>

#include "gpz.h"
#include "gpz_batch.h"
#include "gpz_batch_core.hpp"
#include "gpz_host.hpp"

using namespace gpz;
using namespace gpz::host;

struct gpz_batch {
    BatchCore core;
    void* d_mem = nullptr;  // the device copy of the descriptors
    BatchDevice dev{};
    // captured graph
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_ws = nullptr;
    const void* g_out = nullptr;
    gpz_batch_config g_cfg{};
};

namespace {

constexpr uint64_t kAlign = 256;

bool same_cfg(const gpz_batch_config& a, const gpz_batch_config& b) {
    return a.range_slice == b.range_slice && a.compact_ctas == b.compact_ctas && a.general_ctas == b.general_ctas;
}

void drop_graph(gpz_batch* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    p->g_ws = p->g_out = nullptr;
}

gpz_status upload(gpz_batch* p) {
    std::vector<uint8_t> img(core_device_bytes(p->core));
    core_pack(p->core, img.data());
    return cudaMemcpy(p->d_mem, img.data(), img.size(), cudaMemcpyHostToDevice) == cudaSuccess ? GPZ_OK : GPZ_ERR_CUDA;
}

// Finish the plan once its chunks are added: layout, device copy, stream.
gpz_status make_plan(gpz_batch* p) {
    gpz_status st = core_finish(p->core, nullptr);
    if (st != GPZ_OK) return st;
    if (dev_malloc(&p->d_mem, core_device_bytes(p->core)) != cudaSuccess) {
        p->d_mem = nullptr;
        return GPZ_ERR_OOM;
    }
    p->dev = core_device_view(p->core, static_cast<uint8_t*>(p->d_mem));
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
        p->cap = nullptr;
        return GPZ_ERR_CUDA;
    }
    return upload(p);
}

gpz_status check_ws(const gpz_batch* p, const void* d_ws, uint64_t ws_size) {
    if (!d_ws || !aligned(d_ws, kAlign)) return GPZ_ERR_INVALID_ARG;
    if (ws_size < p->core.L.total) return GPZ_ERR_CAPACITY;
    return GPZ_OK;
}

}  // namespace

extern "C" {

gpz_status gpz_batch_create_compress(const gpz_compress_chunk* h, uint32_t count, gpz_batch** plan) {
    if (!plan) return GPZ_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!h || count == 0 || count >= (1u << 31)) return GPZ_ERR_INVALID_ARG;
    gpz_batch* p = new gpz_batch();
    for (uint32_t c = 0; c < count; ++c) {
        const gpz_status st = core_add_compress(p->core, h[c]);
        if (st != GPZ_OK) {
            delete p;
            return st;
        }
    }
    const gpz_status st = make_plan(p);
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
    if (!h || count == 0 || count >= (1u << 31)) return GPZ_ERR_INVALID_ARG;
    gpz_batch* p = new gpz_batch();
    for (uint32_t c = 0; c < count; ++c) {
        const gpz_status st = core_add_decompress(p->core, h[c]);
        if (st != GPZ_OK) {
            delete p;
            return st;
        }
    }
    const gpz_status st = make_plan(p);
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

uint64_t gpz_batch_workspace_size(const gpz_batch* p) { return p ? p->core.L.total : 0; }

uint32_t gpz_batch_launches(const gpz_batch* p) { return p ? p->core.launches : 0; }

gpz_status gpz_batch_get_config(const gpz_batch* p, gpz_batch_config* cfg) {
    if (!p || !cfg) return GPZ_ERR_INVALID_ARG;
    *cfg = p->core.cfg;
    return GPZ_OK;
}

gpz_status gpz_batch_set_config(gpz_batch* p, const gpz_batch_config* cfg) {
    if (!p || !cfg) return GPZ_ERR_INVALID_ARG;
    drop_graph(p);
    bool redo = false;
    const gpz_status st = core_set_config(p->core, *cfg, &redo);
    if (st != GPZ_OK) return st;
    if (redo) {
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
    if (!use_graph) return core_enqueue(p->core, p->dev, ws, d_out_sizes, s, true);
    if (!p->exec || p->g_ws != d_ws || p->g_out != d_out_sizes || !same_cfg(p->g_cfg, p->core.cfg)) {
        drop_graph(p);
        // the launches draw on the counter when captured; a replay adds them below
        const uint64_t before = g_launches.load();
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GPZ_ERR_CUDA;
        st = core_enqueue(p->core, p->dev, ws, d_out_sizes, p->cap, false);
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
        p->g_cfg = p->core.cfg;
    }
    Recorder rec(s);
    rec.begin(1);
    if (cudaGraphLaunch(p->exec, s) != cudaSuccess) return GPZ_ERR_CUDA;
    rec.mark(p->core.kind == 0 ? "batch_graph_compress" : "batch_graph_decompress");
    g_launches += p->core.launches - 1;  // mark() counted one
    return GPZ_OK;
}

gpz_status gpz_batch_sync_status(const gpz_batch* p, const void* d_ws, uint32_t* h_status, void* stream) {
    if (!p || !d_ws) return GPZ_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GPZ_ERR_CUDA;
    const BatchCore& c = p->core;
    const uint8_t* ws = static_cast<const uint8_t*>(d_ws);
    std::vector<uint32_t> st(c.count());
    uint32_t ctrl[32];
    if (cudaMemcpy(st.data(), ws + c.L.status, 4ull * c.count(), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ctrl, ws + c.L.ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GPZ_ERR_CUDA;
    const uint32_t scan = c.kind == 0 ? ctrl[17] : 0u;  // a failed scan spoils every chunk
    gpz_status first = scan ? (gpz_status)scan : GPZ_OK;
    uint32_t best = 0xffffffffu;
    for (uint32_t k = 0; k < c.count(); ++k) {
        const uint32_t idx = c.chunks[k].index;
        const uint32_t v = st[k] ? st[k] : scan;
        if (h_status) h_status[idx] = v;
        if (!scan && st[k] && idx < best) {  // the first failing chunk in descriptor order
            best = idx;
            first = (gpz_status)st[k];
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
    const BatchCore& c = p->core;
    // one parameter at a time, the others at their best so far: the Q.S.E.
    // body (when a group can take the tile body), the range slice (relative
    // bounds only), then the compaction grid
    std::vector<std::vector<gpz_batch_config>> stages;
    bool any_bulk = false;
    for (const auto& g : c.groups) any_bulk = any_bulk || g.bulk;
    if (c.kind == 0 && any_bulk) stages.push_back({{0, 0, 0, 1}, {0, 0, 0, 2}});
    if (c.kind == 0 && c.any_rel) {
        std::vector<gpz_batch_config> v;
        for (uint32_t sl : {16384u, 65536u, 262144u, 1048576u}) v.push_back({sl, 0, 0, 0});
        stages.push_back(v);
    }
    if (c.kind == 0) {
        std::vector<gpz_batch_config> v;
        for (uint32_t cc : {4u, 8u, 16u, 32u}) v.push_back({0, cc, 0, 0});
        stages.push_back(v);
    }
    if (stages.empty()) stages.push_back({gpz_batch_config{}});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GPZ_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GPZ_ERR_CUDA;
    }
    uint8_t* ws = static_cast<uint8_t*>(d_ws);
    auto time_cfg = [&](const gpz_batch_config& cfg, float* out) -> gpz_status {
        gpz_status r = gpz_batch_set_config(p, &cfg);
        if (r != GPZ_OK) return r;
        if ((r = core_enqueue(p->core, p->dev, ws, d_out_sizes, s, false)) != GPZ_OK) return r;
        if (cudaEventRecord(e0, s) != cudaSuccess) return GPZ_ERR_CUDA;
        for (int k = 0; k < reps; ++k)
            if ((r = core_enqueue(p->core, p->dev, ws, d_out_sizes, s, false)) != GPZ_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return GPZ_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return GPZ_ERR_CUDA;
        *out = ms / (float)reps;
        return GPZ_OK;
    };
    gpz_batch_config best = c.cfg;
    float best_ms = 3.0e38f;
    for (const auto& stage : stages) {
        const gpz_batch_config base = best;
        for (const auto& cand : stage) {
            gpz_batch_config cfg = base;
            if (cand.range_slice) cfg.range_slice = cand.range_slice;
            if (cand.compact_ctas) cfg.compact_ctas = cand.compact_ctas;
            if (cand.qse_form) cfg.qse_form = cand.qse_form;
            float ms = 0.0f;
            if ((st = time_cfg(cfg, &ms)) != GPZ_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = p->core.cfg;
            }
        }
        if (st != GPZ_OK) break;
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
