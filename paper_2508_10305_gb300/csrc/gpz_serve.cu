// gpz_serve.cu -- the serving engine of include/gpz_serve.h: FIFO admission
// against a device arena, continuous batching over a few CUDA streams
// ("lanes"), one completion thread per lane.
//
//   submit  -> pending FIFO (host)
//   scheduler thread: when a lane is free, take requests from the head of the
//       FIFO while their outputs fit in the arena (and the batch limits
//       allow), build one batched compression and one batched decompression
//       of them (gpz_batch_core.hpp), place their workspaces in the arena,
//       copy the descriptors from the lane's pinned staging buffer, enqueue
//       the kernels and the read-back of the per-request statuses and sizes,
//       and record the lane's events;
//   lane thread: wait for the events, stamp the completion times, return the
//       workspaces to the arena, hand the requests to poll();
//   release -> the request's output returns to the arena.
// A batch of one request (always so with max_batch = 1: the plain path)
// runs through gpz_compress / gpz_decompress instead.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gpz.h"
#include "gpz_arena.hpp"
#include "gpz_batch.h"
#include "gpz_batch_core.hpp"
#include "gpz_host.hpp"
#include "gpz_serve.h"

using namespace gpz;
using namespace gpz::host;

namespace {

constexpr uint64_t kAlign = 256;
constexpr uint64_t kSlack = 1ull << 20;  // per-batch control sections beyond the per-request estimate

struct Request {
    uint64_t id = 0;
    int kind = 0;  // 0 compress, 1 decompress
    const float* fields[kMaxFields] = {};
    gpz_params p{};
    const void* in = nullptr;
    uint64_t in_size = 0;
    int F = 0;
    uint64_t n = 0;
    uint64_t out_alloc = 0, out_off = 0, field_stride = 0;
    bool has_out = false;
    uint64_t out_bytes = 0, in_bytes = 0;
    uint64_t t_submit = 0, t_start = 0, t_done = 0;
    uint32_t batch = 0, batch_size = 0;
    int status = 0;
    bool done = false;
};

struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t ev_dec = nullptr, ev_all = nullptr;
    uint8_t* h_desc = nullptr;  // pinned: compression image, then decompression image
    uint8_t* d_desc = nullptr;
    uint8_t* h_res = nullptr;   // pinned: statuses and sizes read back
    uint8_t* d_small = nullptr; // device: the plain path's size word
    std::vector<Request*> comp, dec;                 // the running batch, in descriptor order
    std::unique_ptr<BatchCore> comp_core, dec_core;  // statuses come back in plan order
    std::vector<uint64_t> ws_offs;
    bool single = false;  // the batch is one request: run it through the single-array calls
    bool busy = false, launched = false;
    std::condition_variable cv;
    std::thread waiter;
};

struct Server {
    gpz_server_config cfg{};
    uint8_t* d_arena = nullptr;
    std::unique_ptr<Arena> arena;
    uint64_t desc_cap = 0;  // bytes of one descriptor image
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_idle;
    std::deque<Request*> pending, completed;
    std::unordered_map<uint64_t, Request*> by_id;
    std::vector<std::unique_ptr<Lane>> lanes;
    std::thread scheduler;
    bool stop = false, lanes_stop = false;
    uint64_t next_id = 0, mem_epoch = 0, failed_epoch = ~0ull;
    uint32_t batches = 0;
    int device = 0;
    gpz_server_stats stats{};
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    uint64_t now() const {
        return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

uint64_t compress_ws_estimate(uint64_t n, int F) { return gpz_compress_workspace_size(n, F); }

// Arena bytes one request needs when it runs alone (output + workspace; the
// batched workspace adds 8 bytes of offsets per block to the single call's).
uint64_t need_alone(const Request& r) {
    uint64_t b = align_up(r.out_alloc, kAlign) + kSlack;
    if (r.kind == 0) b += align_up(compress_ws_estimate(r.n, r.F), kAlign) + align_up(8 * (nblocks_of(r.n) + 1), kAlign);
    return b;
}

// Results read back per lane: [comp status u32 x B][dec status u32 x B][comp size u64 x B]
uint64_t res_bytes(uint32_t B) { return align_up(4ull * B, 64) * 2 + 8ull * B; }
uint32_t* res_comp_status(Lane& L, uint32_t) { return reinterpret_cast<uint32_t*>(L.h_res); }
uint32_t* res_dec_status(Lane& L, uint32_t B) { return reinterpret_cast<uint32_t*>(L.h_res + align_up(4ull * B, 64)); }
uint64_t* res_comp_size(Lane& L, uint32_t B) {
    return reinterpret_cast<uint64_t*>(L.h_res + 2 * align_up(4ull * B, 64));
}

// Free an arena range under the lock and wake the scheduler.
void give_back(Server* S, uint64_t off) {
    S->arena->release(off);
    ++S->mem_epoch;
}

void finish_request(Server* S, Request* r, uint64_t t) {
    r->t_done = t;
    r->done = true;
    ++S->stats.completed;
    S->stats.in_bytes += r->in_bytes;
    if (S->stop) {  // the engine is being destroyed: the result is dropped
        if (r->has_out) give_back(S, r->out_off);
        S->by_id.erase(r->id);
        delete r;
        return;
    }
    S->completed.push_back(r);
}

// Enqueue one batch on lane L (mutex NOT held; the lane is marked busy and
// its request lists are filled).  Returns false on a CUDA error.
bool launch(Server* S, Lane& L, uint8_t* ws_comp, uint8_t* ws_dec) {
    const uint32_t B = S->cfg.max_batch;
    cudaStream_t s = L.s;
    bool ok = true;
    if (L.single) {
        Request* r = L.comp.empty() ? L.dec[0] : L.comp[0];
        uint8_t* out = S->d_arena + r->out_off;
        if (r->kind == 0) {
            const uint64_t need = compress_ws_estimate(r->n, r->p.n_fields);
            ok = gpz_compress(r->fields, r->n, &r->p, out, r->out_alloc, reinterpret_cast<uint64_t*>(L.d_small),
                              nullptr, nullptr, ws_comp, need, s) == GPZ_OK;
            ok = ok && cudaMemcpyAsync(res_comp_status(L, B), ws_comp, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(res_comp_size(L, B), L.d_small, 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
            ok = ok && cudaEventRecord(L.ev_dec, s) == cudaSuccess;
        } else {
            float* outs[kMaxFields];
            for (int f = 0; f < r->F; ++f) outs[f] = reinterpret_cast<float*>(out + f * r->field_stride);
            ok = gpz_decompress(r->in, r->in_size, outs, r->F, r->n, ws_dec, gpz_decompress_workspace_size(), s) ==
                 GPZ_OK;
            ok = ok && cudaMemcpyAsync(res_dec_status(L, B), ws_dec, 4, cudaMemcpyDeviceToHost, s) == cudaSuccess;
            ok = ok && cudaEventRecord(L.ev_dec, s) == cudaSuccess;
        }
        return ok && cudaEventRecord(L.ev_all, s) == cudaSuccess;
    }
    // decompression first (it is quicker: its requests finish sooner)
    if (L.dec_core) {
        const BatchCore& c = *L.dec_core;
        uint8_t* h = L.h_desc + S->desc_cap;
        uint8_t* d = L.d_desc + S->desc_cap;
        core_pack(c, h);
        ok = ok && cudaMemcpyAsync(d, h, core_device_bytes(c), cudaMemcpyHostToDevice, s) == cudaSuccess;
        ok = ok && core_enqueue(c, core_device_view(c, d), ws_dec, nullptr, s, false) == GPZ_OK;
        ok = ok && cudaMemcpyAsync(res_dec_status(L, B), ws_dec + c.L.status, 4ull * c.count(), cudaMemcpyDeviceToHost,
                                   s) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(L.ev_dec, s) == cudaSuccess;
    if (L.comp_core) {
        const BatchCore& c = *L.comp_core;
        core_pack(c, L.h_desc);
        ok = ok && cudaMemcpyAsync(L.d_desc, L.h_desc, core_device_bytes(c), cudaMemcpyHostToDevice, s) == cudaSuccess;
        uint64_t* sizes = reinterpret_cast<uint64_t*>(ws_comp + c.L.out_sizes);
        ok = ok && core_enqueue(c, core_device_view(c, L.d_desc), ws_comp, sizes, s, false) == GPZ_OK;
        ok = ok && cudaMemcpyAsync(res_comp_status(L, B), ws_comp + c.L.status, 4ull * c.count(),
                                   cudaMemcpyDeviceToHost, s) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(res_comp_size(L, B), sizes, 8ull * c.count(), cudaMemcpyDeviceToHost, s) ==
                       cudaSuccess;
    }
    return ok && cudaEventRecord(L.ev_all, s) == cudaSuccess;
}

// Build the batch's plans and place its workspaces; mutex held.  Returns
// false (placing nothing) when the workspaces do not fit.
bool place(Server* S, Lane& L, uint8_t** ws_comp, uint8_t** ws_dec) {
    L.comp_core.reset();
    L.dec_core.reset();
    L.ws_offs.clear();
    *ws_comp = *ws_dec = nullptr;
    uint64_t need_c = 0, need_d = 0;
    if (L.single) {
        const Request* r = L.comp.empty() ? L.dec[0] : L.comp[0];
        if (r->kind == 0)
            need_c = compress_ws_estimate(r->n, r->p.n_fields);
        else
            need_d = gpz_decompress_workspace_size();
    } else {
        if (!L.comp.empty()) {
            L.comp_core.reset(new BatchCore());
            for (Request* r : L.comp) {
                gpz_compress_chunk d{};
                for (int f = 0; f < r->p.n_fields; ++f) d.fields[f] = r->fields[f];
                d.n = r->n;
                d.params = r->p;
                d.out = S->d_arena + r->out_off;
                d.out_capacity = r->out_alloc;
                if (core_add_compress(*L.comp_core, d) != GPZ_OK) return false;
            }
            if (core_finish(*L.comp_core, nullptr) != GPZ_OK) return false;
            need_c = L.comp_core->L.total;
        }
        if (!L.dec.empty()) {
            L.dec_core.reset(new BatchCore());
            for (Request* r : L.dec) {
                gpz_decompress_chunk d{};
                d.in = r->in;
                d.in_size = r->in_size;
                d.n_fields = r->F;
                d.n = r->n;
                for (int f = 0; f < r->F; ++f)
                    d.fields[f] = reinterpret_cast<float*>(S->d_arena + r->out_off + f * r->field_stride);
                if (core_add_decompress(*L.dec_core, d) != GPZ_OK) return false;
            }
            if (core_finish(*L.dec_core, nullptr) != GPZ_OK) return false;
            need_d = L.dec_core->L.total;
        }
    }
    uint64_t oc = 0, od = 0;
    if (need_c && !S->arena->alloc(need_c, &oc)) return false;
    if (need_d && !S->arena->alloc(need_d, &od)) {
        if (need_c) S->arena->release(oc);
        return false;
    }
    if (need_c) {
        L.ws_offs.push_back(oc);
        *ws_comp = S->d_arena + oc;
    }
    if (need_d) {
        L.ws_offs.push_back(od);
        *ws_dec = S->d_arena + od;
    }
    return true;
}

// The free lane to fill next, or null.  Lane 0 takes any request; with
// lane_bytes set, the other lanes are express lanes that take only requests
// of at most lane_bytes input bytes (so small requests can pass a large one
// without slowing it much).
Lane* pick_lane(Server* S, bool* express) {
    for (size_t k = 0; k < S->lanes.size(); ++k) {
        Lane* L = S->lanes[k].get();
        if (L->busy) continue;
        if (k == 0 || S->cfg.lane_bytes == 0) {
            *express = false;
            return L;
        }
        for (const Request* r : S->pending)
            if (r->in_bytes <= S->cfg.lane_bytes) {
                *express = true;
                return L;
            }
    }
    return nullptr;
}

void scheduler_loop(Server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool express = false;
        S->cv_sched.wait(lk, [&] {
            if (S->stop && S->pending.empty()) return true;
            return !S->pending.empty() && S->mem_epoch != S->failed_epoch && pick_lane(S, &express);
        });
        if (S->pending.empty()) break;  // stopping, nothing left
        Lane& L = *pick_lane(S, &express);
        // admission: requests in FIFO order (an express lane skips the large
        // ones) while their outputs fit
        std::vector<Request*> take;
        uint64_t bytes_in = 0;
        for (auto it = S->pending.begin(); it != S->pending.end() && take.size() < S->cfg.max_batch;) {
            Request* r = *it;
            if (express && r->in_bytes > S->cfg.lane_bytes) {
                ++it;
                continue;
            }
            if (!take.empty() && S->cfg.max_batch_bytes && bytes_in + r->in_bytes > S->cfg.max_batch_bytes) break;
            uint64_t off = 0;
            if (!S->arena->alloc(r->out_alloc, &off)) break;
            r->out_off = off;
            r->has_out = true;
            take.push_back(r);
            bytes_in += r->in_bytes;
            it = S->pending.erase(it);
        }
        // the workspaces: drop requests from the tail until they fit
        uint8_t *ws_comp = nullptr, *ws_dec = nullptr;
        for (;;) {
            L.comp.clear();
            L.dec.clear();
            for (Request* r : take) (r->kind == 0 ? L.comp : L.dec).push_back(r);
            L.single = take.size() == 1;
            if (take.empty() || place(S, L, &ws_comp, &ws_dec)) break;
            Request* r = take.back();
            take.pop_back();
            S->arena->release(r->out_off);
            r->has_out = false;
            S->pending.push_front(r);
        }
        if (take.empty()) {  // nothing fits now: wait for memory to come back
            S->failed_epoch = S->mem_epoch;
            continue;
        }
        const uint32_t id = ++S->batches;
        ++S->stats.batches;
        const uint64_t t = S->now();
        for (Request* r : take) {
            r->t_start = t;
            r->batch = id;
            r->batch_size = (uint32_t)take.size();
        }
        L.busy = true;
        lk.unlock();
        const bool ok = launch(S, L, ws_comp, ws_dec);
        lk.lock();
        if (!ok)
            for (Request* r : take) r->status = GPZ_ERR_CUDA;
        L.launched = true;
        L.cv.notify_one();
    }
}

void lane_loop(Server* S, Lane* L) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    const uint32_t B = S->cfg.max_batch;
    for (;;) {
        L->cv.wait(lk, [&] { return L->launched || S->lanes_stop; });
        if (!L->launched) break;
        lk.unlock();
        const bool e1 = cudaEventSynchronize(L->ev_dec) == cudaSuccess;
        const uint64_t t1 = S->now();
        const bool e2 = cudaEventSynchronize(L->ev_all) == cudaSuccess;
        const uint64_t t2 = S->now();
        lk.lock();
        // per-request statuses (plan order -> descriptor order) and sizes
        if (L->single) {
            for (Request* r : L->comp) {
                const uint32_t st = *res_comp_status(*L, B);
                r->status = r->status ? r->status : (!e2 ? GPZ_ERR_CUDA : (int)st);
                r->out_bytes = *res_comp_size(*L, B);
            }
            for (Request* r : L->dec) {
                const uint32_t st = *res_dec_status(*L, B);
                r->status = r->status ? r->status : (!e1 ? GPZ_ERR_CUDA : (int)st);
                r->out_bytes = 4ull * r->n * r->F;
            }
        } else {
            if (L->comp_core) {
                const BatchCore& c = *L->comp_core;
                for (uint32_t k = 0; k < c.count(); ++k) {
                    Request* r = L->comp[c.chunks[k].index];
                    const uint32_t st = res_comp_status(*L, B)[k];
                    r->status = r->status ? r->status : (!e2 ? GPZ_ERR_CUDA : (int)st);
                }
                for (uint32_t k = 0; k < c.count(); ++k) L->comp[k]->out_bytes = res_comp_size(*L, B)[k];
            }
            if (L->dec_core) {
                const BatchCore& c = *L->dec_core;
                for (uint32_t k = 0; k < c.count(); ++k) {
                    Request* r = L->dec[c.chunks[k].index];
                    const uint32_t st = res_dec_status(*L, B)[k];
                    r->status = r->status ? r->status : (!e1 ? GPZ_ERR_CUDA : (int)st);
                    r->out_bytes = 4ull * r->n * r->F;
                }
            }
        }
        for (Request* r : L->dec) finish_request(S, r, t1);
        for (Request* r : L->comp) finish_request(S, r, t2);
        for (uint64_t off : L->ws_offs) give_back(S, off);
        L->ws_offs.clear();
        L->comp.clear();
        L->dec.clear();
        L->comp_core.reset();
        L->dec_core.reset();
        L->launched = false;
        L->busy = false;
        S->stats.arena_in_use = S->arena->used_bytes();
        S->cv_sched.notify_all();
        S->cv_done.notify_all();
        S->cv_idle.notify_all();
    }
}

void free_server(Server* S) {
    for (auto& l : S->lanes) {
        if (l->ev_dec) cudaEventDestroy(l->ev_dec);
        if (l->ev_all) cudaEventDestroy(l->ev_all);
        if (l->s) cudaStreamDestroy(l->s);
        if (l->h_desc) cudaFreeHost(l->h_desc);
        if (l->h_res) cudaFreeHost(l->h_res);
        if (l->d_desc) cudaFree(l->d_desc);
        if (l->d_small) cudaFree(l->d_small);
    }
    if (S->d_arena) cudaFree(S->d_arena);
    for (auto& kv : S->by_id) delete kv.second;
    delete S;
}

}  // namespace

extern "C" {

gpz_status gpz_server_create(const gpz_server_config* cfg, gpz_server_config* used, void** server) {
    if (!cfg || !server) return GPZ_ERR_INVALID_ARG;
    *server = nullptr;
    if (cfg->budget_bytes < (1ull << 20) || cfg->lanes < 1 || cfg->lanes > 8 || cfg->max_batch < 1 ||
        cfg->max_batch > 65536)
        return GPZ_ERR_INVALID_ARG;
    Server* S = new Server();
    S->cfg = *cfg;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        free_server(S);
        return GPZ_ERR_CUDA;
    }
    if (dev_malloc(reinterpret_cast<void**>(&S->d_arena), cfg->budget_bytes) != cudaSuccess) {
        S->d_arena = nullptr;
        free_server(S);
        return GPZ_ERR_OOM;
    }
    S->arena.reset(new Arena(cfg->budget_bytes, kAlign));
    S->desc_cap = align_up(sizeof(BatchChunk) * cfg->max_batch, kAlign) + 2 * align_up(4ull * cfg->max_batch, kAlign);
    for (uint32_t k = 0; k < cfg->lanes; ++k) {
        std::unique_ptr<Lane> L(new Lane());
        bool ok = cudaStreamCreateWithFlags(&L->s, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&L->ev_dec, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&L->ev_all, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaHostAlloc(reinterpret_cast<void**>(&L->h_desc), 2 * S->desc_cap, cudaHostAllocDefault) ==
                       cudaSuccess;
        ok = ok && cudaHostAlloc(reinterpret_cast<void**>(&L->h_res), res_bytes(cfg->max_batch),
                                 cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaMalloc(reinterpret_cast<void**>(&L->d_desc), 2 * S->desc_cap) == cudaSuccess;
        ok = ok && cudaMalloc(reinterpret_cast<void**>(&L->d_small), 256) == cudaSuccess;
        S->lanes.push_back(std::move(L));
        if (!ok) {
            free_server(S);
            return GPZ_ERR_CUDA;
        }
    }
    for (auto& l : S->lanes) l->waiter = std::thread(lane_loop, S, l.get());
    S->scheduler = std::thread(scheduler_loop, S);
    if (used) *used = S->cfg;
    *server = S;
    return GPZ_OK;
}

gpz_status gpz_server_submit_compress(void* server, const float* const* d_fields, uint64_t n, const gpz_params* p,
                                      uint64_t* id) {
    Server* S = static_cast<Server*>(server);
    if (!S || !p || !id) return GPZ_ERR_INVALID_ARG;
    const int F = p->n_fields;
    if (F < 1 || F > kMaxFields || p->seg_bits < 0 || p->seg_bits > kMaxSegBits ||
        (p->mode != GPZ_EB_ABS && p->mode != GPZ_EB_REL))
        return GPZ_ERR_INVALID_ARG;
    for (int f = 0; f < F; ++f)
        if (!(p->eb[f] > 0.0) || !std::isfinite(p->eb[f])) return GPZ_ERR_INVALID_ARG;
    if (n > 0) {
        if (!d_fields) return GPZ_ERR_INVALID_ARG;
        for (int f = 0; f < F; ++f)
            if (!d_fields[f] || !aligned(d_fields[f], 4)) return GPZ_ERR_INVALID_ARG;
    }
    if (nblocks_of(n) + (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    Request* r = new Request();
    r->kind = 0;
    for (int f = 0; f < F && n > 0; ++f) r->fields[f] = d_fields[f];
    r->p = *p;
    r->F = F;
    r->n = n;
    r->out_alloc = gpz_bound_size(n, F);
    r->in_bytes = 4ull * n * F;
    if (need_alone(*r) > S->arena->capacity()) {
        delete r;
        return GPZ_ERR_CAPACITY;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        delete r;
        return GPZ_ERR_INVALID_ARG;
    }
    r->id = ++S->next_id;
    r->t_submit = S->now();
    S->pending.push_back(r);
    S->by_id[r->id] = r;
    ++S->stats.submitted;
    *id = r->id;
    S->cv_sched.notify_one();
    return GPZ_OK;
}

gpz_status gpz_server_submit_decompress(void* server, const void* d_in, uint64_t in_size, int F, uint64_t n,
                                        uint64_t* id) {
    Server* S = static_cast<Server*>(server);
    if (!S || !id || !d_in || !aligned(d_in, 4) || F < 1 || F > kMaxFields) return GPZ_ERR_INVALID_ARG;
    if (in_size % 4 != 0 || in_size < 4ull * kHeaderWords) return GPZ_ERR_CORRUPT;
    if (nblocks_of(n) + (uint64_t)F * n >= (1ull << 32)) return GPZ_ERR_UNSUPPORTED;
    Request* r = new Request();
    r->kind = 1;
    r->in = d_in;
    r->in_size = in_size;
    r->F = F;
    r->n = n;
    r->field_stride = align_up(4ull * n, kAlign);
    r->out_alloc = r->field_stride * F;
    r->in_bytes = in_size;
    if (need_alone(*r) > S->arena->capacity()) {
        delete r;
        return GPZ_ERR_CAPACITY;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        delete r;
        return GPZ_ERR_INVALID_ARG;
    }
    r->id = ++S->next_id;
    r->t_submit = S->now();
    S->pending.push_back(r);
    S->by_id[r->id] = r;
    ++S->stats.submitted;
    *id = r->id;
    S->cv_sched.notify_one();
    return GPZ_OK;
}

int gpz_server_poll(void* server, gpz_request_result* out, int max, int timeout_ms) {
    Server* S = static_cast<Server*>(server);
    if (!S || !out || max < 1) return 0;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                        [&] { return !S->completed.empty(); });
    int k = 0;
    while (k < max && !S->completed.empty()) {
        Request* r = S->completed.front();
        S->completed.pop_front();
        gpz_request_result& o = out[k++];
        o.id = r->id;
        o.kind = r->kind;
        o.status = r->status;
        o.out = r->has_out ? S->d_arena + r->out_off : nullptr;
        o.out_bytes = r->out_bytes;
        o.field_stride = r->kind == 1 ? r->field_stride : 0;
        o.in_bytes = r->in_bytes;
        o.t_submit_ns = r->t_submit;
        o.t_start_ns = r->t_start;
        o.t_done_ns = r->t_done;
        o.batch = r->batch;
        o.batch_size = r->batch_size;
    }
    return k;
}

gpz_status gpz_server_release(void* server, uint64_t id) {
    Server* S = static_cast<Server*>(server);
    if (!S) return GPZ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->by_id.find(id);
    if (it == S->by_id.end() || !it->second->done) return GPZ_ERR_INVALID_ARG;
    Request* r = it->second;
    auto c = std::find(S->completed.begin(), S->completed.end(), r);
    if (c != S->completed.end()) S->completed.erase(c);  // released before it was polled
    if (r->has_out) give_back(S, r->out_off);
    S->by_id.erase(it);
    delete r;
    S->stats.arena_in_use = S->arena->used_bytes();
    S->cv_sched.notify_all();
    return GPZ_OK;
}

gpz_status gpz_server_stats_get(void* server, gpz_server_stats* stats) {
    Server* S = static_cast<Server*>(server);
    if (!S || !stats) return GPZ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    *stats = S->stats;
    stats->arena_peak = S->arena->peak_bytes();
    stats->arena_in_use = S->arena->used_bytes();
    stats->queued = S->pending.size();
    return GPZ_OK;
}

uint64_t gpz_server_now_ns(void* server) {
    Server* S = static_cast<Server*>(server);
    return S ? S->now() : 0;
}

void gpz_server_destroy(void* server) {
    Server* S = static_cast<Server*>(server);
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        // results are dropped: their memory lets the queued requests run
        for (auto it = S->by_id.begin(); it != S->by_id.end();) {
            Request* r = it->second;
            if (r->done) {
                if (r->has_out) give_back(S, r->out_off);
                delete r;
                it = S->by_id.erase(it);
            } else {
                ++it;
            }
        }
        S->completed.clear();
        S->stop = true;
        S->cv_sched.notify_all();
    }
    if (S->scheduler.joinable()) S->scheduler.join();
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_idle.wait(lk, [&] {
            for (auto& l : S->lanes)
                if (l->busy) return false;
            return true;
        });
        S->lanes_stop = true;
        for (auto& l : S->lanes) l->cv.notify_all();
    }
    for (auto& l : S->lanes)
        if (l->waiter.joinable()) l->waiter.join();
    free_server(S);
}

}  // extern "C"
