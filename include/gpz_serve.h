/*
 * gpz_serve.h -- a serving engine for libgpz: compress and decompress
 * requests from many clients, admitted against a fixed device-memory budget
 * and run in continuous batches.
 *
 * The paper measures one call at a time (Section 6); it has no serving form.
 * This engine is the system form of the same method for a stream of
 * independent requests: every compress result is byte-for-byte the stream
 * gpz_compress writes for that request alone, and every decompress result is
 * bit-for-bit what gpz_decompress writes alone.  Only the scheduling differs:
 *   - the engine owns one device arena of `budget_bytes` (allocated once when
 *     it is created) from which every admitted request takes its output and
 *     workspace; a request waits in a FIFO queue until its memory fits
 *     (admission), and takes nothing else from the device;
 *   - a scheduler thread launches, on each of `lanes` CUDA streams as soon as
 *     the stream is free, one batch of the requests waiting at that moment
 *     (up to max_batch requests and max_batch_bytes of input): the compress
 *     requests as one batched compression (include/gpz_batch.h) and the
 *     decompress requests as one batched decompression.  A batch of one
 *     request runs through gpz_compress / gpz_decompress; with max_batch = 1
 *     every request does -- the plain path, for comparison;
 *   - a completion thread per lane waits for each batch, records the
 *     completion time and per-request status, and returns the workspace to
 *     the arena; a request's output stays in the arena until the client
 *     releases it.
 *
 * Inputs are the client's device buffers and must stay valid and unchanged
 * until the request's result has been polled.  All entry points are
 * thread-safe.  Times are host clock readings in nanoseconds since the
 * engine was created.
 */
#ifndef GPZ_SERVE_H
#define GPZ_SERVE_H

#include "gpz.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    uint64_t budget_bytes;    /* device arena for outputs and workspaces (admission budget), >= 1 MiB */
    uint32_t lanes;           /* CUDA streams batches run on, 1..8 */
    uint32_t max_batch;       /* requests per batch, >= 1 (1 = the plain one-call-per-request path) */
    uint64_t max_batch_bytes; /* input bytes per batch (0 = no limit); a single larger request still runs */
    uint64_t lane_bytes;      /* 0: every lane takes any request.  Else lanes 1.. are express lanes that
                                 take only requests of at most lane_bytes input bytes, in FIFO order
                                 among those (they may pass larger requests waiting for lane 0) */
} gpz_server_config;

typedef struct {
    uint64_t id;          /* as returned by submit */
    int kind;             /* 0 compress, 1 decompress */
    int status;           /* gpz_status of the request */
    void* out;            /* device, in the arena: compress -> the stream; decompress -> n_fields arrays
                             of n fp32 values (block-sorted order), field f at out + f*field_stride */
    uint64_t out_bytes;   /* stream bytes (compress) or 4*n*n_fields (decompress) */
    uint64_t field_stride;/* decompress: bytes from one field's array to the next (0 for compress) */
    uint64_t in_bytes;    /* input bytes: 4*n*n_fields (compress) or the stream size (decompress) */
    uint64_t t_submit_ns; /* submit returned */
    uint64_t t_start_ns;  /* its batch was launched */
    uint64_t t_done_ns;   /* its batch was seen complete */
    uint32_t batch;       /* sequence number of its batch */
    uint32_t batch_size;  /* requests in its batch */
} gpz_request_result;

typedef struct {
    uint64_t submitted, completed, batches;
    uint64_t in_bytes;        /* input bytes of completed requests */
    uint64_t arena_peak;      /* most arena bytes in use at once */
    uint64_t arena_in_use;    /* arena bytes in use now */
    uint64_t queued;          /* requests waiting for admission now */
} gpz_server_stats;

/* Create an engine on the current device (allocates the arena, the lanes'
 * streams and staging buffers, starts its threads). */
gpz_status gpz_server_create(const gpz_server_config* cfg, gpz_server_config* used, void** server);

/* Queue a compression of n particles of p->n_fields fields (d_fields: host
 * array of device pointers, as gpz_compress).  GPZ_ERR_CAPACITY when the
 * request alone needs more than the budget.  Writes the request id. */
gpz_status gpz_server_submit_compress(void* server, const float* const* d_fields, uint64_t n,
                                      const gpz_params* p, uint64_t* id);

/* Queue a decompression of the stream d_in (in_size bytes) holding n
 * particles of n_fields fields. */
gpz_status gpz_server_submit_decompress(void* server, const void* d_in, uint64_t in_size, int n_fields,
                                        uint64_t n, uint64_t* id);

/* Move up to `max` completed results (oldest first) into out[]; waits up to
 * timeout_ms for the first one.  Returns how many were written. */
int gpz_server_poll(void* server, gpz_request_result* out, int max, int timeout_ms);

/* Return a completed request's output memory to the arena (its out pointer
 * becomes invalid).  GPZ_ERR_INVALID_ARG for an unknown or running id. */
gpz_status gpz_server_release(void* server, uint64_t id);

gpz_status gpz_server_stats_get(void* server, gpz_server_stats* stats);

/* Host clock of the engine (ns since creation), for clients' own timestamps. */
uint64_t gpz_server_now_ns(void* server);

/* Wait for every queued and running request, stop the threads, free the
 * arena and the streams.  Results not yet polled are dropped. */
void gpz_server_destroy(void* server);

#ifdef __cplusplus
}
#endif

#endif /* GPZ_SERVE_H */
