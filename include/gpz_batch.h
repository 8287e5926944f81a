/*
 * gpz_batch.h -- batched compression and decompression in libgpz: many
 * independent particle arrays ("chunks") in a few launches.
 *
 * The paper compresses one array per call (Sections 3.2 and 4); it has no
 * batched form.  This interface is the system form of the same method for
 * workloads of many uneven arrays (simulation ranks' sub-domains, point-cloud
 * tiles): every chunk's stream is byte-for-byte the one gpz_compress produces
 * for it alone, and every chunk's decompressed values are the ones
 * gpz_decompress produces alone.  Only the scheduling differs:
 *   - the chunks of one field count F form a group; per group, ONE launch
 *     computes the value ranges of the relative-bound chunks (one CTA per
 *     slice of a field) and ONE launch runs the fused quantise/sort/encode
 *     stage (Sections 4.1-4.3) over every block of every chunk, one CTA per
 *     block, each finding its chunk through a block-to-chunk map;
 *   - one look-back prefix sum over the blocks of all chunks and one
 *     compaction pass (Section 4.4) place every block in its chunk's stream
 *     and write every chunk's header and block table;
 *   - decompression is one launch per group, one CTA per block;
 *   - a plan can be captured once into a CUDA graph and replayed, and its
 *     launch shape (range slice, compaction and general-path grids) can be
 *     tuned by timing.
 *
 * Conventions are those of gpz.h (device pointers d_*, caller-owned buffers,
 * stream-ordered work, no aborts).  A plan owns a small device copy of its
 * chunk descriptors (allocated when it is created, freed when it is
 * destroyed); everything else is the caller's.  A plan may be run any number
 * of times; it must not be run concurrently with itself (one workspace per
 * concurrent run, and the graph of a plan replays on one stream at a time).
 */
#ifndef GPZ_BATCH_H
#define GPZ_BATCH_H

#include "gpz.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One chunk to compress: the arguments of one gpz_compress call. */
typedef struct {
    const float* fields[GPZ_MAX_FIELDS]; /* device, n fp32 values each (params.n_fields used), 4-byte aligned */
    uint64_t n;                          /* particles; 0 allowed (a bare header) */
    gpz_params params;                   /* as for gpz_compress */
    void* out;                           /* device stream buffer, 4-byte aligned */
    uint64_t out_capacity;               /* bytes, >= gpz_bound_size(n, n_fields) */
    uint32_t* perm;                      /* device [n] permutation output, or NULL */
} gpz_compress_chunk;

/* One chunk to decompress: the arguments of one gpz_decompress call. */
typedef struct {
    const void* in;                      /* device stream, 4-byte aligned */
    uint64_t in_size;                    /* bytes */
    float* fields[GPZ_MAX_FIELDS];       /* device outputs, n fp32 values each, 4-byte aligned */
    int n_fields;                        /* must match the stream */
    uint64_t n;                          /* must match the stream */
} gpz_decompress_chunk;

/* Launch shape of a plan.  A zero field takes the default.
 *   range_slice:   values per range work item (relative bounds: one CTA per
 *                  slice of a field), a multiple of 1024 in 1024..2^24.  Default 65536.
 *   compact_ctas:  CTAs of the compaction launch, 8 warps each, per SM, 1..32.  Default 16.
 *   general_ctas:  CTAs per SM walking the list of general-path blocks, 1..4.  Default 2.
 *   qse_form:      the per-block compression code of a group whose chunks all
 *                  have 16-byte aligned fields: 1 the shared-memory tile body
 *                  (the default), 2 the register body (other groups always
 *                  run the register body).  The stream is the same. */
typedef struct {
    uint32_t range_slice;
    uint32_t compact_ctas;
    uint32_t general_ctas;
    uint32_t qse_form;
} gpz_batch_config;

typedef struct gpz_batch gpz_batch; /* opaque plan */

/* Create a plan over `count` chunk descriptors (host array; copied, so it may
 * be freed after the call).  Checks every descriptor as gpz_compress /
 * gpz_decompress would and returns the first error; a plan needs 1 <= count
 * and fewer than 2^31 blocks (of 1024 particles) and work items in total.
 * Allocates the device copy of the descriptors (GPZ_ERR_OOM on failure) and
 * synchronises the current device once. */
gpz_status gpz_batch_create_compress(const gpz_compress_chunk* h_chunks, uint32_t count, gpz_batch** plan);
gpz_status gpz_batch_create_decompress(const gpz_decompress_chunk* h_chunks, uint32_t count, gpz_batch** plan);

/* Free the plan, its device descriptors and its graph (synchronises the
 * device first).  NULL is ignored. */
void gpz_batch_destroy(gpz_batch* plan);

/* Device workspace in bytes a run of the plan needs (for compression about
 * the total input size, for the per-block temporary outputs; for
 * decompression a few bytes per chunk).  0 for a NULL plan. */
uint64_t gpz_batch_workspace_size(const gpz_batch* plan);

/* Set / read the launch shape (set validates and clamps; invalidates a
 * captured graph). */
gpz_status gpz_batch_set_config(gpz_batch* plan, const gpz_batch_config* cfg);
gpz_status gpz_batch_get_config(const gpz_batch* plan, gpz_batch_config* cfg);

/* Enqueue one run of the plan on `stream`.
 *   d_ws/ws_size:  workspace, 256-byte aligned, >= gpz_batch_workspace_size.
 *   d_out_sizes:   compression: device array [count] receiving each chunk's
 *                  stream size in bytes (in descriptor order), or NULL.
 *                  Ignored for decompression.
 *   use_graph:     0: launch the kernels directly.  1: replay the plan's CUDA
 *                  graph, capturing it first when there is none for these
 *                  (d_ws, d_out_sizes) and this launch shape.  The first run
 *                  with use_graph = 1 therefore captures (on a private stream)
 *                  and is slower; later ones launch one graph.
 * Device-side errors go to per-chunk status words in the workspace, read
 * with gpz_batch_sync_status.  Outputs of a failed chunk are unspecified;
 * the other chunks are unaffected. */
gpz_status gpz_batch_run(gpz_batch* plan, void* d_ws, uint64_t ws_size, uint64_t* d_out_sizes, int use_graph,
                         void* stream);

/* Synchronise `stream`, copy each chunk's status (gpz_status values, in
 * descriptor order) to h_status[count] when it is not NULL, and return the
 * first non-OK status (GPZ_OK if none). */
gpz_status gpz_batch_sync_status(const gpz_batch* plan, const void* d_ws, uint32_t* h_status, void* stream);

/* Time each candidate launch shape on this plan's own chunks (reps timed
 * runs each, after one untimed run, CUDA events on `stream`) and keep the
 * fastest.  Runs the plan up to 10 * (reps + 1) times; the outputs are
 * rewritten each time with the same values.  Writes the chosen shape and its
 * mean time per run (ms) when the pointers are not NULL. */
gpz_status gpz_batch_tune(gpz_batch* plan, void* d_ws, uint64_t ws_size, uint64_t* d_out_sizes, int reps,
                          void* stream, gpz_batch_config* chosen, float* ms_per_run);

/* Kernel launches of one run of the plan (all its groups and stages). */
uint32_t gpz_batch_launches(const gpz_batch* plan);

#ifdef __cplusplus
}
#endif

#endif /* GPZ_BATCH_H */
