/*
 * gpz.h -- C ABI of libgpz, a GB300 (sm_103a) implementation of GPZ, the
 * error-bounded lossy compressor for particle data of Li et al., "GPZ:
 * GPU-Accelerated Lossy Compressor for Particle Data" (arXiv 2508.10305).
 *
 * The library compresses n particles of F fp32 fields (structure of arrays,
 * one device array per field) into a byte stream, and back.  It runs the
 * paper's four-stage pipeline (Section 3.2): spatial quantisation into a
 * per-axis segment id and offset (Section 4.1), a stable per-block sort by
 * segment id (Section 4.2), run-length + delta + fixed-length coding
 * (Section 4.3), and compaction of the per-block outputs through a device-wide
 * prefix sum (Section 4.4).  Decompression undoes them without sorting, so
 * its output is the input permuted within each 1024-particle block; the
 * permutation can be returned by compression.
 *
 * Conventions for every entry point:
 *   - pointers named d_* are device pointers (cudaMalloc'ed or equivalent,
 *     on the current device); h_* are host pointers;
 *   - the caller owns every buffer; the library allocates device memory only
 *     when a workspace argument is NULL (stream-ordered, freed before return);
 *   - `stream` is a cudaStream_t handle (NULL = the legacy default stream);
 *     work is enqueued on it and the call returns without synchronising,
 *     unless a host-side result (h_*) is requested or the workspace is
 *     allocated by the library;
 *   - argument errors are returned at once and enqueue nothing; errors found
 *     by the kernels (corrupt stream, a timed-out wait) are recorded in the
 *     workspace's status word, which each call clears when it starts, and
 *     are read with gpz_sync_status();
 *   - no entry point aborts, traps or prints.
 */
#ifndef GPZ_H
#define GPZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPZ_OK = 0,
    GPZ_ERR_INVALID_ARG = 1, /* a NULL where a pointer is required, a size or a bound out of range */
    GPZ_ERR_CAPACITY = 2,    /* output or workspace smaller than gpz_bound_size / *_workspace_size */
    GPZ_ERR_CORRUPT = 3,     /* the stream fails a format check (decompression) */
    GPZ_ERR_CUDA = 4,        /* a CUDA runtime call failed (launch, copy, stream) */
    GPZ_ERR_OOM = 5,         /* the library could not allocate its workspace */
    GPZ_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (never expected) */
    GPZ_ERR_UNSUPPORTED = 7  /* n too large for 32-bit word offsets: n_blocks + F*n >= 2^32 */
} gpz_status;

typedef enum {
    GPZ_EB_ABS = 0, /* eb[f] is the absolute bound of field f */
    GPZ_EB_REL = 1  /* eb[f] is relative to field f's value range (max - min over non-NaN values) */
} gpz_eb_mode;

#define GPZ_MAX_FIELDS 8
#define GPZ_BLOCK 1024 /* particles per block: one warp, 32 threads x 32 points (Section 4.2) */

/* Compression parameters.
 *   mode:     gpz_eb_mode.
 *   n_fields: F in 1..8.  Fields 0..min(F,3)-1 are the position axes that
 *             are segmented and sorted (Section 4.1); fields 3.. are carried
 *             along in sorted order with their own codes.
 *   seg_bits: G in 0..3, the segment-id bits per axis (at most 2^G segments
 *             per axis and block; the segment size m scales with the block's
 *             extent, Section 4.1).  3 is the default.
 *   flags:    0, or GPZ_FLAG_* bits selecting an implementation variant of
 *             this one call; the stream is the same bytes either way.  Zero-
 *             initialised parameters take the defaults.
 *   eb[f]:    error bound of field f, > 0 and finite.  Every decompressed
 *             value is within eb (absolute) of its input value. */
typedef struct {
    int mode;
    int n_fields;
    int seg_bits;
    unsigned int flags;
    double eb[GPZ_MAX_FIELDS];
} gpz_params;

/* Compaction form (Section 4.4) of one gpz_compress call; the stream is the
 * same bytes in either form.
 *   default (no flag): Section 4.4's three steps -- every block is encoded
 *     into a temporary slot, a scan computes the offsets, a copy kernel moves
 *     every block into the stream.
 *   GPZ_FLAG_FUSED_COMPACTION: every block publishes its size and looks back
 *     over its predecessors' sizes, waiting for them (a decoupled look-back
 *     over blocks, the in-kernel form of Table 1); a block whose offset is
 *     known is written straight into the stream, the others (raw blocks, and
 *     the blocks behind one that needed the general path) go through their
 *     temporary slots and the copy kernel.  After such a call, word 8 of the
 *     compression workspace (bytes 32..35) holds the number of blocks the
 *     copy kernel moved (a diagnostic).
 * Other bits are refused (GPZ_ERR_INVALID_ARG). */
#define GPZ_FLAG_FUSED_COMPACTION 1u

/* Worst-case size in bytes of the stream for n particles of n_fields fields
 * (every block stored raw).  Returns 0 for n_fields outside 1..8. */
uint64_t gpz_bound_size(uint64_t n, int n_fields);

/* Device workspace in bytes needed by gpz_compress for n particles of
 * n_fields fields: per-block temporary outputs (at most the input size) plus
 * the prefix-sum state.  Returns 0 for n_fields outside 1..8. */
uint64_t gpz_compress_workspace_size(uint64_t n, int n_fields);

/* Device workspace in bytes needed by gpz_decompress (its status word). */
uint64_t gpz_decompress_workspace_size(void);

/* Compress (Sections 4.1-4.4).
 *   d_fields:     host array of n_fields device pointers, field f's n fp32
 *                 values at d_fields[f]; each 4-byte aligned (16-byte
 *                 alignment enables bulk-copy staging).
 *   n:            particles (0 allowed: the stream is then a bare header).
 *   p:            parameters (host).
 *   d_out:        device buffer for the stream, 16-byte aligned, of
 *                 out_capacity bytes >= gpz_bound_size(n, F).
 *   d_out_size:   device uint64_t receiving the stream size in bytes, or NULL.
 *   h_out_size:   host uint64_t receiving the stream size, or NULL.  When
 *                 not NULL the call synchronises `stream` and returns the
 *                 device-side status.
 *   d_perm:       device array of n uint32 receiving the permutation
 *                 (d_perm[i] = input index of output particle i), or NULL.
 *   d_ws/ws_size: workspace (256-byte aligned) of at least
 *                 gpz_compress_workspace_size(n, F) bytes, or NULL to let the
 *                 library allocate and free it (the call then synchronises).
 *                 Such workspaces come from the library's stream-ordered
 *                 pool on the current device, which keeps the freed memory
 *                 for later calls (see gpz_release_pooled_memory).
 * The stream is identical for every launch configuration and device. */
gpz_status gpz_compress(const float* const* d_fields, uint64_t n, const gpz_params* p,
                        void* d_out, uint64_t out_capacity, uint64_t* d_out_size,
                        uint64_t* h_out_size, uint32_t* d_perm, void* d_ws, uint64_t ws_size,
                        void* stream);

/* Compress without allocating anything (the paper has no counterpart: this is
 * a convenience of this library).  Same arguments, stream and behaviour as
 * gpz_compress with d_ws = NULL, except that no device memory is allocated:
 * the scratch space comes from a fixed 32 MiB array built into the library.
 * It is meant for callers that cannot allocate device memory when they
 * compress -- for example an in-situ hook inside a simulation whose device
 * memory is fully reserved by the simulation's own pool allocator, or a
 * latency-critical loop in which an allocation may stall the device.
 *   - When the array is taken: with CUDA's lazy module loading (the default
 *     since CUDA 12.2, and what PyTorch sets) the 32 MiB are taken on a
 *     device when the library first looks the array up there, that is at the
 *     first gpz_noalloc_prepare or gpz_compress_noalloc call with that device
 *     current; with eager loading (CUDA_MODULE_LOADING=EAGER) when the
 *     library's module is loaded.  Either way it is held until the process
 *     exits.  A caller whose own pool later reserves all remaining device
 *     memory must call gpz_noalloc_prepare on each device first, and should
 *     also do so before any stream capture.
 *   - Limit: gpz_compress_workspace_size(n, n_fields) must not exceed 32 MiB
 *     (about 8 million values n * n_fields); larger inputs return
 *     GPZ_ERR_CAPACITY and enqueue nothing.
 *   - All calls on a device share the one array, and it keeps the last
 *     call's contents; every call clears what must start at zero.  Calls whose
 *     work overlaps on the GPU (different streams, or host threads issuing
 *     concurrently) race on the array: serialise them.
 *   - Device-side errors are recorded in the array's status word.  With
 *     h_out_size the call synchronises `stream` and returns that status;
 *     without, gpz_noalloc_sync_status reads it.
 *   - The array's address is looked up on every call, so the entry point
 *     stays valid after cudaDeviceReset (the array is then taken again). */
gpz_status gpz_compress_noalloc(const float* const* d_fields, uint64_t n, const gpz_params* p,
                                void* d_out, uint64_t out_capacity, uint64_t* d_out_size,
                                uint64_t* h_out_size, uint32_t* d_perm, void* stream);

/* Take the scratch array of gpz_compress_noalloc on the current device now
 * (see there), so that a later pool reservation or stream capture cannot
 * stand in its way.  Returns GPZ_OK, or GPZ_ERR_CUDA when the array cannot
 * be taken (for example the device has no 32 MiB left). */
gpz_status gpz_noalloc_prepare(void);

/* Synchronise `stream`, return the status that the kernels of earlier
 * gpz_compress_noalloc calls on the current device recorded in the scratch
 * array (GPZ_OK if none), and clear it.  The next gpz_compress_noalloc call
 * also clears it when it starts. */
gpz_status gpz_noalloc_sync_status(void* stream);

/* Decompress (Section 3.2, last paragraph: the inverse without sorting).
 *   d_in/in_size: the stream (device, 4-byte aligned) and its size in bytes.
 *   d_fields:     host array of n_fields device pointers, each receiving n
 *                 fp32 values in the stream's block-sorted order.
 *   n_fields, n:  must match the stream header, else GPZ_ERR_CORRUPT.
 *   d_ws/ws_size: workspace of gpz_decompress_workspace_size() bytes, or
 *                 NULL (the call then allocates from the library's pool,
 *                 synchronises and returns the device-side status).
 * A stream that fails a format check sets GPZ_ERR_CORRUPT in the workspace
 * status; the kernels never read outside [d_in, d_in + in_size) and never
 * write outside the n values of each output field. */
gpz_status gpz_decompress(const void* d_in, uint64_t in_size, float* const* d_fields, int n_fields,
                          uint64_t n, void* d_ws, uint64_t ws_size, void* stream);

/* Copy a stream whose size is known only on the device -- the d_out_size
 * word of an earlier gpz_compress call -- from src to dst, with no host
 * round trip (the paper has no counterpart: a convenience for pipelines that
 * move compressed streams between host and device memory).  Exactly
 * min(*d_size, capacity) bytes (rounded down to whole words) are copied, by
 * a kernel enqueued on `stream` that reads *d_size when it runs.
 *   dst, src: device memory, or page-locked host memory that the device can
 *             address (with unified addressing, every cudaHostAlloc /
 *             cudaMallocHost allocation), 4-byte aligned (16-byte alignment of
 *             both enables 16-byte copies); the ranges must not overlap.
 *   d_size:   device (or device-addressable) uint64, 8-byte aligned.
 *   capacity: the most bytes dst can take.
 * A stream copied this way can be decompressed with in_size = the buffer's
 * capacity: gpz_decompress reads only the words the stream's header says it
 * has.  Returns GPZ_ERR_INVALID_ARG for a NULL or misaligned pointer,
 * GPZ_ERR_CUDA if the launch fails. */
gpz_status gpz_copy_stream(void* dst, const void* src, const uint64_t* d_size, uint64_t capacity, void* stream);

/* Synchronise `stream`, return the status recorded in the workspace d_ws by
 * the kernels of earlier calls (GPZ_OK if none), and clear it. */
gpz_status gpz_sync_status(void* d_ws, void* stream);

/* Parse a stream header held in host memory (at least 64 bytes). */
gpz_status gpz_inspect(const void* h_header, uint64_t len, uint64_t* n, int* n_fields,
                       int* seg_bits, int* mode);

/* Interleaved (array-of-structures) input and output: particle i's fields at
 * d_aos[i*F .. i*F+F-1], the layout of LAS-style point records (4-byte
 * aligned).  The stream is the one gpz_compress writes for the same values,
 * and decompressed particle j (block-sorted order) is d_aos[j*F ..].
 * Compression reads 16-byte aligned records directly; records only 4-byte
 * aligned, or calls with GPZ_FLAG_FUSED_COMPACTION, are first transposed into
 * structure-of-arrays form in the workspace.  Decompression writes the
 * records directly.
 *   d_ws/ws_size: workspace (256-byte aligned) of at least
 *       gpz_compress_aos_workspace_size(n, F) bytes (4*n*F more than
 *       gpz_compress needs, for the transposed copy) /
 *       gpz_decompress_aos_workspace_size(n, F) bytes (what gpz_decompress
 *       needs, rounded up to 256), or NULL to let the library
 *       allocate and free it (the call then synchronises and returns the
 *       device-side status).  With a workspace, gpz_sync_status(d_ws) reads the
 *       device-side status as for the ordinary calls.
 * Other arguments, errors and ordering as gpz_compress / gpz_decompress.
 * The workspace sizes are 0 for n_fields outside 1..8. */
uint64_t gpz_compress_aos_workspace_size(uint64_t n, int n_fields);
uint64_t gpz_decompress_aos_workspace_size(uint64_t n, int n_fields);
gpz_status gpz_compress_aos(const float* d_aos, uint64_t n, const gpz_params* p, void* d_out,
                            uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size,
                            uint32_t* d_perm, void* d_ws, uint64_t ws_size, void* stream);
gpz_status gpz_decompress_aos(const void* d_in, uint64_t in_size, float* d_aos, int n_fields,
                              uint64_t n, void* d_ws, uint64_t ws_size, void* stream);

/* fp64 input and output (Section 5.1: fp64 input is down-cast to fp32 when
 * that suffices for the error bound; Section 5.2: 64-bit intermediates when
 * the value range or precision needs them).  gpz_compress_f64 rounds every
 * value to fp32 on the GPU and finds each field's bound reduced by the largest
 * rounding error over its finite values,
 *     eb'_f = eb_f - max_i |x_i - RN32(x_i)|,
 * where eb_f is the given absolute bound or, with GPZ_EB_REL, the relative
 * bound times the fp64 range of the field's non-NaN values (the relative
 * bound itself when that range is not a finite positive number).
 *   - Every eb'_f positive (and no finite value beyond the fp32 range): the
 *     fp32 values are compressed with absolute bounds eb'_f into an ordinary
 *     version-1 stream (header mode 0); h_eb_used receives eb'_f.
 *   - Otherwise the fp64 values are compressed with the 64-bit form and
 *     bounds eb_f (gpz_compress_wide, below; header mode = p->mode); this
 *     needs out_capacity >= gpz_bound_size_wide(n, F), else GPZ_ERR_CAPACITY;
 *     h_eb_used receives eb_f.
 * Either way every decompressed value lies within eb_f of its fp64 input.
 *   d_fields:   host array of n_fields device pointers to n doubles (8-byte aligned).
 *   d_ws:       required: at least gpz_compress_f64_workspace_size(n, F) bytes,
 *               256-byte aligned.
 *   h_eb_used:  host array of n_fields doubles, or NULL.
 * The call synchronises `stream` once (after the rounding pass, to form eb').
 * Other arguments, errors and ordering as gpz_compress; gpz_sync_status(d_ws)
 * reads the device-side status.
 * gpz_decompress_f64 reads the stream's version word (one synchronisation).
 * A version-1 stream is decoded straight into the n_fields fp64 arrays (each
 * value its fp32 reconstruction, widened exactly); a version-2 stream goes to
 * gpz_decompress_wide.  The workspace (gpz_decompress_f64_workspace_size(n, F)
 * bytes, required, 256-byte aligned) holds the status word.  Otherwise as
 * gpz_decompress. */
uint64_t gpz_compress_f64_workspace_size(uint64_t n, int n_fields);
uint64_t gpz_decompress_f64_workspace_size(uint64_t n, int n_fields);
gpz_status gpz_compress_f64(const double* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                            uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size,
                            uint32_t* d_perm, void* d_ws, uint64_t ws_size, double* h_eb_used,
                            void* stream);
gpz_status gpz_decompress_f64(const void* d_in, uint64_t in_size, double* const* d_fields, int n_fields,
                              uint64_t n, void* d_ws, uint64_t ws_size, void* stream);

/* 64-bit intermediates (Section 5.2): fp64 values quantised in fp64.  Per
 * field: s = RN64(eb * 63/32), inv = RN64(1/s); a value's code is the first of
 * q, q - 1, q + 1, q = floor(fma(x - min, inv, 0.5)), below 2^53 whose
 * reconstruction fma(q, s, min) satisfies |RN64(x - x^)| <= eb less two ulps
 * (so the exact error is at most eb); a block with a non-finite value or no
 * such code is stored raw.  Sorting, run-length + delta + fixed-length coding
 * and compaction are those of the 32-bit form (Sections 4.2-4.4).  Stream
 * version 2: the header's extension holds eb and s per field as doubles (4F
 * words, low word first), block minima are doubles, code widths reach 53 bits,
 * and a raw block holds the fp64 values (two words each).
 *   gpz_bound_size_wide:  the largest stream, in bytes
 *                         (4 * (16 + 4F + 2 nblocks + 1 + 2 F n)).
 *   gpz_compress_wide:    as gpz_compress_f64 but always this form; eb_f is
 *                         the absolute bound or (GPZ_EB_REL) the relative bound
 *                         times the field's fp64 range, the rule above (the
 *                         call then synchronises once for the range);
 *                         d_ws required, gpz_compress_wide_workspace_size(n, F)
 *                         bytes, 256-byte aligned; h_eb_used (or NULL)
 *                         receives eb_f.
 *   gpz_decompress_wide:  the inverse into n_fields fp64 arrays (8-byte
 *                         aligned), block-sorted; d_ws as gpz_decompress
 *                         (required here).  Device-detected errors as
 *                         gpz_decompress. */
uint64_t gpz_bound_size_wide(uint64_t n, int n_fields);
uint64_t gpz_compress_wide_workspace_size(uint64_t n, int n_fields);
gpz_status gpz_compress_wide(const double* const* d_fields, uint64_t n, const gpz_params* p, void* d_out,
                             uint64_t out_capacity, uint64_t* d_out_size, uint64_t* h_out_size,
                             uint32_t* d_perm, void* d_ws, uint64_t ws_size, double* h_eb_used,
                             void* stream);
gpz_status gpz_decompress_wide(const void* d_in, uint64_t in_size, double* const* d_fields, int n_fields,
                               uint64_t n, void* d_ws, uint64_t ws_size, void* stream);

/* Static text for a status code. */
const char* gpz_status_str(gpz_status s);

/* Measurement hooks.  gpz_set_stage_timing(stream, 1) makes every later call
 * enqueued on that one stream (the handle passed as the calls' `stream`)
 * record CUDA events before its first kernel and after each kernel (up to
 * 8192 events between reads); calls on other streams are not affected.
 * gpz_set_stage_timing(stream, 0) stops it.  gpz_stage_times synchronises on
 * the last recorded event, writes up to max stage names ("range", "qse",
 * "scan", "compact", "decompress", ...) with their summed elapsed
 * milliseconds and launch counts since the previous read, returns the number
 * of stages, and clears the log.  names[] receives static strings. */
void gpz_set_stage_timing(void* stream, int enable);
int gpz_stage_times(const char** names, float* total_ms, int* launches, int max);

/* Kernel launches enqueued by this process since the last reset. */
uint64_t gpz_launch_count(int reset);

/* The library's workspace pool (the paper has no counterpart).  Calls given
 * no workspace (gpz_compress, gpz_decompress, gpz_compress_aos, ... with
 * d_ws = NULL) allocate it, stream-ordered, from a memory pool that the
 * library creates on the current device at the first such call.  The pool
 * keeps memory that calls have freed, so that later calls map no new pages;
 * it holds at most what the calls running at the same time needed.
 * gpz_pooled_bytes returns the bytes the current device's pool holds (0
 * before its first use).  gpz_release_pooled_memory synchronises the current
 * device and returns the pool's unused memory to the driver: GPZ_OK, or
 * GPZ_ERR_CUDA. */
uint64_t gpz_pooled_bytes(void);
gpz_status gpz_release_pooled_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* GPZ_H */
