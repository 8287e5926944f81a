/*
 * gpz_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the GPZ particle
 * compressor (Li et al., "GPZ: GPU-Accelerated Lossy Compressor for Particle
 * Data", arXiv 2508.10305).  It exists to check the CUDA library bit for bit.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does.  It shares no code, header,
 * table or constant with the CUDA library: everything below is defined here
 * again, from the paper and from the stream-format readings documented in
 * the repository's design notes.
 *
 * All entry points are synchronous, take host pointers, allocate only host
 * memory, and return one of the GPZO_* status codes.
 */
#ifndef GPZ_ORACLE_H
#define GPZ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GPZO_OK = 0,
    GPZO_ERR_INVALID_ARG = 1,
    GPZO_ERR_CAPACITY = 2,
    GPZO_ERR_CORRUPT = 3,
    GPZO_ERR_UNSUPPORTED = 7
};

/* Per-field quantisation constants (Section 4.1 and Section 5.1):
 * eb = error bound, s = the quantisation step (2*eb less 1/64, see the
 * source), inv = 1/s rounded once to fp32 (the "precomputed reciprocal"),
 * ebchk = the fp32 threshold used by the per-value verification. */
typedef struct {
    float eb;
    float s;
    float inv;
    float ebchk;
} gpzo_field_params;

/* Finalise the constants of one field from an absolute bound eb (> 0). */
int gpzo_params_abs(double eb, gpzo_field_params* out);

/* Relative bound: eb = rel * (max - min) over the non-NaN values of x[0..n). */
int gpzo_params_rel(double rel, const float* x, uint64_t n, gpzo_field_params* out);

/* Worst-case stream size in bytes for n particles of n_fields fields
 * (block size 1024; _b: block size B in {256, 512, 1024, 2048}, else 0). */
uint64_t gpzo_bound_size(uint64_t n, int n_fields);
uint64_t gpzo_bound_size_b(uint64_t n, int n_fields, uint32_t block_size);

/* Encode one block of n_b (1..2048) particles.  fields[f] points at the
 * block's n_b values of field f.  Writes the block's words to out
 * (capacity cap_words), their count to *nwords, and, if perm_b is not NULL,
 * the block-local permutation (perm_b[j] = input index of output slot j). */
int gpzo_encode_block(const float* const* fields, int n_fields, int n_b, int seg_bits,
                      const gpzo_field_params* params, uint32_t* out, uint32_t cap_words,
                      uint32_t* nwords, uint32_t* perm_b);

/* Decode one block's words (encoded or raw) into out[f][0..n_b), given the
 * segment bits G and the per-field steps s[f] from the stream header. */
int gpzo_decode_block(const uint32_t* words, uint32_t nwords, int n_fields, int n_b, int seg_bits,
                      const float* s, float* const* out);

/* The intermediate results of encoding one block, exposed so that tests can
 * pin each step on its own.  Arrays are sized by the caller:
 *   mins[F], bits[F], q[F*n_b] (field-major), seg_id[F*n_b], seg_off[F*n_b],
 *   key[n_b], perm_b[n_b], uniq[n_b], counts[n_b].
 * *is_raw is 1 when the block falls back to raw storage; in that case only
 * the fields computed before the fallback are meaningful.  *n_unique = U. */
int gpzo_block_stages(const float* const* fields, int n_fields, int n_b, int seg_bits,
                      const gpzo_field_params* params, int* is_raw, float* mins,
                      uint32_t* bits, uint32_t* q, uint32_t* seg_id, uint32_t* seg_off,
                      uint32_t* key, uint32_t* perm_b, uint32_t* n_unique, uint32_t* uniq,
                      uint32_t* counts);

/* Fixed-length code of len values at a uniform width w (0..32): value j
 * occupies stream bits [j*w, j*w+w), least significant bit first, stream bit
 * t being bit (t mod 32) of word t/32.  Writes ceil(len*w/32) words. */
uint32_t gpzo_pack_fixed(const uint32_t* values, uint32_t len, uint32_t w, uint32_t* out);
void gpzo_unpack_fixed(const uint32_t* words, uint32_t len, uint32_t w, uint32_t* values);

/* Whole-array compression.  fields[f] -> n values (host).  mode 0 = absolute
 * bound, 1 = relative bound; eb[f] per field.  perm may be NULL, else it
 * receives n entries: perm[i] = input index of output particle i. */
int gpzo_compress(const float* const* fields, uint64_t n, int n_fields, int mode,
                  const double* eb, int seg_bits, uint8_t* out, uint64_t cap,
                  uint64_t* out_size, uint32_t* perm);

/* The same with particles grouped in blocks of block_size in {256, 512,
 * 1024, 2048} (Section 4.2 fixes 1024: 32 threads x 32 points); the header
 * records the block size, and gpzo_decompress takes it from there.  Used to
 * sweep the block size; the GPU library writes 1024 only. */
int gpzo_compress_b(const float* const* fields, uint64_t n, int n_fields, int mode,
                    const double* eb, int seg_bits, uint32_t block_size, uint8_t* out,
                    uint64_t cap, uint64_t* out_size, uint32_t* perm);

/* fp64 input (Section 5.1: fp64 input is lowered to fp32 when that is enough
 * for the bound; the test used here is the following): each
 * value is rounded to fp32 (round to nearest), and the fp32 values are
 * compressed with an absolute bound per field reduced by the largest rounding
 * error over the field's finite values:
 *     eb'_f = eb_f - max_i |x_i - RN32(x_i)|,
 * where eb_f is eb[f] (mode 0) or rel = eb[f] times the fp64 range of the
 * non-NaN values (mode 1; rel itself when that range or the product is not a
 * finite positive number).  The stream is an ordinary absolute-bound stream
 * of the fp32 values, so every decompressed value lies within eb_f of its
 * fp64 input.  GPZO_ERR_UNSUPPORTED when some eb'_f is not positive (also when
 * a finite value rounds beyond the fp32 range).  eb_used (nullable) receives
 * the F values eb'_f. */
int gpzo_compress_f64(const double* const* fields, uint64_t n, int n_fields, int mode,
                      const double* eb, int seg_bits, uint8_t* out, uint64_t cap,
                      uint64_t* out_size, uint32_t* perm, double* eb_used);

/* Inverse.  Writes n values per field, in the stream's (block-sorted) order. */
int gpzo_decompress(const uint8_t* in, uint64_t in_size, float* const* out, int n_fields,
                    uint64_t n);

/* The same, accepting a stream of any block size gpzo_compress_b writes when
 * any_block_size is nonzero (gpzo_decompress, like the GPU library, takes
 * block size 1024 only: a header with another is a corrupt stream). */
int gpzo_decompress_b(const uint8_t* in, uint64_t in_size, float* const* out, int n_fields, uint64_t n,
                      int any_block_size);

/* 64-bit intermediates (Section 5.2: 32-bit intermediates unless the value
 * range or the precision needs 64-bit ones).  fp64 values are quantised in
 * fp64 to codes below 2^53 and coded with the same four stages; the stream
 * has version 2, its per-field constants and block minima are doubles (two
 * words, low first), a raw block holds the fp64 values (two words each).
 *   gpzo_params_wide:   the step s = eb * 63/32, inv = 1/s and the check
 *                       threshold (eb less two ulps) of a bound eb.
 *   gpzo_compress_wide: eb[f] absolute (mode 0) or relative to the field's
 *                       fp64 range (mode 1, the rule of gpzo_compress_f64);
 *                       eb_used (nullable) receives the absolute bounds.
 *   gpzo_decompress_wide: the inverse, fp64 output in block-sorted order. */
int gpzo_params_wide(double eb, double* s, double* inv, double* ebchk);
uint64_t gpzo_bound_size_wide(uint64_t n, int n_fields);
int gpzo_compress_wide(const double* const* fields, uint64_t n, int n_fields, int mode,
                       const double* eb, int seg_bits, uint8_t* out, uint64_t cap,
                       uint64_t* out_size, uint32_t* perm, double* eb_used);
int gpzo_decompress_wide(const uint8_t* in, uint64_t in_size, double* const* out, int n_fields,
                         uint64_t n);

/* How many of x[0..n) fail the check with their first candidate
 * floor(fma(x - boundary_min, inv, 0.5)) under bound eb (the 64-bit form's
 * arithmetic); tests use it to probe when the check can be skipped. */
int gpzo_wide_first_candidate_failures(const double* x, uint64_t n, double boundary_min, double eb,
                                       uint64_t* failures);

#ifdef __cplusplus
}
#endif

#endif /* GPZ_ORACLE_H */
