/*
 * gpz_oracle.cpp -- TEST INFRASTRUCTURE ONLY (see gpz_oracle.h).
 *
 * Plain single-threaded CPU restatement of GPZ (arXiv 2508.10305), written
 * for a reader who checks it against the paper by eye: the four stages of
 * Section 3.2 in the paper's order and notation -- spatial quantisation into
 * (segId, segOffset) with m*segId + segOffset = (p - min)/(2 eb) (Section
 * 4.1), a stable per-block sort by segId (Section 4.2), run-length + delta +
 * fixed-length coding (Section 4.3) and the three-step compaction (temporary
 * per-block output, prefix sum of sizes, copy; Section 4.4) -- plus the
 * decompressor, which undoes them without sorting (Section 3.2, last
 * paragraph).  Where the paper is silent or ambiguous, the choice made is
 * stated where it is applied, marked "Reading of the paper".
 *
 * Built with -O2 -ffp-contract=off -fno-fast-math: every fp32 operation is
 * the single IEEE operation written here (fmaf is the fused one).
 */
#include "gpz_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

/* Section 4 / Section 4.2: one block = one warp of 32 threads x 32 points. */
const uint32_t BLOCK = 1024;
/* Reading of the paper: the block size B is recorded in the stream header,
 * and the sweep of Section 4.2's trade-off (smaller blocks, more per-block
 * overhead; larger blocks, more values per sort) takes B from {256, 512,
 * 1024, 2048}; 1024 is the paper's and the default. */
const uint32_t MAX_BLOCK = 2048;
bool valid_block_size(uint32_t B) { return B == 256 || B == 512 || B == 1024 || B == 2048; }
const uint32_t STREAM_MAGIC = 0x315A5047u; /* bytes 'G','P','Z','1' */
const uint32_t STREAM_VERSION = 1;
const uint32_t STREAM_HEADER_WORDS = 16;
const int MAX_FIELDS = 8;
const int MAX_SEG_BITS = 3;
/* Reading of the paper: values are quantised only while (p-min)/(2eb)+1/2 < 2^31. */
const float Q_LIMIT = 2147483648.0f;

uint32_t bits_of(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

float float_of(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

/* Number of bits needed to write v: 0 for v = 0. */
uint32_t bit_width(uint32_t v) {
    uint32_t w = 0;
    while (v != 0) {
        ++w;
        v >>= 1;
    }
    return w;
}

uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

/* Largest float <= y (round toward -infinity). */
float float_round_down(double y) {
    float f = (float)y;
    if ((double)f > y) f = std::nextafterf(f, -INFINITY);
    return f;
}

/* Reading of the paper: the constants of one field from its bound eb (double).  The
 * step is 2 eb shrunk by 1/64 (eb * 63/32, one double product): with the
 * step at exactly 2 eb a value half-way between two lattice points is eb
 * from both, and the fp32 rounding of the reconstruction then pushes both
 * past eb.  The 1/64 margin absorbs that rounding whenever half an ulp of
 * |x| is below eb/64, and costs log2(64/63) = 0.023 bits per value. */
const double STEP_PER_EB = 1.96875;

void finalise_params(double eb, gpzo_field_params* p) {
    p->eb = (float)eb;
    p->s = (float)(eb * STEP_PER_EB);
    p->inv = (float)(1.0 / (double)p->s);
    p->ebchk = float_round_down(eb * (1.0 - std::ldexp(1.0, -22)));
}

/* ---------------- Stage 1: spatial quantisation (Section 4.1) ---------------- */

/* Reconstruction of code q: the value decompression will produce. */
float reconstruct(uint32_t q, float s, float boundary_min) {
    return std::fmaf((float)q, s, boundary_min);
}

bool within_bound(float p, uint32_t q, const gpzo_field_params& fp, float boundary_min) {
    float err = std::fabs(p - reconstruct(q, fp.s, boundary_min));
    return err <= fp.ebchk;
}

/* Reading of the paper: q = floor((p - min) * (1/(2 eb)) + 1/2) with one fused
 * multiply-add (Section 5.1), then verified; on failure q-1, then q+1.
 * Returns false when no code meets the bound (the block then goes raw). */
bool quantise(float p, float boundary_min, const gpzo_field_params& fp, uint32_t* q_out) {
    float d = p - boundary_min;
    float t = std::fmaf(d, fp.inv, 0.5f);
    if (!(t < Q_LIMIT)) return false;
    uint32_t q = (uint32_t)std::floor(t);
    if (within_bound(p, q, fp, boundary_min)) {
        *q_out = q;
        return true;
    }
    if (q > 0 && within_bound(p, q - 1, fp, boundary_min)) {
        *q_out = q - 1;
        return true;
    }
    if (within_bound(p, q + 1, fp, boundary_min)) {
        *q_out = q + 1;
        return true;
    }
    return false;
}

/* Everything the encoder derives from one block. */
struct BlockStages {
    bool raw = false;
    std::vector<float> boundary_min;          /* [F] */
    std::vector<uint32_t> bits;               /* [F] bit width of the largest code */
    std::vector<uint32_t> g;                  /* [F] segId bits (positions only) */
    std::vector<uint32_t> o;                  /* [F] segOffset bits, log2 m */
    std::vector<std::vector<uint32_t>> q;     /* [F][n_b] */
    std::vector<std::vector<uint32_t>> seg_id, seg_off; /* [F][n_b] */
    std::vector<uint32_t> key;                /* [n_b] linearised segId */
    std::vector<uint32_t> perm;               /* [n_b] sorted slot -> input index */
    std::vector<uint32_t> uniq, counts;       /* [U] run-length code */
    std::vector<uint32_t> delta;              /* [U] */
    uint32_t w_delta = 0, w_count = 0, w_record = 0;
};

int position_fields(int n_fields) { return n_fields < 3 ? n_fields : 3; }

void compute_stages(const float* const* fields, int F, int n_b, int G,
                    const gpzo_field_params* params, BlockStages* st) {
    const int P = position_fields(F);
    st->boundary_min.assign(F, 0.0f);
    st->bits.assign(F, 0);
    st->g.assign(F, 0);
    st->o.assign(F, 0);
    st->q.assign(F, std::vector<uint32_t>(n_b, 0));
    st->seg_id.assign(F, std::vector<uint32_t>(n_b, 0));
    st->seg_off.assign(F, std::vector<uint32_t>(n_b, 0));

    /* Reading of the paper: a block holding any NaN or infinity is stored raw. */
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < n_b; ++i)
            if (!std::isfinite(fields[f][i])) {
                st->raw = true;
                return;
            }

    /* Block boundary: per-axis minimum (and maximum) of the block. */
    for (int f = 0; f < F; ++f) {
        float mn = fields[f][0], mx = fields[f][0];
        for (int i = 1; i < n_b; ++i) {
            mn = std::min(mn, fields[f][i]);
            mx = std::max(mx, fields[f][i]);
        }
        (void)mx; /* Reading of the paper: only the minimum is stored; the maximum code's
                     width replaces the maximum. */
        if (mn == 0.0f) mn = 0.0f; /* Reading of the paper: a zero minimum is stored as +0 */
        st->boundary_min[f] = mn;
    }

    /* (p - boundary.min) / (2 eb) -> integer code q. */
    for (int f = 0; f < F; ++f) {
        uint32_t qmax = 0;
        for (int i = 0; i < n_b; ++i) {
            uint32_t q;
            if (!quantise(fields[f][i], st->boundary_min[f], params[f], &q)) {
                st->raw = true;
                return;
            }
            st->q[f][i] = q;
            qmax = std::max(qmax, q);
        }
        st->bits[f] = bit_width(qmax);
    }

    /* Reading of the paper: segment size m = 2^o with o = bits - min(G, bits), so each
     * axis has at most 2^G segments and m grows with the block's extent.
     * m * segId + segOffset = q. */
    for (int f = 0; f < P; ++f) {
        st->g[f] = std::min<uint32_t>((uint32_t)G, st->bits[f]);
        st->o[f] = st->bits[f] - st->g[f];
        uint32_t m = 1u << st->o[f];
        for (int i = 0; i < n_b; ++i) {
            st->seg_id[f][i] = st->q[f][i] / m;
            st->seg_off[f][i] = st->q[f][i] % m;
        }
    }

    /* Reading of the paper: the per-axis segIds are linearised row-major, axis 0 most
     * significant: key = (segId_0 * 2^g1 + segId_1) * 2^g2 + segId_2. */
    st->key.assign(n_b, 0);
    for (int i = 0; i < n_b; ++i) {
        uint32_t k = 0;
        for (int f = 0; f < P; ++f) k = k * (1u << st->g[f]) + st->seg_id[f][i];
        st->key[i] = k;
    }

    /* ---------------- Stage 2: spatial sorting (Section 4.2) ---------------- */
    /* Reading of the paper: sort by segId only; a radix sort is stable, so equal
     * segIds keep their storage order. */
    st->perm.resize(n_b);
    for (int i = 0; i < n_b; ++i) st->perm[i] = (uint32_t)i;
    std::stable_sort(st->perm.begin(), st->perm.end(),
                     [&](uint32_t a, uint32_t b) { return st->key[a] < st->key[b]; });

    /* ---------------- Stage 3: encoding (Section 4.3) ---------------- */
    /* Run-length coding of the sorted segIds: a run starts wherever the id
     * differs from its predecessor (the "transition flag"). */
    st->uniq.clear();
    st->counts.clear();
    for (int j = 0; j < n_b; ++j) {
        uint32_t id = st->key[st->perm[j]];
        bool transition = (j == 0) || (id != st->key[st->perm[j - 1]]);
        if (transition) {
            st->uniq.push_back(id);
            st->counts.push_back(1);
        } else {
            st->counts.back() += 1;
        }
    }
    /* Delta coding of the unique ids (our reading of the paper: literal differences, the
     * first against 0; counts stored as they are). */
    const size_t U = st->uniq.size();
    st->delta.assign(U, 0);
    for (size_t k = 0; k < U; ++k) st->delta[k] = (k == 0) ? st->uniq[0] : st->uniq[k] - st->uniq[k - 1];

    uint32_t dmax = 0, cmax = 0;
    for (size_t k = 0; k < U; ++k) {
        dmax = std::max(dmax, st->delta[k]);
        cmax = std::max(cmax, st->counts[k]);
    }
    st->w_delta = bit_width(dmax);
    st->w_count = bit_width(cmax);

    /* Reading of the paper: the per-particle record is the linearised segOffset of
     * the position axes followed by the codes of the extra fields, field 0
     * most significant; its width is the sum of the per-field widths. */
    uint32_t W = 0;
    for (int f = 0; f < F; ++f) W += (f < P) ? st->o[f] : st->bits[f];
    st->w_record = W;
}

/* The code of field f carried in the record of input particle i. */
uint32_t record_part(const BlockStages& st, int f, int P, uint32_t i) {
    return f < P ? st.seg_off[f][i] : st.q[f][i];
}

/* Append the low w bits of v to an LSB-first bit stream held in words. */
void put_bits(std::vector<uint32_t>& words, uint64_t& bitpos, uint32_t v, uint32_t w) {
    for (uint32_t b = 0; b < w; ++b) {
        uint64_t t = bitpos + b;
        if (t / 32 >= words.size()) words.resize(t / 32 + 1, 0);
        if ((v >> b) & 1u) words[t / 32] |= 1u << (t % 32);
    }
    bitpos += w;
}

uint32_t get_bits(const uint32_t* words, uint64_t bitpos, uint32_t w) {
    uint32_t v = 0;
    for (uint32_t b = 0; b < w; ++b) {
        uint64_t t = bitpos + b;
        v |= ((words[t / 32] >> (t % 32)) & 1u) << b;
    }
    return v;
}

/* Fixed-length coding (Section 4.3): each value at width w, words
 * ceil(len*w/32). */
std::vector<uint32_t> pack_fixed(const std::vector<uint32_t>& values, uint32_t w) {
    std::vector<uint32_t> words(ceil_div((uint64_t)values.size() * w, 32), 0);
    uint64_t bitpos = 0;
    for (uint32_t v : values) put_bits(words, bitpos, v, w);
    return words;
}

uint32_t encoded_words_needed(int F, const BlockStages& st, int n_b) {
    const uint32_t U = (uint32_t)st.uniq.size();
    return (uint32_t)F + 1 + ceil_div(F, 4) + ceil_div((uint64_t)U * st.w_delta, 32) +
           ceil_div((uint64_t)U * st.w_count, 32) + ceil_div((uint64_t)n_b * st.w_record, 32);
}

/* The words of one block: encoded, or raw when the encoder must fall back
 * or when the encoding would not be smaller (our reading of the paper). */
std::vector<uint32_t> encode_block(const float* const* fields, int F, int n_b, int G,
                                   const gpzo_field_params* params, std::vector<uint32_t>* perm_b) {
    BlockStages st;
    compute_stages(fields, F, n_b, G, params, &st);
    const int P = position_fields(F);
    const uint32_t raw_words = 1 + (uint32_t)F * (uint32_t)n_b;
    if (!st.raw && encoded_words_needed(F, st, n_b) >= raw_words) st.raw = true;

    std::vector<uint32_t> out;
    if (st.raw) {
        out.push_back(1u); /* mode word: bit 0 = raw */
        for (int f = 0; f < F; ++f)
            for (int i = 0; i < n_b; ++i) out.push_back(bits_of(fields[f][i]));
        if (perm_b) {
            perm_b->resize(n_b);
            for (int i = 0; i < n_b; ++i) (*perm_b)[i] = (uint32_t)i;
        }
        return out;
    }

    const uint32_t U = (uint32_t)st.uniq.size();
    /* Block header: mode word (bit 0 = 0: encoded) | U | w_delta | w_count,
     * then the boundary minima, then the per-field code widths, one byte
     * each. */
    out.push_back(0u | (U << 1) | (st.w_delta << 12) | (st.w_count << 17));
    for (int f = 0; f < F; ++f) out.push_back(bits_of(st.boundary_min[f]));
    std::vector<uint32_t> widths(ceil_div(F, 4), 0);
    for (int f = 0; f < F; ++f) widths[f / 4] |= st.bits[f] << (8 * (f % 4));
    out.insert(out.end(), widths.begin(), widths.end());

    /* The three arrays of Section 4.3: unique ids (as differences), their
     * counts, and the segment offsets (sorted order). */
    std::vector<uint32_t> d_words = pack_fixed(st.delta, st.w_delta);
    std::vector<uint32_t> c_words = pack_fixed(st.counts, st.w_count);
    std::vector<uint32_t> r_words(ceil_div((uint64_t)n_b * st.w_record, 32), 0);
    uint64_t bitpos = 0;
    for (int j = 0; j < n_b; ++j) {
        uint32_t i = st.perm[j];
        for (int f = F - 1; f >= 0; --f) {
            uint32_t w = f < P ? st.o[f] : st.bits[f];
            put_bits(r_words, bitpos, record_part(st, f, P, i), w);
        }
    }
    out.insert(out.end(), d_words.begin(), d_words.end());
    out.insert(out.end(), c_words.begin(), c_words.end());
    out.insert(out.end(), r_words.begin(), r_words.end());
    if (perm_b) *perm_b = st.perm;
    return out;
}

/* Decode one encoded or raw block into out[f][0..n_b).  Returns false on a
 * malformed block. */
bool decode_block(const uint32_t* w, uint32_t nwords, int F, int n_b, int G, const float* s,
                  float* const* out, uint32_t B = BLOCK) {
    if (nwords < 1) return false;
    if (w[0] & 1u) {
        if (w[0] != 1u || nwords != 1 + (uint32_t)F * (uint32_t)n_b) return false;
        for (int f = 0; f < F; ++f)
            for (int i = 0; i < n_b; ++i) out[f][i] = float_of(w[1 + (uint32_t)f * n_b + i]);
        return true;
    }
    const int P = position_fields(F);
    const uint32_t hdr = (uint32_t)F + 1 + ceil_div(F, 4);
    if (nwords < hdr) return false;
    std::vector<float> boundary_min(F);
    for (int f = 0; f < F; ++f) boundary_min[f] = float_of(w[1 + f]);
    const uint32_t mode = w[0];
    const uint32_t U = (mode >> 1) & 0x7FFu;
    const uint32_t w_delta = (mode >> 12) & 31u;
    const uint32_t w_count = (mode >> 17) & 31u;
    if ((mode >> 22) != 0) return false;
    std::vector<uint32_t> bits(F), g(F, 0), o(F, 0);
    for (int f = 0; f < F; ++f) {
        bits[f] = (w[F + 1 + f / 4] >> (8 * (f % 4))) & 0xFFu;
        if (bits[f] > 31) return false;
    }
    for (int f = F; f < 4 * (int)ceil_div(F, 4); ++f)
        if ((w[F + 1 + f / 4] >> (8 * (f % 4))) & 0xFFu) return false;
    uint32_t key_bits = 0, W = 0;
    for (int f = 0; f < F; ++f) {
        if (f < P) {
            g[f] = std::min<uint32_t>((uint32_t)G, bits[f]);
            o[f] = bits[f] - g[f];
            key_bits += g[f];
        }
        W += f < P ? o[f] : bits[f];
    }
    if (U < 1 || U > (uint32_t)n_b || U > (1u << key_bits)) return false;
    /* The deltas are at most 2^key_bits - 1 and the counts at most B
       (Section 4.3), so a width above key_bits or bit_width(B) is never
       written. */
    if (w_delta > key_bits || w_count > bit_width(B)) return false;
    const uint32_t d_len = ceil_div((uint64_t)U * w_delta, 32);
    const uint32_t c_len = ceil_div((uint64_t)U * w_count, 32);
    const uint32_t r_len = ceil_div((uint64_t)n_b * W, 32);
    if (nwords != hdr + d_len + c_len + r_len) return false;
    const uint32_t* d_words = w + hdr;
    const uint32_t* c_words = d_words + d_len;
    const uint32_t* r_words = c_words + c_len;

    /* Undo the delta and run-length codes: unique ids and their counts. */
    std::vector<uint32_t> uniq(U), counts(U);
    uint64_t total = 0;
    for (uint32_t k = 0; k < U; ++k) {
        uint32_t delta = get_bits(d_words, (uint64_t)k * w_delta, w_delta);
        if (k > 0 && delta == 0) return false; /* ids strictly increase */
        uint64_t id = (k == 0) ? delta : (uint64_t)uniq[k - 1] + delta;
        if (id >= (1ull << key_bits)) return false;
        uniq[k] = (uint32_t)id;
        counts[k] = get_bits(c_words, (uint64_t)k * w_count, w_count);
        if (counts[k] == 0) return false; /* a run holds at least one particle */
        total += counts[k];
    }
    if (total != (uint64_t)n_b) return false;

    /* Expand the runs and rebuild each code: q = m * segId + segOffset. */
    int j = 0;
    uint64_t bitpos = 0;
    for (uint32_t k = 0; k < U; ++k) {
        for (uint32_t c = 0; c < counts[k]; ++c, ++j) {
            std::vector<uint32_t> part(F, 0);
            for (int f = F - 1; f >= 0; --f) {
                uint32_t wf = f < P ? o[f] : bits[f];
                part[f] = get_bits(r_words, bitpos, wf);
                bitpos += wf;
            }
            uint32_t rest = uniq[k];
            std::vector<uint32_t> seg_id(P, 0);
            for (int f = P - 1; f >= 0; --f) {
                seg_id[f] = rest % (1u << g[f]);
                rest /= (1u << g[f]);
            }
            for (int f = 0; f < F; ++f) {
                uint32_t q = f < P ? (1u << o[f]) * seg_id[f] + part[f] : part[f];
                out[f][j] = reconstruct(q, s[f], boundary_min[f]);
            }
        }
    }
    return true;
}

uint64_t n_blocks_of(uint64_t n, uint32_t B = BLOCK) { return (n + B - 1) / B; }

bool valid_shape(int F, int G) { return F >= 1 && F <= MAX_FIELDS && G >= 0 && G <= MAX_SEG_BITS; }

} /* namespace */

extern "C" {

int gpzo_params_abs(double eb, gpzo_field_params* out) {
    if (!out || !(eb > 0.0) || !std::isfinite(eb)) return GPZO_ERR_INVALID_ARG;
    finalise_params(eb, out);
    return GPZO_OK;
}

int gpzo_params_rel(double rel, const float* x, uint64_t n, gpzo_field_params* out) {
    if (!out || !(rel > 0.0) || !std::isfinite(rel) || (n > 0 && !x)) return GPZO_ERR_INVALID_ARG;
    /* Reading of the paper: range over the non-NaN values; when it is not a finite
     * positive number the relative bound is used as an absolute one. */
    bool any = false;
    float lo = 0.0f, hi = 0.0f;
    for (uint64_t i = 0; i < n; ++i) {
        if (std::isnan(x[i])) continue;
        if (!any) {
            lo = hi = x[i];
            any = true;
        } else {
            lo = std::min(lo, x[i]);
            hi = std::max(hi, x[i]);
        }
    }
    double eb = rel;
    if (any) {
        double range = (double)hi - (double)lo;
        if (range > 0.0 && std::isfinite(range)) {
            double e = rel * range;
            if (e > 0.0 && std::isfinite(e)) eb = e;
        }
    }
    finalise_params(eb, out);
    return GPZO_OK;
}

uint64_t gpzo_bound_size_b(uint64_t n, int F, uint32_t B) {
    if (F < 1 || F > MAX_FIELDS || !valid_block_size(B)) return 0;
    uint64_t nb = n_blocks_of(n, B);
    return 4ull * (STREAM_HEADER_WORDS + 2ull * F + (nb + 1) + nb + (uint64_t)F * n);
}

uint64_t gpzo_bound_size(uint64_t n, int F) { return gpzo_bound_size_b(n, F, BLOCK); }

int gpzo_encode_block(const float* const* fields, int F, int n_b, int G,
                      const gpzo_field_params* params, uint32_t* out, uint32_t cap_words,
                      uint32_t* nwords, uint32_t* perm_b) {
    if (!fields || !params || !out || !nwords || !valid_shape(F, G) || n_b < 1 || n_b > (int)MAX_BLOCK)
        return GPZO_ERR_INVALID_ARG;
    std::vector<uint32_t> perm;
    std::vector<uint32_t> words = encode_block(fields, F, n_b, G, params, perm_b ? &perm : nullptr);
    if (words.size() > cap_words) return GPZO_ERR_CAPACITY;
    std::copy(words.begin(), words.end(), out);
    *nwords = (uint32_t)words.size();
    if (perm_b) std::copy(perm.begin(), perm.end(), perm_b);
    return GPZO_OK;
}

int gpzo_block_stages(const float* const* fields, int F, int n_b, int G,
                      const gpzo_field_params* params, int* is_raw, float* mins, uint32_t* bits,
                      uint32_t* q, uint32_t* seg_id, uint32_t* seg_off, uint32_t* key,
                      uint32_t* perm_b, uint32_t* n_unique, uint32_t* uniq, uint32_t* counts) {
    if (!fields || !params || !valid_shape(F, G) || n_b < 1 || n_b > (int)MAX_BLOCK)
        return GPZO_ERR_INVALID_ARG;
    BlockStages st;
    compute_stages(fields, F, n_b, G, params, &st);
    if (is_raw) *is_raw = st.raw ? 1 : 0;
    if (mins) std::copy(st.boundary_min.begin(), st.boundary_min.end(), mins);
    if (bits) std::copy(st.bits.begin(), st.bits.end(), bits);
    for (int f = 0; f < F; ++f) {
        if (q) std::copy(st.q[f].begin(), st.q[f].end(), q + (size_t)f * n_b);
        if (seg_id) std::copy(st.seg_id[f].begin(), st.seg_id[f].end(), seg_id + (size_t)f * n_b);
        if (seg_off) std::copy(st.seg_off[f].begin(), st.seg_off[f].end(), seg_off + (size_t)f * n_b);
    }
    if (key && !st.key.empty()) std::copy(st.key.begin(), st.key.end(), key);
    if (perm_b && !st.perm.empty()) std::copy(st.perm.begin(), st.perm.end(), perm_b);
    if (n_unique) *n_unique = (uint32_t)st.uniq.size();
    if (uniq) std::copy(st.uniq.begin(), st.uniq.end(), uniq);
    if (counts) std::copy(st.counts.begin(), st.counts.end(), counts);
    return GPZO_OK;
}

uint32_t gpzo_pack_fixed(const uint32_t* values, uint32_t len, uint32_t w, uint32_t* out) {
    std::vector<uint32_t> v(values, values + len);
    std::vector<uint32_t> words = pack_fixed(v, w);
    std::copy(words.begin(), words.end(), out);
    return (uint32_t)words.size();
}

void gpzo_unpack_fixed(const uint32_t* words, uint32_t len, uint32_t w, uint32_t* values) {
    for (uint32_t j = 0; j < len; ++j) values[j] = get_bits(words, (uint64_t)j * w, w);
}

int gpzo_decode_block(const uint32_t* words, uint32_t nwords, int F, int n_b, int G, const float* s,
                      float* const* out) {
    if (!words || !s || !out || !valid_shape(F, G) || n_b < 1 || n_b > (int)MAX_BLOCK)
        return GPZO_ERR_INVALID_ARG;
    /* the block size of a stream holding a block of n_b particles: 1024, or 2048 above it */
    const uint32_t B = n_b <= (int)BLOCK ? BLOCK : MAX_BLOCK;
    return decode_block(words, nwords, F, n_b, G, s, out, B) ? GPZO_OK : GPZO_ERR_CORRUPT;
}

int gpzo_compress(const float* const* fields, uint64_t n, int F, int mode, const double* eb,
                  int G, uint8_t* out, uint64_t cap, uint64_t* out_size, uint32_t* perm) {
    return gpzo_compress_b(fields, n, F, mode, eb, G, BLOCK, out, cap, out_size, perm);
}

int gpzo_compress_b(const float* const* fields, uint64_t n, int F, int mode, const double* eb,
                    int G, uint32_t B, uint8_t* out, uint64_t cap, uint64_t* out_size, uint32_t* perm) {
    if (!valid_shape(F, G) || !valid_block_size(B) || (mode != 0 && mode != 1) || !eb || !out || !out_size)
        return GPZO_ERR_INVALID_ARG;
    if (n > 0 && !fields) return GPZO_ERR_INVALID_ARG;
    for (int f = 0; f < F && n > 0; ++f)
        if (!fields[f]) return GPZO_ERR_INVALID_ARG;
    const uint64_t nb = n_blocks_of(n, B);
    if (nb + (uint64_t)F * n > 0xFFFFFFFFull) return GPZO_ERR_UNSUPPORTED;
    if (cap < gpzo_bound_size_b(n, F, B)) return GPZO_ERR_CAPACITY;

    std::vector<gpzo_field_params> params(F);
    for (int f = 0; f < F; ++f) {
        int rc = mode == 0 ? gpzo_params_abs(eb[f], &params[f])
                           : gpzo_params_rel(eb[f], n ? fields[f] : nullptr, n, &params[f]);
        if (rc != GPZO_OK) return rc;
    }

    /* Stages 1-3 per block into temporary per-block buffers. */
    std::vector<std::vector<uint32_t>> temp(nb);
    std::vector<uint32_t> sizes(nb);
    std::vector<const float*> block_fields(F);
    for (uint64_t b = 0; b < nb; ++b) {
        const uint64_t first = b * B;
        const int n_b = (int)std::min<uint64_t>(B, n - first);
        for (int f = 0; f < F; ++f) block_fields[f] = fields[f] + first;
        std::vector<uint32_t> perm_b;
        temp[b] = encode_block(block_fields.data(), F, n_b, G, params.data(), perm ? &perm_b : nullptr);
        sizes[b] = (uint32_t)temp[b].size();
        if (perm)
            for (int j = 0; j < n_b; ++j) perm[first + j] = (uint32_t)(first + perm_b[j]);
    }

    /* Stage 4 (Section 4.4): prefix sum of the block sizes, then copy each
     * block to its offset. */
    std::vector<uint32_t> offsets(nb + 1, 0);
    for (uint64_t b = 0; b < nb; ++b) offsets[b + 1] = offsets[b] + sizes[b];

    std::vector<uint32_t> words;
    words.push_back(STREAM_MAGIC);
    words.push_back(STREAM_VERSION);
    words.push_back((uint32_t)F);
    words.push_back((uint32_t)G);
    words.push_back(B);
    words.push_back((uint32_t)mode);
    words.push_back((uint32_t)(n & 0xFFFFFFFFull));
    words.push_back((uint32_t)(n >> 32));
    words.push_back((uint32_t)nb);
    words.push_back(offsets[nb]);
    while (words.size() < STREAM_HEADER_WORDS) words.push_back(0);
    for (int f = 0; f < F; ++f) {
        words.push_back(bits_of(params[f].eb));
        words.push_back(bits_of(params[f].s));
    }
    words.insert(words.end(), offsets.begin(), offsets.end());
    for (uint64_t b = 0; b < nb; ++b) words.insert(words.end(), temp[b].begin(), temp[b].end());

    const uint64_t bytes = 4ull * words.size();
    if (bytes > cap) return GPZO_ERR_CAPACITY;
    std::memcpy(out, words.data(), bytes);
    *out_size = bytes;
    return GPZO_OK;
}

int gpzo_compress_f64(const double* const* fields, uint64_t n, int F, int mode, const double* eb,
                      int G, uint8_t* out, uint64_t cap, uint64_t* out_size, uint32_t* perm,
                      double* eb_used) {
    if (F < 1 || F > MAX_FIELDS || (mode != 0 && mode != 1) || !eb) return GPZO_ERR_INVALID_ARG;
    if (n > 0 && !fields) return GPZO_ERR_INVALID_ARG;
    for (int f = 0; f < F && n > 0; ++f)
        if (!fields[f]) return GPZO_ERR_INVALID_ARG;
    std::vector<std::vector<float>> x32(F, std::vector<float>(n));
    std::vector<const float*> ptrs(F);
    std::vector<double> ebp(F);
    for (int f = 0; f < F; ++f) {
        if (!(eb[f] > 0.0) || !std::isfinite(eb[f])) return GPZO_ERR_INVALID_ARG;
        /* Round every value to fp32; the largest rounding error over the finite
           values, and the fp64 range of the non-NaN values. */
        double delta = 0.0, lo = 0.0, hi = 0.0;
        bool any = false;
        for (uint64_t i = 0; i < n; ++i) {
            const double v = fields[f][i];
            const float r = (float)v;
            x32[f][i] = r;
            if (std::isfinite(v)) delta = std::max(delta, std::fabs(v - (double)r));
            if (std::isnan(v)) continue;
            if (!any) {
                lo = hi = v;
                any = true;
            } else {
                lo = std::min(lo, v);
                hi = std::max(hi, v);
            }
        }
        double e = eb[f];
        if (mode == 1 && any) {
            const double range = hi - lo;
            if (range > 0.0 && std::isfinite(range)) {
                const double t = eb[f] * range;
                if (t > 0.0 && std::isfinite(t)) e = t;
            }
        }
        const double reduced = e - delta;
        if (!(reduced > 0.0) || !std::isfinite(reduced)) return GPZO_ERR_UNSUPPORTED;
        ebp[f] = reduced;
        ptrs[f] = x32[f].data();
    }
    if (eb_used)
        for (int f = 0; f < F; ++f) eb_used[f] = ebp[f];
    return gpzo_compress(ptrs.data(), n, F, 0, ebp.data(), G, out, cap, out_size, perm);
}

int gpzo_decompress(const uint8_t* in, uint64_t in_size, float* const* out, int F, uint64_t n) {
    return gpzo_decompress_b(in, in_size, out, F, n, 0);
}

int gpzo_decompress_b(const uint8_t* in, uint64_t in_size, float* const* out, int F, uint64_t n,
                      int any_block_size) {
    if (!in || F < 1 || F > MAX_FIELDS || (n > 0 && !out)) return GPZO_ERR_INVALID_ARG;
    if (in_size % 4 != 0 || in_size < 4ull * STREAM_HEADER_WORDS) return GPZO_ERR_CORRUPT;
    const uint64_t total_words = in_size / 4;
    std::vector<uint32_t> w(total_words);
    std::memcpy(w.data(), in, in_size);
    const uint32_t B = w[4];
    if (any_block_size ? !valid_block_size(B) : B != BLOCK) return GPZO_ERR_CORRUPT;
    const uint64_t nb = n_blocks_of(n, B);
    const uint64_t stream_n = (uint64_t)w[6] | ((uint64_t)w[7] << 32);
    if (w[0] != STREAM_MAGIC || w[1] != STREAM_VERSION || w[2] != (uint32_t)F ||
        w[3] > (uint32_t)MAX_SEG_BITS || w[5] > 1 || stream_n != n || w[8] != nb)
        return GPZO_ERR_CORRUPT;
    for (uint32_t k = 10; k < STREAM_HEADER_WORDS; ++k)
        if (w[k] != 0) return GPZO_ERR_CORRUPT;
    const int G = (int)w[3];
    const uint64_t table = STREAM_HEADER_WORDS + 2ull * F;
    const uint64_t payload = table + nb + 1;
    if (payload > total_words) return GPZO_ERR_CORRUPT;
    std::vector<float> s(F);
    for (int f = 0; f < F; ++f) s[f] = float_of(w[STREAM_HEADER_WORDS + 2 * f + 1]);
    const uint32_t* offsets = w.data() + table;
    if (offsets[0] != 0 || offsets[nb] != w[9] || payload + offsets[nb] > total_words)
        return GPZO_ERR_CORRUPT;
    std::vector<float*> block_out(F);
    for (uint64_t b = 0; b < nb; ++b) {
        if (offsets[b + 1] < offsets[b]) return GPZO_ERR_CORRUPT;
        const uint64_t first = b * B;
        const int n_b = (int)std::min<uint64_t>(B, n - first);
        for (int f = 0; f < F; ++f) block_out[f] = out[f] + first;
        if (!decode_block(w.data() + payload + offsets[b], offsets[b + 1] - offsets[b], F, n_b, G,
                          s.data(), block_out.data(), B))
            return GPZO_ERR_CORRUPT;
    }
    return GPZO_OK;
}

} /* extern "C" */

/* ================= 64-bit intermediates (stream version 2) =================
 *
 * Section 5.2 (shared memory usage) keeps 32-bit intermediates by default and
 * falls back to 64-bit ones when the value range or the precision needs
 * them.  Reading of the paper: the 64-bit form quantises fp64 values in fp64
 * to codes below 2^53, with the same four stages as above; what changes is
 * the arithmetic (double instead of float, 64-bit codes), the stored minima
 * and constants (doubles, two words each, low word first) and the version
 * word of the stream (2).  Everything else -- block size, segment bits, key,
 * sort, run-length + delta code, record order, offset table -- is the
 * 32-bit form's. */
namespace {

const uint32_t STREAM_VERSION_WIDE = 2;
/* Codes stay below 2^53, so every code converts to double exactly. */
const double Q_LIMIT_WIDE = 9007199254740992.0;
const uint32_t MAX_CODE_BITS_WIDE = 53;

struct WideParams {
    double eb, s, inv, ebchk;
};

/* The constants in double: the step 2 eb shrunk by 1/64 (as in the 32-bit
 * form), its reciprocal, and the check threshold eb less two ulps, so that a
 * rounded difference at most ebchk implies an exact difference at most eb
 * (the rounding of x - x^ is below 2^-53 of its size). */
void finalise_wide(double eb, WideParams* p) {
    p->eb = eb;
    p->s = eb * STEP_PER_EB;
    p->inv = 1.0 / p->s;
    p->ebchk = std::nextafter(std::nextafter(eb, 0.0), 0.0);
}

uint32_t bit_width64(uint64_t v) {
    uint32_t w = 0;
    while (v != 0) {
        ++w;
        v >>= 1;
    }
    return w;
}

void words_of_double(double d, uint32_t* lo, uint32_t* hi) {
    uint64_t u;
    std::memcpy(&u, &d, 8);
    *lo = (uint32_t)(u & 0xFFFFFFFFull);
    *hi = (uint32_t)(u >> 32);
}

double double_of_words(uint32_t lo, uint32_t hi) {
    const uint64_t u = (uint64_t)lo | ((uint64_t)hi << 32);
    double d;
    std::memcpy(&d, &u, 8);
    return d;
}

double reconstruct_wide(uint64_t q, double s, double boundary_min) {
    return std::fma((double)q, s, boundary_min);
}

bool within_bound_wide(double p, uint64_t q, const WideParams& fp, double boundary_min) {
    return std::fabs(p - reconstruct_wide(q, fp.s, boundary_min)) <= fp.ebchk;
}

/* q = floor((p - min) / (2 eb) + 1/2) with one fused multiply-add, verified;
 * then q - 1, then q + 1 (each only while it is a code below 2^53). */
bool quantise_wide(double p, double boundary_min, const WideParams& fp, uint64_t* q_out) {
    const double t = std::fma(p - boundary_min, fp.inv, 0.5);
    if (!(t < Q_LIMIT_WIDE)) return false;
    const uint64_t q = (uint64_t)std::floor(t);
    if (within_bound_wide(p, q, fp, boundary_min)) {
        *q_out = q;
        return true;
    }
    if (q > 0 && within_bound_wide(p, q - 1, fp, boundary_min)) {
        *q_out = q - 1;
        return true;
    }
    if ((double)(q + 1) < Q_LIMIT_WIDE && within_bound_wide(p, q + 1, fp, boundary_min)) {
        *q_out = q + 1;
        return true;
    }
    return false;
}

/* Append / read the low w (<= 64) bits of v, LSB first. */
void put_bits64(std::vector<uint32_t>& words, uint64_t& bitpos, uint64_t v, uint32_t w) {
    for (uint32_t b = 0; b < w; ++b) {
        const uint64_t t = bitpos + b;
        if (t / 32 >= words.size()) words.resize(t / 32 + 1, 0);
        if ((v >> b) & 1ull) words[t / 32] |= 1u << (t % 32);
    }
    bitpos += w;
}

uint64_t get_bits64(const uint32_t* words, uint64_t bitpos, uint32_t w) {
    uint64_t v = 0;
    for (uint32_t b = 0; b < w; ++b) {
        const uint64_t t = bitpos + b;
        v |= (uint64_t)((words[t / 32] >> (t % 32)) & 1u) << b;
    }
    return v;
}

/* The words of one block in the 64-bit form (see encode_block for the
 * 32-bit form, which this follows step by step). */
std::vector<uint32_t> encode_block_wide(const double* const* fields, int F, int n_b, int G,
                                        const WideParams* params, std::vector<uint32_t>* perm_b) {
    const int P = position_fields(F);
    const uint32_t raw_words = 1 + 2 * (uint32_t)F * (uint32_t)n_b;
    bool raw = false;
    /* Reading of the paper: a block holding any NaN or infinity is stored raw. */
    for (int f = 0; f < F && !raw; ++f)
        for (int i = 0; i < n_b; ++i)
            if (!std::isfinite(fields[f][i])) raw = true;

    std::vector<double> boundary_min(F, 0.0);
    std::vector<std::vector<uint64_t>> q(F, std::vector<uint64_t>(n_b, 0));
    std::vector<uint32_t> bits(F, 0), g(F, 0), o(F, 0);
    if (!raw) {
        /* Stage 1 (Section 4.1): block minimum, codes, their widths. */
        for (int f = 0; f < F && !raw; ++f) {
            double mn = fields[f][0];
            for (int i = 1; i < n_b; ++i) mn = std::min(mn, fields[f][i]);
            if (mn == 0.0) mn = 0.0; /* a zero minimum is stored as +0 */
            boundary_min[f] = mn;
            uint64_t qmax = 0;
            for (int i = 0; i < n_b; ++i) {
                if (!quantise_wide(fields[f][i], mn, params[f], &q[f][i])) {
                    raw = true;
                    break;
                }
                qmax = std::max(qmax, q[f][i]);
            }
            bits[f] = bit_width64(qmax);
        }
    }
    std::vector<uint32_t> key(n_b, 0), perm(n_b);
    std::vector<uint32_t> uniq, counts, delta;
    uint32_t w_delta = 0, w_count = 0, W = 0;
    if (!raw) {
        /* segId / segOffset with m = 2^o, o = bits - min(G, bits) */
        for (int f = 0; f < P; ++f) {
            g[f] = std::min<uint32_t>((uint32_t)G, bits[f]);
            o[f] = bits[f] - g[f];
        }
        for (int i = 0; i < n_b; ++i) {
            uint32_t k = 0;
            for (int f = 0; f < P; ++f) k = k * (1u << g[f]) + (uint32_t)(q[f][i] >> o[f]);
            key[i] = k;
        }
        /* Stage 2 (Section 4.2): stable sort by the linearised segId. */
        for (int i = 0; i < n_b; ++i) perm[i] = (uint32_t)i;
        std::stable_sort(perm.begin(), perm.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
        /* Stage 3 (Section 4.3): runs, deltas, widths. */
        for (int j = 0; j < n_b; ++j) {
            const uint32_t id = key[perm[j]];
            if (j == 0 || id != key[perm[j - 1]]) {
                uniq.push_back(id);
                counts.push_back(1);
            } else {
                counts.back() += 1;
            }
        }
        uint32_t dmax = 0, cmax = 0;
        for (size_t k = 0; k < uniq.size(); ++k) {
            delta.push_back(k == 0 ? uniq[0] : uniq[k] - uniq[k - 1]);
            dmax = std::max(dmax, delta.back());
            cmax = std::max(cmax, counts[k]);
        }
        w_delta = bit_width(dmax);
        w_count = bit_width(cmax);
        for (int f = 0; f < F; ++f) W += f < P ? o[f] : bits[f];
        const uint32_t U = (uint32_t)uniq.size();
        const uint32_t enc = 1 + 2 * (uint32_t)F + ceil_div(F, 4) + ceil_div((uint64_t)U * w_delta, 32) +
                             ceil_div((uint64_t)U * w_count, 32) + ceil_div((uint64_t)n_b * W, 32);
        if (enc >= raw_words) raw = true; /* never larger than the raw block */
    }

    std::vector<uint32_t> out;
    if (raw) {
        out.push_back(1u);
        for (int f = 0; f < F; ++f)
            for (int i = 0; i < n_b; ++i) {
                uint32_t lo, hi;
                words_of_double(fields[f][i], &lo, &hi);
                out.push_back(lo);
                out.push_back(hi);
            }
        if (perm_b) {
            perm_b->resize(n_b);
            for (int i = 0; i < n_b; ++i) (*perm_b)[i] = (uint32_t)i;
        }
        return out;
    }
    const uint32_t U = (uint32_t)uniq.size();
    out.push_back((U << 1) | (w_delta << 12) | (w_count << 17));
    for (int f = 0; f < F; ++f) {
        uint32_t lo, hi;
        words_of_double(boundary_min[f], &lo, &hi);
        out.push_back(lo);
        out.push_back(hi);
    }
    std::vector<uint32_t> widths(ceil_div(F, 4), 0);
    for (int f = 0; f < F; ++f) widths[f / 4] |= bits[f] << (8 * (f % 4));
    out.insert(out.end(), widths.begin(), widths.end());
    std::vector<uint32_t> d_words = pack_fixed(delta, w_delta);
    std::vector<uint32_t> c_words = pack_fixed(counts, w_count);
    std::vector<uint32_t> r_words(ceil_div((uint64_t)n_b * W, 32), 0);
    uint64_t bitpos = 0;
    for (int j = 0; j < n_b; ++j) {
        const uint32_t i = perm[j];
        for (int f = F - 1; f >= 0; --f) {
            const uint32_t wf = f < P ? o[f] : bits[f];
            const uint64_t part = f < P ? (q[f][i] & ((1ull << o[f]) - 1ull)) : q[f][i];
            put_bits64(r_words, bitpos, part, wf);
        }
    }
    out.insert(out.end(), d_words.begin(), d_words.end());
    out.insert(out.end(), c_words.begin(), c_words.end());
    out.insert(out.end(), r_words.begin(), r_words.end());
    if (perm_b) *perm_b = perm;
    return out;
}

bool decode_block_wide(const uint32_t* w, uint32_t nwords, int F, int n_b, int G, const double* s,
                       double* const* out) {
    if (nwords < 1) return false;
    if (w[0] & 1u) {
        if (w[0] != 1u || nwords != 1 + 2 * (uint32_t)F * (uint32_t)n_b) return false;
        for (int f = 0; f < F; ++f)
            for (int i = 0; i < n_b; ++i) {
                const uint32_t k = 1 + 2 * ((uint32_t)f * n_b + i);
                out[f][i] = double_of_words(w[k], w[k + 1]);
            }
        return true;
    }
    const int P = position_fields(F);
    const uint32_t hdr = 1 + 2 * (uint32_t)F + ceil_div(F, 4);
    if (nwords < hdr) return false;
    const uint32_t mode = w[0];
    const uint32_t U = (mode >> 1) & 0x7FFu, w_delta = (mode >> 12) & 31u, w_count = (mode >> 17) & 31u;
    if ((mode >> 22) != 0) return false;
    std::vector<double> boundary_min(F);
    for (int f = 0; f < F; ++f) boundary_min[f] = double_of_words(w[1 + 2 * f], w[2 + 2 * f]);
    const uint32_t* wb = w + 1 + 2 * F;
    std::vector<uint32_t> bits(F), g(F, 0), o(F, 0);
    for (int f = 0; f < F; ++f) {
        bits[f] = (wb[f / 4] >> (8 * (f % 4))) & 0xFFu;
        if (bits[f] > MAX_CODE_BITS_WIDE) return false;
    }
    for (int f = F; f < 4 * (int)ceil_div(F, 4); ++f)
        if ((wb[f / 4] >> (8 * (f % 4))) & 0xFFu) return false;
    uint32_t key_bits = 0, W = 0;
    for (int f = 0; f < F; ++f) {
        if (f < P) {
            g[f] = std::min<uint32_t>((uint32_t)G, bits[f]);
            o[f] = bits[f] - g[f];
            key_bits += g[f];
        }
        W += f < P ? o[f] : bits[f];
    }
    if (U < 1 || U > (uint32_t)n_b || U > (1u << key_bits)) return false;
    if (w_delta > key_bits || w_count > bit_width(BLOCK)) return false;
    const uint32_t d_len = ceil_div((uint64_t)U * w_delta, 32);
    const uint32_t c_len = ceil_div((uint64_t)U * w_count, 32);
    const uint32_t r_len = ceil_div((uint64_t)n_b * W, 32);
    if (nwords != hdr + d_len + c_len + r_len) return false;
    const uint32_t* d_words = w + hdr;
    const uint32_t* c_words = d_words + d_len;
    const uint32_t* r_words = c_words + c_len;
    std::vector<uint32_t> uniq(U), counts(U);
    uint64_t total = 0;
    for (uint32_t k = 0; k < U; ++k) {
        const uint32_t d = get_bits(d_words, (uint64_t)k * w_delta, w_delta);
        if (k > 0 && d == 0) return false;
        const uint64_t id = (k == 0) ? d : (uint64_t)uniq[k - 1] + d;
        if (id >= (1ull << key_bits)) return false;
        uniq[k] = (uint32_t)id;
        counts[k] = get_bits(c_words, (uint64_t)k * w_count, w_count);
        if (counts[k] == 0) return false;
        total += counts[k];
    }
    if (total != (uint64_t)n_b) return false;
    int j = 0;
    uint64_t bitpos = 0;
    for (uint32_t k = 0; k < U; ++k) {
        for (uint32_t c = 0; c < counts[k]; ++c, ++j) {
            std::vector<uint64_t> part(F, 0);
            for (int f = F - 1; f >= 0; --f) {
                const uint32_t wf = f < P ? o[f] : bits[f];
                part[f] = get_bits64(r_words, bitpos, wf);
                bitpos += wf;
            }
            uint32_t rest = uniq[k];
            std::vector<uint64_t> seg_id(P, 0);
            for (int f = P - 1; f >= 0; --f) {
                seg_id[f] = rest % (1u << g[f]);
                rest /= (1u << g[f]);
            }
            for (int f = 0; f < F; ++f) {
                const uint64_t qv = f < P ? (seg_id[f] << o[f]) + part[f] : part[f];
                out[f][j] = reconstruct_wide(qv, s[f], boundary_min[f]);
            }
        }
    }
    return true;
}

/* The bound of field f: eb (mode 0), or rel times the fp64 range of the
 * non-NaN values (mode 1; rel itself when that is not a finite positive
 * number) -- the rule of gpzo_compress_f64. */
double field_bound_f64(const double* x, uint64_t n, int mode, double eb) {
    if (mode == 0) return eb;
    bool any = false;
    double lo = 0.0, hi = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        if (std::isnan(x[i])) continue;
        if (!any) {
            lo = hi = x[i];
            any = true;
        } else {
            lo = std::min(lo, x[i]);
            hi = std::max(hi, x[i]);
        }
    }
    if (!any) return eb;
    const double range = hi - lo;
    if (!(range > 0.0) || !std::isfinite(range)) return eb;
    const double t = eb * range;
    return (t > 0.0 && std::isfinite(t)) ? t : eb;
}

} /* namespace */

extern "C" {

int gpzo_params_wide(double eb, double* s, double* inv, double* ebchk) {
    if (!(eb > 0.0) || !std::isfinite(eb) || !s || !inv || !ebchk) return GPZO_ERR_INVALID_ARG;
    WideParams p;
    finalise_wide(eb, &p);
    *s = p.s;
    *inv = p.inv;
    *ebchk = p.ebchk;
    return GPZO_OK;
}

int gpzo_wide_first_candidate_failures(const double* x, uint64_t n, double boundary_min, double eb,
                                       uint64_t* failures) {
    if ((n > 0 && !x) || !failures || !(eb > 0.0) || !std::isfinite(eb)) return GPZO_ERR_INVALID_ARG;
    WideParams p;
    finalise_wide(eb, &p);
    uint64_t bad = 0;
    for (uint64_t i = 0; i < n; ++i) {
        /* the first candidate of quantise_wide, and its check */
        const double t = std::fma(x[i] - boundary_min, p.inv, 0.5);
        if (!(t < Q_LIMIT_WIDE) || !within_bound_wide(x[i], (uint64_t)std::floor(t), p, boundary_min)) ++bad;
    }
    *failures = bad;
    return GPZO_OK;
}

uint64_t gpzo_bound_size_wide(uint64_t n, int F) {
    if (F < 1 || F > MAX_FIELDS) return 0;
    const uint64_t nb = n_blocks_of(n);
    return 4ull * (STREAM_HEADER_WORDS + 4ull * F + (nb + 1) + nb + 2ull * F * n);
}

int gpzo_compress_wide(const double* const* fields, uint64_t n, int F, int mode, const double* eb, int G,
                       uint8_t* out, uint64_t cap, uint64_t* out_size, uint32_t* perm, double* eb_used) {
    if (!valid_shape(F, G) || (mode != 0 && mode != 1) || !eb || !out || !out_size)
        return GPZO_ERR_INVALID_ARG;
    if (n > 0 && !fields) return GPZO_ERR_INVALID_ARG;
    for (int f = 0; f < F && n > 0; ++f)
        if (!fields[f]) return GPZO_ERR_INVALID_ARG;
    const uint64_t nb = n_blocks_of(n);
    if (nb + 2ull * F * n > 0xFFFFFFFFull) return GPZO_ERR_UNSUPPORTED;
    if (cap < gpzo_bound_size_wide(n, F)) return GPZO_ERR_CAPACITY;
    std::vector<WideParams> params(F);
    for (int f = 0; f < F; ++f) {
        if (!(eb[f] > 0.0) || !std::isfinite(eb[f])) return GPZO_ERR_INVALID_ARG;
        finalise_wide(field_bound_f64(n ? fields[f] : nullptr, n, mode, eb[f]), &params[f]);
        if (eb_used) eb_used[f] = params[f].eb;
    }
    /* Stages 1-3 per block, then the three-step compaction (Section 4.4). */
    std::vector<std::vector<uint32_t>> temp(nb);
    std::vector<uint32_t> offsets(nb + 1, 0);
    std::vector<const double*> block_fields(F);
    for (uint64_t b = 0; b < nb; ++b) {
        const uint64_t first = b * BLOCK;
        const int n_b = (int)std::min<uint64_t>(BLOCK, n - first);
        for (int f = 0; f < F; ++f) block_fields[f] = fields[f] + first;
        std::vector<uint32_t> perm_b;
        temp[b] = encode_block_wide(block_fields.data(), F, n_b, G, params.data(), perm ? &perm_b : nullptr);
        offsets[b + 1] = offsets[b] + (uint32_t)temp[b].size();
        if (perm)
            for (int j = 0; j < n_b; ++j) perm[first + j] = (uint32_t)(first + perm_b[j]);
    }
    std::vector<uint32_t> words = {STREAM_MAGIC, STREAM_VERSION_WIDE, (uint32_t)F, (uint32_t)G, BLOCK,
                                   (uint32_t)mode, (uint32_t)(n & 0xFFFFFFFFull), (uint32_t)(n >> 32),
                                   (uint32_t)nb, offsets[nb]};
    while (words.size() < STREAM_HEADER_WORDS) words.push_back(0);
    for (int f = 0; f < F; ++f) {
        uint32_t lo, hi;
        words_of_double(params[f].eb, &lo, &hi);
        words.push_back(lo);
        words.push_back(hi);
        words_of_double(params[f].s, &lo, &hi);
        words.push_back(lo);
        words.push_back(hi);
    }
    words.insert(words.end(), offsets.begin(), offsets.end());
    for (uint64_t b = 0; b < nb; ++b) words.insert(words.end(), temp[b].begin(), temp[b].end());
    const uint64_t bytes = 4ull * words.size();
    if (bytes > cap) return GPZO_ERR_CAPACITY;
    std::memcpy(out, words.data(), bytes);
    *out_size = bytes;
    return GPZO_OK;
}

int gpzo_decompress_wide(const uint8_t* in, uint64_t in_size, double* const* out, int F, uint64_t n) {
    if (!in || F < 1 || F > MAX_FIELDS || (n > 0 && !out)) return GPZO_ERR_INVALID_ARG;
    if (in_size % 4 != 0 || in_size < 4ull * STREAM_HEADER_WORDS) return GPZO_ERR_CORRUPT;
    const uint64_t total_words = in_size / 4;
    std::vector<uint32_t> w(total_words);
    std::memcpy(w.data(), in, in_size);
    const uint64_t nb = n_blocks_of(n);
    const uint64_t stream_n = (uint64_t)w[6] | ((uint64_t)w[7] << 32);
    if (w[0] != STREAM_MAGIC || w[1] != STREAM_VERSION_WIDE || w[2] != (uint32_t)F ||
        w[3] > (uint32_t)MAX_SEG_BITS || w[4] != BLOCK || w[5] > 1 || stream_n != n || w[8] != nb)
        return GPZO_ERR_CORRUPT;
    for (uint32_t k = 10; k < STREAM_HEADER_WORDS; ++k)
        if (w[k] != 0) return GPZO_ERR_CORRUPT;
    const int G = (int)w[3];
    const uint64_t table = STREAM_HEADER_WORDS + 4ull * F;
    const uint64_t payload = table + nb + 1;
    if (payload > total_words) return GPZO_ERR_CORRUPT;
    std::vector<double> s(F);
    for (int f = 0; f < F; ++f) s[f] = double_of_words(w[STREAM_HEADER_WORDS + 4 * f + 2], w[STREAM_HEADER_WORDS + 4 * f + 3]);
    const uint32_t* offsets = w.data() + table;
    if (offsets[0] != 0 || offsets[nb] != w[9] || payload + offsets[nb] > total_words) return GPZO_ERR_CORRUPT;
    std::vector<double*> block_out(F);
    for (uint64_t b = 0; b < nb; ++b) {
        if (offsets[b + 1] < offsets[b]) return GPZO_ERR_CORRUPT;
        const uint64_t first = b * BLOCK;
        const int n_b = (int)std::min<uint64_t>(BLOCK, n - first);
        for (int f = 0; f < F; ++f) block_out[f] = out[f] + first;
        if (!decode_block_wide(w.data() + payload + offsets[b], offsets[b + 1] - offsets[b], F, n_b, G, s.data(),
                               block_out.data()))
            return GPZO_ERR_CORRUPT;
    }
    return GPZO_OK;
}

} /* extern "C" */
