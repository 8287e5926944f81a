"""Editing GPZ streams at the level of the format (test helper; no part of
the method): locate a block, read and re-pack its delta and count arrays at
other widths, and rebuild the offset table and the payload size.  The tests
use it to build streams that break one rule of the format while staying
consistent in every other respect, so that a decoder is shown to reject them
for that rule alone.

Format (version 1): a 16-word header (magic, version, F, G, block size,
bound mode, n low, n high, number of blocks, payload words, six zero words),
then per field (eb, step), then nb + 1 block offsets into the payload, then
the payload.  An encoded block is: the mode word (bit 0 raw, bits 1-11 the
number of unique ids U, bits 12-16 the delta width, bits 17-21 the count
width), F minima, ceil(F/4) words of per-field code widths (one byte each),
then the deltas, the counts and the records, each a fixed-length array packed
least significant bit first (Section 4.3)."""
import numpy as np

HEADER_WORDS = 16


def get_bits(words, pos, w):
    v = 0
    for b in range(w):
        t = pos + b
        v |= ((int(words[t // 32]) >> (t % 32)) & 1) << b
    return v


def pack(values, w):
    words = [0] * ((len(values) * w + 31) // 32)
    pos = 0
    for v in values:
        assert v < (1 << w) or w == 0 and v == 0
        for b in range(w):
            if (v >> b) & 1:
                words[(pos + b) // 32] |= 1 << ((pos + b) % 32)
        pos += w
    return words


def layout(words, F):
    nb = int(words[8])
    table = HEADER_WORDS + 2 * F
    payload = table + nb + 1
    return nb, table, payload


def block_words(words, F, b):
    nb, table, payload = layout(words, F)
    lo, hi = int(words[table + b]), int(words[table + b + 1])
    return [int(v) for v in words[payload + lo:payload + hi]]


def parse_block(blk, F, G):
    """An encoded block -> dict with U, wd, wc, bits, keybits, deltas, counts, records (word list)."""
    mode = blk[0]
    assert mode & 1 == 0, "raw block"
    U, wd, wc = (mode >> 1) & 0x7FF, (mode >> 12) & 31, (mode >> 17) & 31
    hdr = 1 + F + (F + 3) // 4
    bits = [(blk[1 + F + f // 4] >> (8 * (f % 4))) & 0xFF for f in range(F)]
    P = min(F, 3)
    keybits = sum(min(G, bits[f]) for f in range(P))
    dlen, clen = (U * wd + 31) // 32, (U * wc + 31) // 32
    D = blk[hdr:hdr + dlen]
    C = blk[hdr + dlen:hdr + dlen + clen]
    return {"mode": mode, "U": U, "wd": wd, "wc": wc, "bits": bits, "keybits": keybits, "hdr": blk[:hdr],
            "deltas": [get_bits(D, k * wd, wd) for k in range(U)],
            "counts": [get_bits(C, k * wc, wc) for k in range(U)],
            "records": blk[hdr + dlen + clen:]}


def rebuild_block(p, deltas=None, counts=None, wd=None, wc=None):
    deltas = p["deltas"] if deltas is None else deltas
    counts = p["counts"] if counts is None else counts
    wd = p["wd"] if wd is None else wd
    wc = p["wc"] if wc is None else wc
    U = len(deltas)
    mode = (U << 1) | (wd << 12) | (wc << 17)
    return [mode] + list(p["hdr"][1:]) + pack(deltas, wd) + pack(counts, wc) + list(p["records"])


def replace_block(words, F, b, new_blk):
    """The stream with block b replaced (offsets and payload size adjusted)."""
    w = [int(v) for v in words]
    nb, table, payload = layout(w, F)
    lo, hi = w[table + b], w[table + b + 1]
    delta = len(new_blk) - (hi - lo)
    out = w[:payload + lo] + list(new_blk) + w[payload + hi:]
    for k in range(b + 1, nb + 1):
        out[table + k] += delta
    out[9] += delta
    return np.array(out, dtype=np.uint32)


def encoded_blocks(words, F, G):
    """Indices of the blocks that are encoded (not raw)."""
    nb, _, _ = layout(words, F)
    return [b for b in range(nb) if block_words(words, F, b)[0] & 1 == 0]
