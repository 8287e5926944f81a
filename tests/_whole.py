"""The oracle over a whole full-size array, split by contiguous ranges of
whole blocks across host threads (blocks are independent, Section 4.2), for
the whole-stream parity tests.  With a relative bound each field's absolute
bound is first taken over the whole array, exactly as the oracle's own
relative mode computes it (rel times the double range of the non-NaN
values), so that every block is encoded as in one call on the whole array.
Only the oracle runs here; ctypes releases the interpreter lock during its
C calls."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BLOCK = 1024


def absolute_bounds(x, eb, mode):
    F = x.shape[0]
    if mode == 0:
        return [float(eb)] * F
    out = []
    for f in range(F):
        v = x[f][~np.isnan(x[f])]
        rng = float(v.max()) - float(v.min()) if v.size else 0.0
        e = eb * rng
        out.append(e if (0.0 < rng < float("inf") and 0.0 < e < float("inf")) else float(eb))
    return out


def oracle_parts(oracle, x, eb, mode, G, threads=None):
    """Returns [(first particle, part stream words, part perm, part output)]."""
    F, n = x.shape
    threads = threads or os.cpu_count() or 1
    ebs = absolute_bounds(x, eb, mode)
    nb = (n + BLOCK - 1) // BLOCK
    cuts = sorted(set(min(n, (nb * k // threads) * BLOCK) for k in range(threads + 1)))

    def work(k):
        lo, hi = cuts[k], cuts[k + 1]
        part = np.ascontiguousarray(x[:, lo:hi])
        stream, perm = oracle.compress(part, ebs, 0, G, want_perm=True)
        out = oracle.decompress(stream, F, hi - lo)
        return lo, stream.view(np.uint32), perm, out

    with ThreadPoolExecutor(len(cuts) - 1) as ex:
        return list(ex.map(work, range(len(cuts) - 1)))


def compare_whole(oracle, x, eb, mode, G, stream_words, perm, out):
    """Every word of the GPU stream (header, per-field constants, offset
    table, payload), every permutation entry and every output bit against
    the oracle.  Returns the number of raw blocks in the stream."""
    F, n = x.shape
    nb = (n + BLOCK - 1) // BLOCK
    w = stream_words
    table_start = 16 + 2 * F
    payload = table_start + nb + 1
    table = w[table_start:payload].astype(np.int64)
    # header: magic, version, F, G, B, mode, n, nblocks, payload words
    assert w[0] == 0x315A5047 and w[1] == 1 and w[2] == F and w[3] == G and w[4] == BLOCK and w[5] == mode
    assert (int(w[6]) | (int(w[7]) << 32)) == n and w[8] == nb and w[9] == table[-1]
    assert w.size == payload + table[-1]
    for f in range(F):
        p = oracle.params_rel(eb, x[f]) if mode == 1 else oracle.params_abs(eb)
        assert w[table_start - 2 * F + 2 * f] == np.float32(p.eb).view(np.uint32)
        assert w[table_start - 2 * F + 2 * f + 1] == np.float32(p.s).view(np.uint32)
    raw = 0
    for lo, ps, pp, po in oracle_parts(oracle, x, eb, mode, G):
        nb_p = (po.shape[1] + BLOCK - 1) // BLOCK
        b0 = lo // BLOCK
        p_table = ps[16 + 2 * F:16 + 2 * F + nb_p + 1].astype(np.int64)
        p_payload = ps[16 + 2 * F + nb_p + 1:]
        assert np.array_equal(table[b0:b0 + nb_p + 1] - table[b0], p_table), "offset table, blocks from %d" % b0
        got = w[payload + table[b0]:payload + table[b0 + nb_p]]
        if not np.array_equal(got, p_payload):
            k = int(np.argmax(got != p_payload))
            blk = b0 + int(np.searchsorted(p_table, k, side="right")) - 1
            raise AssertionError("payload differs at word %d (block %d)" % (k, blk))
        hi = lo + po.shape[1]
        assert np.array_equal(perm[lo:hi], pp + np.uint32(lo)), "permutation, blocks from %d" % b0
        assert np.array_equal(out[:, lo:hi].view(np.uint32), po.view(np.uint32)), "output, blocks from %d" % b0
        raw += int(np.count_nonzero(p_payload[p_table[:-1]] & 1))
    return raw
