"""Decompression of damaged streams on the GPU (through the C ABI) against the
oracle.  Every stream is written by the oracle and damaged on the host; the
GPU's status must equal the oracle's, and where both accept a stream the
decoded values must agree bit for bit (NaN payloads aside: a damaged step or
minimum may be NaN, and the payload of a NaN result is not specified).

The kernels check every word they read against the stream's size and the
format's rules (header constants, offset table, widths, run counts) before
they use it, so none of these cases reads outside the stream; the cases
cover each rule and then random single-bit flips and random words."""
import numpy as np
import pytest
import torch

from tests import _stream_edit as se

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


SEEDS = {"uniform3": 11, "clustered6": 12, "wide8": 13, "single_run": 14}


def base_stream(oracle, name):
    rng = np.random.default_rng(SEEDS[name])
    if name == "uniform3":  # five blocks, the last one partial
        F, n, G, eb = 3, 5000, 3, 1e-2
        x = (rng.random((F, n)) * 256).astype(np.float32)
    elif name == "clustered6":
        F, n, G, eb = 6, 3000, 3, 1e-3
        c = rng.random((F, 20)) * 100
        lab = np.sort(rng.integers(0, 20, n))
        x = (c[:, lab] + rng.standard_normal((F, n)) * 0.5).astype(np.float32)
    elif name == "wide8":  # records wider than 128 bits
        F, n, G, eb = 8, 2100, 3, 1e-3
        x = (rng.random((F, n)) * 1000).astype(np.float32)
    else:  # no segment bits: one run per block
        F, n, G, eb = 3, 1500, 0, 1e-2
        x = (rng.random((F, n)) * 50).astype(np.float32)
    s, _ = oracle.compress(x, eb, 0, G)
    return s.view(np.uint32).copy(), F, n, G


class GpuDecoder:
    def __init__(self, gpz, F, n, cap_words):
        self.gpz, self.F, self.n = gpz, F, n
        self.buf = torch.zeros(cap_words + 64, dtype=torch.int32, device="cuda")
        self.dec = gpz.Decompressor(n, F)

    def __call__(self, words, size_bytes=None):
        size = words.size * 4 if size_bytes is None else size_bytes
        if words.size > self.buf.numel():
            self.buf = torch.zeros(words.size + 64, dtype=torch.int32, device="cuda")
        self.buf[:words.size].copy_(torch.from_numpy(words.view(np.int32)))
        self.dec.out.fill_(0)
        try:
            out = self.dec(self.buf, size)
        except self.gpz.GpzError as e:
            return e.status, None
        return self.gpz.OK, out.cpu().numpy().copy()


def oracle_decode(oracle, words, F, n, size_bytes=None):
    b = words.view(np.uint8)
    if size_bytes is not None:
        b = b[:size_bytes]
    st = oracle.decompress_status(b, F, n)
    return st, (oracle.decompress(b, F, n) if st == oracle.OK else None)


def same_values(a, b):
    ua, ub = a.view(np.uint32), b.view(np.uint32)
    nan = np.isnan(a) & np.isnan(b)
    return bool(np.all((ua == ub) | nan))


def damaged(w, F, G, rng):
    """(label, words, size in bytes or None) for every rule, then random damage."""
    nb, table, payload = se.layout(w, F)
    cases = []

    def put(label, idx, val):
        bad = w.copy()
        bad[idx] = np.uint32(val)
        cases.append((label, bad, None))

    for idx, vals in [(0, [0, int(w[0]) ^ 1]), (1, [0, 2]), (2, [F + 1, 0]), (3, [4, 31]), (4, [512, 2048]),
                      (5, [1 - int(w[5]), 2]), (6, [int(w[6]) - 1, int(w[6]) + 1]), (7, [1]),
                      (8, [nb - 1, nb + 1]), (9, [int(w[9]) - 1, int(w[9]) + 1, 0xFFFFFFFF])]:
        for v in vals:
            put("header[%d]=%d" % (idx, v), idx, v % (1 << 32))
    for k in range(10, 16):
        put("reserved header[%d]" % k, k, 1)
    put("first offset", table, 1)
    put("last offset", table + nb, int(w[table + nb]) + 1)
    if nb >= 2:
        bad = w.copy()
        bad[table + 1], bad[table + 2] = bad[table + 2], bad[table + 1]
        cases.append(("offsets out of order", bad, None))
        put("empty block", table + 1, 0)
    cases.append(("truncated by a word", w, 4 * (w.size - 1)))
    cases.append(("header only", w, 4 * se.HEADER_WORDS))
    cases.append(("table cut", w, 4 * (payload - 1)))
    cases.append(("payload cut", w, 4 * (payload + int(w[9]) // 2)))
    cases.append(("trailing words", np.concatenate([w, np.zeros(5, np.uint32)]), None))
    for b in range(nb):
        lo = int(w[table + b])
        mode = int(w[payload + lo])
        put("block %d reserved mode bits" % b, payload + lo, mode | (1 << 22))
        put("block %d raw flag" % b, payload + lo, mode ^ 1)
        if mode & 1:
            continue
        U = (mode >> 1) & 0x7FF
        put("block %d U+1" % b, payload + lo, (mode & ~(0x7FF << 1)) | (((U + 1) & 0x7FF) << 1))
        put("block %d U-1" % b, payload + lo, (mode & ~(0x7FF << 1)) | (((U - 1) & 0x7FF) << 1))
        hdr = 1 + F + (F + 3) // 4
        put("block %d width 40" % b, payload + lo + 1 + F, (int(w[payload + lo + 1 + F]) & ~0xFF) | 40)
        if F % 4:
            put("block %d width padding" % b, payload + lo + hdr - 1, int(w[payload + lo + hdr - 1]) | (1 << 31))
        p = se.parse_block(se.block_words(w, F, b), F, G)
        for kw in [dict(wd=min(p["keybits"], 31)), dict(wd=p["keybits"] + 1), dict(wd=31), dict(wc=11),
                   dict(wc=12), dict(wc=31)]:
            cases.append(("block %d %s" % (b, kw), se.replace_block(w, F, b, se.rebuild_block(p, **kw)), None))
        if p["U"] >= 2:
            counts = list(p["counts"])
            counts[1] += counts[0]
            counts[0] = 0
            cases.append(("block %d zero count" % b,
                          se.replace_block(w, F, b, se.rebuild_block(p, counts=counts, wc=11)), None))
            deltas = list(p["deltas"])
            deltas[1] = 0
            cases.append(("block %d repeated id" % b, se.replace_block(w, F, b, se.rebuild_block(p, deltas=deltas)),
                          None))
    for i in range(150):
        bad = w.copy()
        k = int(rng.integers(0, w.size))
        bad[k] ^= np.uint32(1 << int(rng.integers(0, 32)))
        cases.append(("flip %d" % i, bad, None))
    for i in range(50):
        bad = w.copy()
        k = int(rng.integers(0, w.size))
        bad[k] = np.uint32(rng.integers(0, 1 << 32, dtype=np.uint64))
        cases.append(("random word %d" % i, bad, None))
    return cases


@pytest.mark.parametrize("name", ["uniform3", "clustered6", "wide8", "single_run"])
def test_damaged_streams_match_the_oracle(gpz, oracle, name):
    w, F, n, G = base_stream(oracle, name)
    dec = GpuDecoder(gpz, F, n, w.size + 8)
    st, out = dec(w)
    rst, ref = oracle_decode(oracle, w, F, n)
    assert st == rst == gpz.OK and same_values(out, ref)
    rng = np.random.default_rng(len(name))
    rejected = accepted = 0
    for label, words, size in damaged(w, F, G, rng):
        rst, ref = oracle_decode(oracle, words, F, n, size)
        st, out = dec(words, size)
        assert st == rst, "%s: GPU %d, oracle %d" % (label, st, rst)
        if st == gpz.OK:
            accepted += 1
            assert same_values(out, ref), label
        else:
            rejected += 1
    assert rejected > 40 and accepted > 10
    st, out = dec(w)  # the decoder is still usable
    assert st == gpz.OK and same_values(out, oracle_decode(oracle, w, F, n)[1])


def test_batch_reports_damaged_chunks(gpz, oracle):
    """Damaged chunks in a batched decompression get their own status; the
    intact ones decode exactly."""
    chunks = [base_stream(oracle, nm) for nm in ["uniform3", "clustered6", "wide8", "single_run"]]
    items, expect, refs, keep = [], [], [], []
    for c, (w, F, n, G) in enumerate(chunks):
        words = w.copy()
        if c % 2 == 1:  # damage: a rule the oracle rejects
            p = se.parse_block(se.block_words(w, F, 0), F, G)
            words = se.replace_block(w, F, 0, se.rebuild_block(p, wc=12))
        st, ref = oracle_decode(oracle, words, F, n)
        expect.append(st)
        refs.append(ref)
        d = torch.from_numpy(words.view(np.uint8).copy()).cuda()
        keep.append(d)
        items.append((d, d.numel(), F, n))
    assert expect == [oracle.OK, oracle.ERR_CORRUPT, oracle.OK, oracle.ERR_CORRUPT]
    bd = gpz.BatchDecompressor(items, use_graph=False)
    bd()
    st, per = bd.status()
    assert st == gpz.ERR_CORRUPT
    assert per == expect
    for c, (w, F, n, G) in enumerate(chunks):
        if expect[c] == oracle.OK:
            assert same_values(bd.outs[c][:, :n].cpu().numpy(), refs[c])
    bd.close()
