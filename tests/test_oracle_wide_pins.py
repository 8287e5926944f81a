"""Pins of the oracle's 64-bit-intermediate form (stream version 2) to facts
that do not come from the oracle itself:

- a hand-worked stream for five values (every word derived on paper from
  the format: header, constants, table, block header, deltas, counts);
- closed forms: values on the lattice min + k*s decode exactly and carry
  the codes k (read back from the records by the stream layout), including
  codes of 33..46 bits;
- the error bound, checked exactly with rational arithmetic, at bounds far
  below the fp32 rounding error of the values (where the fp32 form refuses);
- special cases: constant block, single-value block, NaN / infinity (raw
  block holding the fp64 bit patterns);
- structural invariants: offset table, size bound, rejection of widths
  above 53 bits."""
from fractions import Fraction

import numpy as np
import pytest

STEP = 63 / 32


def words_of(x):
    return [int(v) for v in np.array([x], dtype=np.float64).view(np.uint32)]


def block_words(stream, F, n):
    """(payload start, table) of a version-2 stream."""
    w = stream.view(np.uint32)
    nb = (n + 1023) // 1024
    table = 16 + 4 * F
    return w, table + nb + 1, w[table:table + nb + 1]


def test_params_wide():
    from oracle import gpz_oracle as o
    for eb in (1.0, 1e-9, 3.7e-300, 2.0 ** -1074 * 7):
        s, inv, chk = o.params_wide(eb)
        assert s == eb * STEP and inv == 1.0 / s
        # two ulps below eb, toward zero
        assert chk == np.nextafter(np.nextafter(eb, 0.0), 0.0)
        assert Fraction(chk) <= Fraction(eb) * (1 - Fraction(1, 2 ** 53))


def test_hand_worked_stream():
    """F = 1, G = 3, eb = 2^-10, so s = 63 * 2^-15 exactly; x = 10 + k s for
    k = 5, 0, 7, 2, 5.  Codes are k (bits 3, g 3, o 0, key k, no record bits);
    stable order of the keys: inputs 1, 3, 0, 4, 2; runs (0,1) (2,1) (5,2)
    (7,1); deltas 0 2 3 2 at 2 bits -> 0b10_11_10_00 = 184; counts 1 1 2 1 at
    2 bits -> 0b01_10_01_01 = 101; mode word U<<1 | 2<<12 | 2<<17 = 270344."""
    from oracle import gpz_oracle as o
    eb = 2.0 ** -10
    s = 63 * 2.0 ** -15
    k = np.array([5, 0, 7, 2, 5])
    x = 10.0 + k * s
    stream, perm, used = o.compress_wide(x[None, :], eb, 0, 3)
    expect = [0x315A5047, 2, 1, 3, 1024, 0, 5, 0, 1, 6, 0, 0, 0, 0, 0, 0]
    expect += words_of(eb) + words_of(s)
    expect += [0, 6]
    expect += [270344] + words_of(10.0) + [3, 184, 101]
    assert stream.view(np.uint32).tolist() == expect
    assert perm.tolist() == [1, 3, 0, 4, 2]
    assert used.tolist() == [eb]
    y = o.decompress_wide(stream, 1, 5)
    assert y[0].tolist() == x[perm].tolist()  # on the lattice: exact


def read_records(w, start, n_b, widths):
    """Record j's field codes from the LSB-first record array; the last
    field is the least significant part of a record."""
    W = sum(widths)
    bits = int.from_bytes(np.ascontiguousarray(w[start:]).tobytes(), "little")
    out = []
    for j in range(n_b):
        r = (bits >> (j * W)) & ((1 << W) - 1)
        parts = []
        for wf in reversed(widths):
            parts.append(r & ((1 << wf) - 1))
            r >>= wf
        out.append(parts[::-1])
    return out


@pytest.mark.parametrize("kmax_bits,F,G", [(12, 1, 0), (33, 1, 0), (40, 2, 2), (46, 4, 3)])
def test_lattice_codes(kmax_bits, F, G):
    """x = m + k s with k < 2^kmax_bits: the codes are exactly k (the first
    candidate is exact on the lattice), the widths are bit_length(max k),
    and decompression returns x bit for bit."""
    from oracle import gpz_oracle as o
    rng = np.random.default_rng(kmax_bits)
    eb = 2.0 ** -10
    s = 63 * 2.0 ** -15
    n = 700
    k = rng.integers(0, 2 ** kmax_bits, size=(F, n), dtype=np.uint64)
    k[:, 0] = 0  # the block minimum is m
    m = np.array([3.0, -2.5, 0.0, 1.0])[:F, None]
    x = m + k.astype(np.float64) * s
    assert np.array_equal((x - m) / s, k.astype(np.float64))  # x is on the lattice exactly
    stream, perm, _ = o.compress_wide(x, eb, 0, G)
    w, pay, table = block_words(stream, F, n)
    blk = w[pay + table[0]:pay + table[1]]
    assert blk[0] & 1 == 0
    bits = [(int(blk[1 + 2 * F + f // 4]) >> (8 * (f % 4))) & 0xFF for f in range(F)]
    assert bits == [int(k[f].max()).bit_length() for f in range(F)]
    P = min(F, 3)
    g = [min(G, b) for b in bits[:P]]
    o_ = [bits[f] - g[f] for f in range(P)]
    widths = [o_[f] if f < P else bits[f] for f in range(F)]
    U = (int(blk[0]) >> 1) & 0x7FF
    wd, wc = (int(blk[0]) >> 12) & 31, (int(blk[0]) >> 17) & 31
    start = 1 + 2 * F + (F + 3) // 4 + (U * wd + 31) // 32 + (U * wc + 31) // 32
    recs = read_records(blk, start, n, widths)
    for j in range(n):
        i = perm[j]
        for f in range(F):
            kk = int(k[f, i])
            assert recs[j][f] == (kk & ((1 << o_[f]) - 1) if f < P else kk)
    y = o.decompress_wide(stream, F, n)
    assert np.array_equal(y.view(np.uint64), x[:, perm].view(np.uint64))


def exact_within(x, y, eb):
    return all(abs(Fraction(float(a)) - Fraction(float(b))) <= Fraction(float(e))
               for a, b, e in zip(x, y, eb))


@pytest.mark.parametrize("scale,eb,mode", [(1e3, 1e-9, 0), (1.0, 1e-15, 0), (5e5, 1e-12, 1), (1e-3, 1e-20, 0)])
def test_bound_exact(scale, eb, mode):
    """Every value within its bound, in exact rational arithmetic, at bounds
    that fp32 cannot meet (the fp32 form refuses these inputs)."""
    from oracle import gpz_oracle as o
    rng = np.random.default_rng(int(-np.log10(eb)))
    F, n = 3, 2500
    x = (rng.random((F, n)) - 0.3) * scale
    assert o.compress_f64_status(x, eb, mode) == o.ERR_UNSUPPORTED
    stream, perm, used = o.compress_wide(x, eb, mode)
    if mode == 1:
        assert np.allclose(used, eb * (x.max(axis=1) - x.min(axis=1)), rtol=1e-15)
    y = o.decompress_wide(stream, F, n)
    xs = x[:, perm]
    for f in range(F):
        assert exact_within(xs[f], y[f], np.full(n, used[f]))
    assert stream.size <= o.bound_size_wide(n, F)


def test_constant_and_single_value_blocks():
    from oracle import gpz_oracle as o
    x = np.full((2, 1025), 0.1)  # a full constant block, then a block of one value
    stream, perm, _ = o.compress_wide(x, 1e-12)
    w, pay, table = block_words(stream, 2, 1025)
    blk = w[pay + table[0]:pay + table[1]]
    U = (int(blk[0]) >> 1) & 0x7FF
    assert U == 1 and blk[1 + 4] == 0  # one run, widths 0
    cnt_w = (int(blk[0]) >> 17) & 31
    assert cnt_w == 11  # the run holds 1024 particles
    y = o.decompress_wide(stream, 2, 1025)
    assert np.array_equal(y, x)
    assert perm.tolist() == list(range(1025))


def test_non_finite_block_is_raw():
    from oracle import gpz_oracle as o
    rng = np.random.default_rng(3)
    x = rng.random((2, 2048))
    x[1, 1030] = np.nan
    x[0, 2000] = -np.inf
    stream, perm, _ = o.compress_wide(x, 1e-10)
    w, pay, table = block_words(stream, 2, 2048)
    blk = w[pay + table[1]:pay + table[2]]
    assert blk[0] == 1 and blk.size == 1 + 2 * 2 * 1024
    raw = blk[1:].view(np.float64).reshape(2, 1024)
    assert np.array_equal(raw.view(np.uint64), x[:, 1024:].view(np.uint64))
    assert perm[1024:].tolist() == list(range(1024, 2048))
    y = o.decompress_wide(stream, 2, 2048)
    assert np.array_equal(y[:, 1024:].view(np.uint64), x[:, 1024:].view(np.uint64))


def test_table_and_rejections():
    from oracle import gpz_oracle as o
    rng = np.random.default_rng(4)
    F, n = 3, 5000
    x = rng.random((F, n)) * 100
    stream, _, _ = o.compress_wide(x, 1e-6)
    w, pay, table = block_words(stream, F, n)
    assert table[0] == 0 and np.all(np.diff(table.astype(np.int64)) > 0)
    assert table[-1] == w[9] and w.size == pay + w[9]
    assert o.decompress_wide_status(stream, F, n)[0] == o.OK
    # a width byte above 53 is rejected
    bad = w.copy()
    b0 = pay + table[0]
    bad[b0 + 1 + 2 * F] = (bad[b0 + 1 + 2 * F] & ~np.uint32(0xFF)) | np.uint32(54)
    assert o.decompress_wide_status(bad.view(np.uint8), F, n)[0] == o.ERR_CORRUPT
    # a version-1 stream is not a version-2 stream
    s1, _ = o.compress(x.astype(np.float32), 1e-2)
    assert o.decompress_wide_status(s1, F, n)[0] == o.ERR_CORRUPT
