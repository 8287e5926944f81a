"""The 64-bit-intermediate codec through the C ABI (gpz_compress_wide /
gpz_decompress_wide) against the oracle, bit for bit: the stream, the
permutation, the bounds used and the decompressed fp64 values, on sizes that
span several blocks and a ragged tail, every field count, segment width and
bound mode, codes of up to 53 bits; damaged streams get the oracle's
status; the 2^26 x 6 snapshot in fp64 is checked on sampled blocks (each
re-encoded by the oracle with the same absolute bound) and on the bound of
every value."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


def gen(kind, F, n, rng):
    if kind == "uniform":
        return (rng.random((F, n)) - 0.25) * 1e3
    if kind == "clustered":
        c = rng.random((F, 30)) * 200
        lab = np.sort(rng.integers(0, 30, n))
        return c[:, lab] + rng.standard_normal((F, n)) * rng.uniform(0.05, 3.0)
    if kind == "walk":
        base = np.array([9000.0, 5000.0, 120.0, 3.0, 1.0, 0.5, 7.0, 2.0])[:F, None]
        return base + np.cumsum(rng.standard_normal((F, n)) * 0.3, axis=1)
    scale = np.array([1e3, 1e-2, 1.0, 300.0, 5.0, 1e4, 0.1, 50.0])[:F, None]  # mixed
    return rng.standard_normal((F, n)) * scale


SIZES = [1, 5, 1023, 1024, 1025, 3000, 40_000, 100_003]
CASES = []
_r = np.random.default_rng(64)
for _i in range(28):
    CASES.append((int(_r.choice(SIZES)), int(_r.choice([1, 2, 3, 4, 6, 8])), int(_r.integers(0, 4)),
                  int(_r.integers(0, 2)), str(_r.choice(["uniform", "clustered", "walk", "mixed"])),
                  float(_r.choice([1e-3, 1e-7, 1e-10, 1e-13])), int(_r.integers(0, 10**6))))


def check_parity(gpz, oracle, x, eb, mode, G):
    F, n = x.shape
    s, p, used = gpz.compress_wide(torch.from_numpy(x).cuda(), eb, mode, G, want_perm=True)
    rs, rp, rused = oracle.compress_wide(x, eb, mode, G)
    assert np.array_equal(np.array(used), rused), "bounds differ"
    g = s.cpu().numpy()
    if g.size != rs.size or not np.array_equal(g, rs):
        w, rw = g.view(np.uint32), rs.view(np.uint32)
        m = min(w.size, rw.size)
        first = int(np.argmax(w[:m] != rw[:m])) if np.any(w[:m] != rw[:m]) else m
        raise AssertionError("stream differs: sizes %d vs %d, first differing word %d" % (g.size, rs.size, first))
    assert np.array_equal(p.cpu().numpy().astype(np.uint32), rp), "permutation differs"
    out = gpz.decompress_wide(s, F, n).cpu().numpy()
    ref = oracle.decompress_wide(rs, F, n)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64)), "decompressed values differ"
    return out, rp, rused


@pytest.mark.parametrize("n,F,G,mode,kind,eb,seed", CASES)
def test_random_parity(gpz, oracle, n, F, G, mode, kind, eb, seed):
    rng = np.random.default_rng(seed)
    x = gen(kind, F, n, rng)
    out, rp, used = check_parity(gpz, oracle, x, eb, mode, G)
    assert np.all(np.abs(x[:, rp] - out) <= np.array(used)[:, None])


def test_special_blocks(gpz, oracle):
    """Raw blocks (NaN, infinities), a constant block, a block whose codes
    reach 2^53 (stored raw), and a block of one value."""
    rng = np.random.default_rng(5)
    F, n = 4, 5 * 1024 + 1
    x = rng.random((F, n)) * 100
    x[1, 10] = np.nan
    x[3, 1100] = np.inf
    x[:, 2048:3072] = 42.0
    x[0, 3072:4096] = np.linspace(0.0, 1e6, 1024)  # 1e6 / 2e-13 > 2^53: raw
    check_parity(gpz, oracle, x, 1e-13, 0, 3)


def test_unchecked_first_candidates(gpz, oracle):
    """Blocks at the edge of the condition under which the GPU skips the
    check of first candidates (code range up to 2^40 steps, |x| up to
    2^45 eb): values on the half-steps between lattice points, where the
    first candidate's error is s/2 = 0.984 eb, and the same values shifted by
    a few ulps.  The stream must equal the oracle's, which always checks;
    a second field just outside the condition takes the checked path."""
    rng = np.random.default_rng(40)
    eb, s = 1.0, 1.96875
    base = 2.0 ** 45 - 2.0 ** 41
    k = np.sort(rng.integers(0, 2 ** 40 - 2, size=3000)).astype(np.float64)
    k[0], k[-1] = 0.0, 2.0 ** 40 - 2
    x0 = base + (k + 0.5) * s  # on the 2^-6 grid, exactly representable
    x1 = np.nextafter(np.nextafter(x0, np.inf), np.inf)
    x2 = -(2.0 ** 46) + (k + 0.5) * s * 2  # |x| above 2^45 eb: checked
    x = np.stack([x0, x1, x2])
    check_parity(gpz, oracle, x, eb, 0, 3)


@pytest.mark.parametrize("W", [1, 3, 7, 8, 9, 13, 31, 32, 33, 41, 47])
@pytest.mark.parametrize("n", [1025, 3000])
def test_record_widths(gpz, oracle, W, n):
    """One field, no segment bits, values on the lattice k s with codes up to
    2^W - 1: records of exactly W bits (below 8 bits words are gathered from
    the codes, from 8 bits on each thread appends its four records), with a
    last block of 1 or 952 records."""
    rng = np.random.default_rng(W * 7 + n)
    s = 63 * 2.0 ** -15
    k = rng.integers(0, 2 ** W, size=n, dtype=np.uint64)
    k[0], k[1] = 0, 2 ** W - 1
    check_parity(gpz, oracle, (k.astype(np.float64) * s)[None, :], 2.0 ** -10, 0, 0)


def test_empty_and_single(gpz, oracle):
    check_parity(gpz, oracle, np.zeros((3, 0)), 1e-6, 0, 3)
    check_parity(gpz, oracle, np.array([[1.5], [-2.0]]), 1e-6, 1, 2)


def test_damaged_streams(gpz, oracle):
    """Single-bit flips and random words anywhere in a 3-field stream: the
    GPU decoder's status equals the oracle's, and an accepted stream decodes
    to the oracle's values."""
    rng = np.random.default_rng(21)
    F, n = 3, 5000
    x = gen("clustered", F, n, rng)
    s, _, _ = oracle.compress_wide(x, 1e-9, 0, 3)
    w = s.view(np.uint32)
    buf = torch.zeros(w.size + 8, dtype=torch.int32, device="cuda")
    out = torch.empty((F, n), dtype=torch.float64, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    L = gpz.lib

    def gpu(words):
        buf[:words.size].copy_(torch.from_numpy(words.view(np.int32)))
        st = L.gpz_decompress_wide(buf.data_ptr(), words.size * 4, gpz._ptr_array([out[f] for f in range(F)]), F, n,
                                   ws.data_ptr(), 256, None)
        if st != gpz.OK:
            return st, None
        st = gpz.gpz_sync_status(ws, None)
        return st, (out.cpu().numpy().copy() if st == gpz.OK else None)

    st, o = gpu(w)
    assert st == gpz.OK
    nb = (n + 1023) // 1024
    pay = 16 + 4 * F + nb + 1
    table = w[16 + 4 * F:pay]
    hdr = 1 + 2 * F + (F + 3) // 4
    rejected = accepted = 0
    for i in range(160):
        bad = w.copy()
        if i % 2 == 0:  # the stream header, constants and offset table
            k = int(rng.integers(0, pay))
        elif i % 4 == 1:  # a block's header, deltas or counts
            b = int(rng.integers(0, nb))
            mode = int(w[pay + table[b]])
            U, wd, wc = (mode >> 1) & 0x7FF, (mode >> 12) & 31, (mode >> 17) & 31
            k = pay + int(table[b]) + int(rng.integers(0, hdr + (U * wd + 31) // 32 + (U * wc + 31) // 32))
        else:  # anywhere
            k = int(rng.integers(0, w.size))
        if i % 4 == 3:
            bad[k] = np.uint32(rng.integers(0, 1 << 32, dtype=np.uint64))
        else:
            bad[k] ^= np.uint32(1 << int(rng.integers(0, 32)))
        rst, ref = oracle.decompress_wide_status(bad.view(np.uint8), F, n)
        st, o = gpu(bad)
        assert st == rst, "word %d: GPU %d, oracle %d" % (k, st, rst)
        if st == gpz.OK:
            accepted += 1
            assert np.array_equal(np.nan_to_num(o).view(np.uint64), np.nan_to_num(ref).view(np.uint64))
        else:
            rejected += 1
    assert rejected > 20 and accepted > 10
    st, o = gpu(w)  # still usable
    assert st == gpz.OK


def test_full_snapshot_sampled(gpz, oracle):
    """2^26 x 6 cosmology-like values in fp64 with a relative bound of 1e-12
    (far below fp32 precision): every value within its bound, and 40 sampled
    blocks equal to the oracle's encoding of the same values with the same
    absolute bounds."""
    from paper_2508_10305_gb300 import synth
    x32 = synth.cosmology(1 << 26, seed=2, device="cuda")
    F, n = x32.shape
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x = x32.double() + (torch.rand(x32.shape, generator=g, device="cuda", dtype=torch.float64) - 0.5) * 1e-3
    del x32
    s, perm, used = gpz.compress_wide(x, 1e-12, gpz.EB_REL, 3, want_perm=True)
    out = gpz.decompress_wide(s, F, n)
    p = perm.long()
    for f in range(F):
        assert torch.all((x[f][p] - out[f]).abs() <= used[f])
    w = s.cpu().numpy().view(np.uint32)
    nb = (n + 1023) // 1024
    table = w[16 + 4 * F:16 + 4 * F + nb + 1]
    pay = 16 + 4 * F + nb + 1
    rng = np.random.default_rng(3)
    for b in rng.choice(nb, 40, replace=False):
        xb = x[:, b * 1024:(b + 1) * 1024].cpu().numpy()
        rs, rp, _ = oracle.compress_wide(xb, np.array(used), 0, 3)
        rw = rs.view(np.uint32)
        mine = w[pay + table[b]:pay + table[b + 1]]
        theirs = rw[16 + 4 * F + 2:]
        assert np.array_equal(mine, theirs), "block %d" % b
        assert np.array_equal(perm[b * 1024:(b + 1) * 1024].cpu().numpy() - b * 1024, rp)
    assert x.numel() * 8 / s.numel() > 1.5
