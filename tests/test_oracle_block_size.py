"""Pins of the oracle's block-size parameter B (Section 4.2 fixes B = 1024,
32 threads x 32 points; the sweep also takes 256, 512 and 2048).

- A block's encoding depends only on its own particles and the field
  constants, so for B <= 1024 every block of a stream written with block
  size B equals the one block of the same particles compressed alone with
  the paper's B = 1024 (which the other pins fix), and so do its
  permutation and its decoded values.
- An array no larger than the smallest block gives the same payload at
  every B; only the header's block-size word differs.
- A block of B identical particles is hand-worked: one run of B particles,
  whose count needs bit_width(B) bits (12 at B = 2048, beyond what a
  1024-particle block ever writes).
- On keys spread uniformly over the 512 segment ids, the mean number of
  runs per block matches its closed form at every B.
"""
import numpy as np
import pytest

HDR = 16


def payload_blocks(stream, F, nb):
    w = stream.view(np.uint32)
    table = w[HDR + 2 * F:HDR + 2 * F + nb + 1]
    pay = w[HDR + 2 * F + nb + 1:]
    return [pay[table[b]:table[b + 1]] for b in range(nb)]


@pytest.mark.parametrize("B", [256, 512])
@pytest.mark.parametrize("F,G,kind", [(3, 3, "clustered"), (6, 2, "uniform"), (1, 1, "uniform")])
def test_blocks_equal_their_own_one_block_streams(oracle, B, F, G, kind):
    rng = np.random.default_rng(B + 10 * F + G)
    n = 5 * B + 37
    if kind == "uniform":
        x = (rng.random((F, n)) * 256).astype(np.float32)
    else:
        c = rng.random((F, 9)) * 200
        lab = np.sort(rng.integers(0, 9, n))
        x = (c[:, lab] + rng.standard_normal((F, n)) * 0.7).astype(np.float32)
    eb = 1e-2
    s, p = oracle.compress(x, eb, 0, G, block=B)
    w = s.view(np.uint32)
    nb = (n + B - 1) // B
    assert w[4] == B and w[8] == nb
    blocks = payload_blocks(s, F, nb)
    out = oracle.decompress(s, F, n, any_block=True)
    for k in range(nb):
        lo, hi = k * B, min(n, k * B + B)
        sk, pk = oracle.compress(np.ascontiguousarray(x[:, lo:hi]), eb, 0, G)  # B = 1024: one block
        assert np.array_equal(blocks[k], payload_blocks(sk, F, 1)[0]), k
        assert np.array_equal(p[lo:hi] - lo, pk), k
        assert np.array_equal(out[:, lo:hi].view(np.uint32), oracle.decompress(sk, F, hi - lo).view(np.uint32)), k
    assert np.abs(x[:, p].astype(np.float64) - out.astype(np.float64)).max() <= eb


def test_small_arrays_do_not_depend_on_the_block_size(oracle):
    rng = np.random.default_rng(3)
    x = (rng.random((3, 200)) * 50).astype(np.float32)
    ref = oracle.compress(x, 1e-3, 0, 3)[0].view(np.uint32)
    for B in (256, 512, 2048):
        s = oracle.compress(x, 1e-3, 0, 3, block=B)[0].view(np.uint32)
        assert s[4] == B
        d = np.flatnonzero(s != ref)
        assert d.tolist() == [4]
        assert np.array_equal(oracle.decompress(s.view(np.uint8), 3, 200, any_block=True),
                              oracle.decompress(ref.view(np.uint8), 3, 200))


@pytest.mark.parametrize("B", [256, 2048])
def test_constant_block_hand_worked(oracle, B):
    """B copies of (1.5, 2.5, 3.5), eb = 0.01: every code is 0, so every
    width is 0 and the one run holds B particles.  Block words: the mode
    word (U = 1 in bits 1-11, w_delta = 0, w_count = bit_width(B) in bits
    17-20), the three minima, one word of widths (all 0), no deltas (width
    0), one word of counts (B), no records (width 0)."""
    x = np.tile(np.array([[1.5], [2.5], [3.5]], np.float32), (1, B))
    s, p = oracle.compress(x, 1e-2, 0, 3, block=B)
    w = s.view(np.uint32)
    assert w[4] == B and w[8] == 1
    wc = int(B).bit_length()  # 9 at B = 256, 12 at B = 2048
    expect = [(1 << 1) | (0 << 12) | (wc << 17), np.float32(1.5).view(np.uint32), np.float32(2.5).view(np.uint32),
              np.float32(3.5).view(np.uint32), 0, B]
    assert payload_blocks(s, 3, 1)[0].tolist() == [int(v) for v in expect]
    assert p.tolist() == list(range(B))
    out = oracle.decompress(s, 3, B, any_block=True)
    assert np.array_equal(out, x)


def test_the_library_format_takes_block_size_1024_only(oracle):
    x = np.tile(np.array([[1.5], [2.5], [3.5]], np.float32), (1, 300))
    s, _ = oracle.compress(x, 1e-2, 0, 3, block=512)
    assert oracle.decompress_status(s, 3, 300) == oracle.ERR_CORRUPT
    assert oracle.bound_size(300, 3, block=384) == 0


@pytest.mark.parametrize("B", [256, 512, 1024, 2048])
def test_runs_per_block_match_the_closed_form(oracle, B):
    """Codes on exact lattice points k * s, k < 2^14 on every axis: each
    block's first particle has code 0 and its second 2^14 - 1, so every
    axis takes 14 bits, its segment id the top 3 (G = 3, 8 segments), and
    the key the 9-bit concatenation.  The other B - 2 particles draw their
    codes uniformly, so each of the 512 keys is hit with probability 1/512
    per particle, and the expected number of runs (distinct keys) of a
    block is 2 + 510 * (1 - (511/512)^(B - 2)) (keys 0 and 511 are always
    present)."""
    rng = np.random.default_rng(B)
    nblocks = max(16, 65536 // B)
    p = oracle.params_abs(1e-2)
    s = np.float32(p.s)
    codes = rng.integers(0, 1 << 14, size=(3, nblocks, B))
    codes[:, :, 0] = 0
    codes[:, :, 1] = (1 << 14) - 1
    x = (codes.astype(np.float64) * np.float64(s)).astype(np.float32).reshape(3, -1)
    stream, _ = oracle.compress(x, 1e-2, 0, 3, block=B)
    blocks = payload_blocks(stream, 3, nblocks)
    runs = np.array([(int(b[0]) >> 1) & 0x7FF for b in blocks])
    widths = np.array([int(b[4]) for b in blocks])
    assert np.all(widths == 14 | (14 << 8) | (14 << 16))  # every block: 14 bits per axis
    expect = 2 + 510 * (1 - (511 / 512) ** (B - 2))
    var = 510 * ((511 / 512) ** (B - 2) - (511 / 512) ** (2 * (B - 2)))  # ~ the variance, keys nearly independent
    tol = 4 * np.sqrt(var / nblocks) + 0.5
    assert abs(runs.mean() - expect) < tol, (runs.mean(), expect, tol)
