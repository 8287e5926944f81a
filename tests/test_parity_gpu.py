"""GPU (sm_103a, through the C ABI) against the CPU oracle, bit for bit:
the compressed stream, the permutation and the decompressed fp32 values.

Small cases are compared whole (sizes spanning several blocks and a ragged
tail, every field count, segment width, bound mode and distribution kind).
The full-size workloads -- 2^26 x 6 cosmology-like with a relative bound
(the benchmark's workload, in the benchmark's launch configuration) and
2e8 x 3 LiDAR-like with an absolute bound -- are compared on sampled blocks,
which the oracle encodes and decodes one by one, plus properties that hold at
any size (every value within eb, the offset table, the size bound)."""
import numpy as np
import pytest
import torch

from tests import _golden as gold

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


def run_gpu(gpz, x, eb, mode, G, offset=0, flags=0):
    """Compress + decompress x [F, n] on the GPU; `offset` shifts every field
    by that many floats from a 16-byte boundary (exercises the plain-load
    staging path)."""
    F, n = x.shape
    buf = torch.zeros((F, n + 8), dtype=torch.float32, device="cuda")
    buf[:, offset:offset + n] = torch.from_numpy(x).cuda()
    fields = [buf[f, offset:offset + n] for f in range(F)]
    c = gpz.Compressor(n, F, eb, mode, G, want_perm=True, flags=flags)
    size = c(fields)
    stream = c.out[:size].clone()
    d = gpz.Decompressor(n, F)
    out = d(stream, size)
    torch.cuda.synchronize()
    return stream.cpu().numpy(), c.perm[:n].cpu().numpy().astype(np.uint32), out.cpu().numpy().copy()


def assert_parity(gpz, oracle, x, eb, mode=0, G=3, offset=0, flags=0):
    F, n = x.shape
    s, p, o = run_gpu(gpz, x, eb, mode, G, offset, flags)
    rs, rp = oracle.compress(x, eb, mode, G)
    if s.size != rs.size or not np.array_equal(s, rs):
        w, rw = s.view(np.uint32), rs.view(np.uint32)
        m = min(w.size, rw.size)
        first = int(np.argmax(w[:m] != rw[:m])) if np.any(w[:m] != rw[:m]) else m
        raise AssertionError("stream differs: sizes %d vs %d, first differing word %d" % (s.size, rs.size, first))
    assert np.array_equal(p, rp), "permutation differs"
    ro = oracle.decompress(rs, F, n)
    assert np.array_equal(o.view(np.uint32), ro.view(np.uint32)), "decompressed values differ"
    return s, p, o


# ----------------------------------------------------------------------------- fixtures

@pytest.mark.parametrize("name", [n for n in gold.all_names() if "out" in gold.load(n) or "stream_words" in gold.load(n)])
def test_golden(gpz, oracle, name):
    g = gold.load(name)
    s, p, o = assert_parity(gpz, oracle, g["fields"], g["eb"], g["mode"], g["seg_bits"])
    if "stream_words" in g:
        assert s.view(np.uint32).tolist() == g["stream_words"].tolist()
    if "block_words" in g:
        F = g["n_fields"]
        assert s.view(np.uint32)[16 + 2 * F + 2:].tolist() == g["block_words"].tolist()
    if "out" in g:
        assert o.view(np.uint32).tolist() == g["out"].view(np.uint32).tolist()


# ----------------------------------------------------------------------------- randomised sweep

def gen(kind, F, n, rng):
    if kind == "uniform":
        return (rng.random((F, n)) * 256).astype(np.float32)
    if kind == "clustered":
        c = rng.random((F, 30)) * 200
        lab = np.sort(rng.integers(0, 30, n))
        return (c[:, lab] + rng.standard_normal((F, n)) * rng.uniform(0.05, 3.0)).astype(np.float32)
    if kind == "lidar":
        base = np.array([9000.0, 5000.0, 120.0, 3.0, 1.0, 0.5, 7.0, 2.0])[:F, None]
        walk = np.cumsum(rng.standard_normal((F, n)) * 0.3, axis=1)
        return (base + walk).astype(np.float32)
    if kind == "mixed":
        scale = np.array([1e3, 1e-2, 1.0, 300.0, 5.0, 1e4, 0.1, 50.0])[:F, None]
        return (rng.standard_normal((F, n)) * scale).astype(np.float32)
    raise ValueError(kind)


SIZES = [1, 2, 31, 32, 33, 1000, 1023, 1024, 1025, 2047, 3000, 4113, 5000]
CASES = []
_r = np.random.default_rng(2024)
for _i in range(48):
    CASES.append((int(_r.choice(SIZES)), int(_r.choice([1, 2, 3, 4, 6, 8])), int(_r.integers(0, 4)),
                  int(_r.integers(0, 2)), str(_r.choice(["uniform", "clustered", "lidar", "mixed"])),
                  float(_r.choice([1e-1, 1e-2, 1e-3, 1e-4])), int(_r.integers(0, 10**6))))


@pytest.mark.parametrize("n,F,G,mode,kind,eb,seed", CASES)
def test_random_parity(gpz, oracle, n, F, G, mode, kind, eb, seed):
    rng = np.random.default_rng(seed)
    x = gen(kind, F, n, rng)
    assert_parity(gpz, oracle, x, eb, mode, G)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_fields(gpz, oracle, offset):
    rng = np.random.default_rng(offset)
    x = gen("clustered", 3, 4100, rng)
    assert_parity(gpz, oracle, x, 1e-3, 0, 3, offset=offset)


def test_wide_records(gpz, oracle):
    """Records wider than 64 bits take the field-by-field packer."""
    rng = np.random.default_rng(7)
    x = (rng.random((8, 3000)) * 1000).astype(np.float32)
    s, _, _ = assert_parity(gpz, oracle, x, 1e-3, 0, 3)
    assert s.size < x.nbytes


# ----------------------------------------------------------------------------- edge cases

def test_empty(gpz, oracle):
    x = np.zeros((3, 0), np.float32)
    c = gpz.Compressor(0, 3, 1e-2)
    dummy = [torch.zeros(4, device="cuda") for _ in range(3)]
    size = c(dummy)
    rs, _ = oracle.compress(x, 1e-2)
    assert size == rs.size and np.array_equal(c.out[:size].cpu().numpy(), rs)


def test_nonfinite_blocks(gpz, oracle):
    x = (np.arange(3 * 3000, dtype=np.float32).reshape(3, 3000) * 0.01)
    x[0, 7] = np.nan
    x[1, 1500] = np.inf
    x[2, 2999] = -np.inf
    assert_parity(gpz, oracle, x, 1e-3)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("case", range(6))
def test_nonfinite_variants(gpz, oracle, case, mode):
    """Non-finite values anywhere in a block (first or last particle of a
    thread's row, a partial last block, any field), negative NaN and NaN
    payloads, blocks that are entirely +Inf or -Inf, and the largest finite
    magnitudes next to them: such blocks are stored raw, the others not."""
    rng = np.random.default_rng(300 + case)
    F = [6, 3, 1, 8, 2, 6][case]
    n = [5000, 4100, 3000, 2500, 1024, 7000][case]
    x = (rng.random((F, n)) * 100).astype(np.float32)
    u = x.view(np.uint32)
    picks = rng.integers(0, n, 6)
    u[rng.integers(0, F), 0] = 0xFFC00000  # negative NaN at a block's first particle
    u[F - 1, n - 1] = 0x7F800001           # signalling-pattern NaN at the last particle
    u[0, picks[0]] = 0x7FBFFFFF            # NaN with payload
    x[F // 2, picks[1]] = np.inf
    x[F - 1, picks[2]] = -np.inf
    x[0, picks[3]] = np.float32(3.4028235e38)    # finite extremes
    x[F - 1, picks[4]] = np.float32(-3.4028235e38)
    if n >= 3072:
        x[:, 1024:2048] = np.inf if case % 2 else -np.inf  # a whole block
    # relative bound: the range pass finds each block's extremes and marks
    # the non-finite ones for the fused kernel
    s, _, o = assert_parity(gpz, oracle, x, 1e-2 if mode == 0 else 1e-4, mode)
    assert np.isnan(o).sum() == np.isnan(x).sum() >= 2


def test_out_of_range_and_coarse(gpz, oracle):
    y = np.array([[0.0, 3e38, -3e38] * 400], np.float32)
    assert_parity(gpz, oracle, y, 1e-6)
    z = (np.float32(20000.0) + np.arange(2048, dtype=np.float32) * np.float32(0.37))[None, :]
    assert_parity(gpz, oracle, z.astype(np.float32), 1e-3)


def test_constant_and_signed_zero(gpz, oracle):
    x = np.full((4, 2500), 7.25, np.float32)
    x[0] = np.linspace(0, 1, 2500, dtype=np.float32)
    x[3, ::2] = -0.0
    x[3, 1::2] = 0.0
    assert_parity(gpz, oracle, x, 1e-4)
    assert_parity(gpz, oracle, x, 1e-4, mode=1)


def test_incompressible_goes_raw(gpz, oracle):
    rng = np.random.default_rng(1)
    x = (rng.random((3, 2048)) * 1e6).astype(np.float32)
    s, _, _ = assert_parity(gpz, oracle, x, 1e-7)
    assert s.size == oracle.bound_size(2048, 3)


def test_repeatable(gpz):
    rng = np.random.default_rng(3)
    x = gen("clustered", 6, 9000, rng)
    a = run_gpu(gpz, x, 1e-3, 1, 3)
    b = run_gpu(gpz, x, 1e-3, 1, 3)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


# ----------------------------------------------------------------------------- full-size workloads

def _full_size_check(gpz, oracle, x_dev, eb, mode, G, n_samples, seed):
    F, n = x_dev.shape
    c = gpz.Compressor(n, F, eb, mode, G, want_perm=True)
    size = c([x_dev[f] for f in range(F)])
    assert size <= gpz.gpz_bound_size(n, F)
    stream = c.out[:size]
    d = gpz.Decompressor(n, F)
    out = d(stream, size)
    perm = c.perm[:n].long()
    # every value within its bound (on the device, in double)
    x = x_dev.cpu().numpy()
    if mode == 1:
        params = [oracle.params_rel(eb, x[f]) for f in range(F)]
    else:
        params = [oracle.params_abs(eb) for _ in range(F)]
    for f in range(F):
        err = (x_dev[f][perm].double() - out[f].double()).abs().max().item()
        bound = float(np.float32(params[f].eb)) if mode == 1 else eb
        assert err <= bound, (f, err, bound)
    # header constants equal the oracle's
    w = stream.cpu().numpy().view(np.uint32)
    for f in range(F):
        assert w[16 + 2 * f] == np.float32(params[f].eb).view(np.uint32)
        assert w[16 + 2 * f + 1] == np.float32(params[f].s).view(np.uint32)
    nb = (n + 1023) // 1024
    table = w[16 + 2 * F:16 + 2 * F + nb + 1].astype(np.int64)
    assert table[0] == 0 and np.all(np.diff(table) >= 1) and table[-1] == w[9]
    payload = 16 + 2 * F + nb + 1
    # sampled blocks: oracle encodes and decodes them one by one
    rng = np.random.default_rng(seed)
    blocks = np.unique(np.concatenate([[0, nb - 1], rng.integers(0, nb, n_samples)]))
    pm = c.perm[:n].cpu().numpy().astype(np.uint32)
    o = out.cpu().numpy()
    steps = np.array([params[f].s for f in range(F)], np.float32)
    for b in blocks:
        lo, hi = b * 1024, min(n, b * 1024 + 1024)
        ref_words, ref_perm = oracle.encode_block(x[:, lo:hi], G, params)
        got = w[payload + table[b]:payload + table[b + 1]]
        assert np.array_equal(got, ref_words), "block %d differs" % b
        assert np.array_equal(pm[lo:hi] - lo, ref_perm), "block %d permutation differs" % b
        ref_out = oracle.decode_block(ref_words, F, hi - lo, G, steps)
        assert np.array_equal(o[:, lo:hi].view(np.uint32), ref_out.view(np.uint32)), "block %d output" % b
    return size


def test_small_configuration_whole(gpz, oracle):
    """1e6 particles uniform in [0,256)^3, seed 0, eb = 1e-2: whole stream."""
    from paper_2508_10305_gb300 import synth
    x = synth.uniform_box(1_000_000, seed=0)
    s, p, o = assert_parity(gpz, oracle, x, 1e-2, 0, 3)
    err = np.abs(x[:, p].astype(np.float64) - o.astype(np.float64)).max()
    assert err <= 1e-2


def test_cosmology_64m_sampled(gpz, oracle):
    """2^26 particles x 6 fields, relative bound 1e-4 (the benchmark workload)."""
    from paper_2508_10305_gb300 import synth
    x = synth.cosmology(1 << 26, seed=2, device="cuda")
    size = _full_size_check(gpz, oracle, x, 1e-4, 1, 3, n_samples=300, seed=1)
    assert x.numel() * 4 / size > 2.0


def test_lidar_200m_sampled(gpz, oracle):
    """2e8 points x 3, absolute bound 1e-3 m, scan order."""
    from paper_2508_10305_gb300 import synth
    x = synth.lidar(200_000_000, seed=3, device="cuda")
    size = _full_size_check(gpz, oracle, x, 1e-3, 0, 3, n_samples=300, seed=2)
    assert x.numel() * 4 / size > 2.0


def _whole_stream(gpz, oracle, x_dev, eb, mode, G):
    """Compress and decompress the whole array on the GPU (the benchmark's
    launch configuration) and compare everything with the oracle run over
    all host threads by block ranges.  Returns (ratio, raw blocks, blocks
    left to the general kernel)."""
    from tests import _whole
    F, n = x_dev.shape
    c = gpz.Compressor(n, F, eb, mode, G, want_perm=True)
    size = c([x_dev[f] for f in range(F)])
    general = int(c.ws[12:16].view(torch.int32).item())
    d = gpz.Decompressor(n, F)
    out = d(c.out[:size], size).cpu().numpy()
    words = c.out[:size].cpu().numpy().view(np.uint32)
    perm = c.perm[:n].cpu().numpy().view(np.uint32)
    x = x_dev.cpu().numpy()
    raw = _whole.compare_whole(oracle, x, eb, mode, G, words, perm, out)
    return x.nbytes / size, raw, general


def test_cosmology_64m_whole(gpz, oracle):
    """2^26 particles x 6 fields, relative bound 1e-4 (the benchmark
    workload): the whole stream, permutation and output, bit for bit."""
    from paper_2508_10305_gb300 import synth
    x = synth.cosmology(1 << 26, seed=2, device="cuda")
    ratio, raw, general = _whole_stream(gpz, oracle, x, 1e-4, 1, 3)
    print("cosmology 2^26 x 6: ratio %.4f, raw blocks %d, general-path blocks %d" % (ratio, raw, general))
    assert ratio > 2.0


def test_lidar_200m_whole(gpz, oracle):
    """2e8 points x 3, absolute bound 1e-3 m: the whole stream, bit for bit,
    including the blocks the fast kernel leaves to the general kernel
    (values that need a fallback candidate)."""
    from paper_2508_10305_gb300 import synth
    x = synth.lidar(200_000_000, seed=3, device="cuda")
    ratio, raw, general = _whole_stream(gpz, oracle, x, 1e-3, 0, 3)
    print("lidar 2e8 x 3: ratio %.4f, raw blocks %d, general-path blocks %d" % (ratio, raw, general))
    assert ratio > 2.0 and general > 0


@pytest.mark.parametrize("case", ["all_fast", "raw_blocks", "general_block"])
@pytest.mark.parametrize("flags", [0, 1])
def test_midsize_compaction(gpz, oracle, case, flags):
    """Arrays of a few thousand blocks (more than one wave of CTAs), with raw
    blocks and a block left to the general path, in both compaction forms:
    the stream, permutation and decompressed values are the oracle's, bit
    for bit."""
    rng = np.random.default_rng({"all_fast": 11, "raw_blocks": 12, "general_block": 13}[case])
    F, nb = 3, 3000
    n = (nb - 1) * 1024 + 333  # ragged last block
    x = (rng.random((F, n)) * 256).astype(np.float32)
    if case == "raw_blocks":
        for b in (0, 5, 1535, 1536, 1700, nb - 1):
            x[b % F, b * 1024 + 3 if b < nb - 1 else n - 2] = np.nan
    if case == "general_block":
        x[0, 2000 * 1024:2001 * 1024] *= 1e5  # codes far above 2^23: the general path
    assert_parity(gpz, oracle, x, 1e-2, 0, 3, flags=flags)


@pytest.mark.parametrize("n,F,G,mode,kind,eb,seed", [
    (1600 * 1024 + 1, 6, 3, 1, "clustered", 1e-4, 5),
    (1537 * 1024, 3, 2, 0, "lidar", 1e-3, 6),
    (2100 * 1024 + 777, 8, 1, 1, "mixed", 1e-3, 7),
    (1800 * 1024 + 5, 2, 0, 0, "uniform", 1e-2, 8),
])
def test_midsize_random(gpz, oracle, n, F, G, mode, kind, eb, seed):
    rng = np.random.default_rng(seed)
    assert_parity(gpz, oracle, gen(kind, F, n, rng), eb, mode, G)


def test_compaction_forms_agree(gpz):
    """Both compaction forms write the same bytes on the 2^26 x 6 cosmology
    snapshot (the benchmark workload); the fused form places every block
    itself."""
    from paper_2508_10305_gb300 import synth
    x = synth.cosmology(1 << 26, seed=2, device="cuda")
    F, n = x.shape
    ref = None
    for flags in (0, gpz.FLAG_FUSED_COMPACTION):
        c = gpz.Compressor(n, F, 1e-4, gpz.EB_REL, 3, flags=flags)
        size = c([x[f] for f in range(F)])
        if ref is None:
            ref = c.out[:size].clone()
        else:
            assert size == ref.numel() and torch.equal(c.out[:size], ref)
            assert gpz.compress_deferred_blocks(c.ws) < n // 1024 // 100
        del c


@pytest.mark.parametrize("case", ["all_fast", "raw_blocks", "general_block"])
def test_fused_compaction(gpz, oracle, case):
    """Fused compaction writes a block straight into the stream once every
    block before it has published its size.  Raw blocks (non-finite values)
    keep that chain going; a block left to the general path breaks it, and
    the blocks behind it go through the temporary slots and the copy kernel.
    Either way the stream is the oracle's, bit for bit."""
    rng = np.random.default_rng({"all_fast": 1, "raw_blocks": 2, "general_block": 3}[case])
    F, n = 3, 300_000
    x = (rng.random((F, n)) * 256).astype(np.float32)
    if case == "raw_blocks":
        x[1, 2 * 1024 + 5] = np.nan
        x[0, 40 * 1024 + 7] = np.inf
    if case == "general_block":
        x[0, 5 * 1024:6 * 1024] *= 1e5  # codes far above 2^23 at eb 1e-2: the general path
    nb = (n + 1023) // 1024
    xd = torch.from_numpy(x).cuda()
    c = gpz.Compressor(n, F, 1e-2, 0, 3, want_perm=True, flags=gpz.FLAG_FUSED_COMPACTION)
    size = c([xd[f] for f in range(F)])
    torch.cuda.synchronize()
    rs, rp = oracle.compress(x, 1e-2, 0, 3)
    assert size == rs.size and np.array_equal(c.out[:size].cpu().numpy(), rs)
    assert np.array_equal(c.perm[:n].cpu().numpy().astype(np.uint32), rp)
    deferred = gpz.compress_deferred_blocks(c.ws)  # blocks the copy kernel moved
    if case == "general_block":
        assert 0 < deferred <= nb - 5
    elif case == "raw_blocks":
        assert deferred == 2  # raw blocks always go through their slots
    else:
        assert deferred == 0  # every block found its offset (ordinary launch order)


@pytest.mark.parametrize("n,F,G,mode,kind,eb,seed", CASES[:16])
def test_fused_compaction_random(gpz, oracle, n, F, G, mode, kind, eb, seed):
    rng = np.random.default_rng(seed)
    assert_parity(gpz, oracle, gen(kind, F, n, rng), eb, mode, G, flags=gpz.FLAG_FUSED_COMPACTION)


def test_unchecked_first_candidates_boundary(gpz, oracle):
    """Blocks at the edge of the condition under which the fast path skips
    the check of first candidates (codes just below 2^15, ulp(max |x|) just
    below eb/512), with values on and around the midpoints between lattice
    points: the stream must equal the oracle's, which always checks."""
    from tests.test_first_candidate_bound import adversarial_block
    rng = np.random.default_rng(77)
    cases = 0
    while cases < 24:
        eb = 10.0 ** rng.uniform(-5, 1)
        blk = adversarial_block(rng, eb, int(rng.integers(13, 16)), 512)
        if blk is None:
            continue
        x1 = blk[0]
        x = np.stack([x1, rng.permutation(x1), rng.permutation(x1)]).astype(np.float32)
        assert_parity(gpz, oracle, x, float(blk[2]), 0, 3)
        cases += 1


@pytest.mark.parametrize("F,n", [(1, 4_290_000_000), (6, 715_000_000)])
def test_largest_supported_arrays_sampled(gpz, oracle, F, n):
    """The largest arrays the format addresses (blocks + F n just below 2^32
    words; about 17 GB of input), of nearly incompressible values, so that
    the stream passes 2^31 words: the offset table is monotone and closes at
    the payload size, and sampled blocks -- the first, the last, and the ones
    around the 2^31-word offset -- equal the oracle's words and decode to
    the oracle's values.  One above the limit is refused."""
    nb = (n + 1023) // 1024
    assert nb + F * n < 1 << 32
    big = gpz.make_params(F, 1e-7)
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.rand((F, n), generator=g, device="cuda", dtype=torch.float32)
    c = gpz.Compressor(n, F, 1e-7, 0, 3)
    size = c([x[f] for f in range(F)])
    payload = 16 + 2 * F + nb + 1
    assert size // 4 > (1 << 31)
    w_head = c.out[:4 * payload].view(torch.int32).cpu().numpy().view(np.uint32)
    table = w_head[16 + 2 * F:16 + 2 * F + nb + 1].astype(np.int64)
    assert table[0] == 0 and np.all(np.diff(table) >= 1) and table[-1] == w_head[9]
    assert 4 * (payload + table[-1]) == size
    d = gpz.Decompressor(n, F)
    out = d(c.out[:size], size)
    half = int(np.searchsorted(table + payload, 1 << 31))
    blocks = sorted({0, 1, nb // 2, half - 2, half - 1, min(half, nb - 1), nb - 2, nb - 1})
    params = [oracle.params_abs(1e-7) for _ in range(F)]
    steps = np.array([p.s for p in params], np.float32)
    for b in blocks:
        lo, hi = b * 1024, min(n, b * 1024 + 1024)
        xb = x[:, lo:hi].cpu().numpy()
        ref_words, _ = oracle.encode_block(xb, 3, params)
        a0, a1 = 4 * (payload + int(table[b])), 4 * (payload + int(table[b + 1]))
        got = c.out[a0:a1].view(torch.int32).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref_words), "block %d differs" % b
        ref_out = oracle.decode_block(ref_words, F, hi - lo, 3, steps)
        assert np.array_equal(out[:, lo:hi].cpu().numpy().view(np.uint32), ref_out.view(np.uint32)), b
    del c, d, out, x
    torch.cuda.empty_cache()
    # one particle more than the format addresses
    n_over = n
    while (n_over + 1023) // 1024 + F * n_over < 1 << 32:
        n_over += 1024
    dummy = torch.empty(16, dtype=torch.uint8, device="cuda")
    ptrs = [dummy] * F
    assert gpz.gpz_compress(ptrs, n_over, big, dummy, 1 << 62) == gpz.ERR_UNSUPPORTED
