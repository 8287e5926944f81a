"""fp64 input and output through the C ABI (gpz_compress_f64 /
gpz_decompress_f64) against the oracle's fp64 path: the stream, the
permutation and the reduced bounds bit for bit, the widened output equal to
the oracle's values, and every value within eb of its fp64 input."""
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


def make(F, n, seed, special):
    rng = np.random.default_rng(seed)
    scale = np.array([1e4, 3.0, 250.0, 1e-3, 7.0, 1e6, 0.5, 40.0])[:F, None]
    x = (rng.random((F, n)) - 0.3) * scale
    if special and n > 10:
        x[0, 3] = np.nan
        x[F - 1, n - 2] = -np.inf
    return x


@pytest.mark.parametrize("F,n,mode,eb,special", [
    (3, 100_000, 0, 1e-3, False),
    (3, 5000, 1, 1e-4, True),
    (1, 1, 0, 1e-2, False),
    (6, 40_000, 1, 1e-5, False),
    (8, 3000, 0, 1e-1, True),  # field 5 reaches 7e5: half an fp32 ulp there is 0.016
    (2, 7777, 1, 1e-4, True),  # odd length: field 0 16-byte aligned (pairs and a last single value), field 1 not
])
def test_f64_matches_oracle(gpz, oracle, F, n, mode, eb, special):
    x = make(F, n, F * 7 + n % 13, special)
    xd = torch.from_numpy(x).cuda()
    stream, perm, used = gpz.compress_f64(xd, eb, mode, 3, want_perm=True)
    rs, rp, rused = oracle.compress_f64(x, eb, mode)
    assert np.array_equal(np.array(used), rused)
    assert stream.numel() == rs.size and np.array_equal(stream.cpu().numpy(), rs)
    assert np.array_equal(perm.cpu().numpy().astype(np.uint32), rp)
    out = gpz.decompress_f64(stream, F, n).cpu().numpy()
    ro = oracle.decompress(rs, F, n).astype(np.float64)
    assert np.array_equal(out.view(np.uint64), ro.view(np.uint64))
    xs = x[:, rp]
    with np.errstate(invalid="ignore"):
        err = np.abs(xs - out)
    ebf = np.array(used) + 0.0  # reduced bounds; the full bound adds the rounding error back
    fin = np.isfinite(xs)
    r = x.astype(np.float32).astype(np.float64)[:, rp]
    delta = np.array([np.max(np.abs(xs[f][fin[f]] - r[f][fin[f]]), initial=0.0) for f in range(F)])
    assert np.all(err[fin] <= ((ebf + delta) * (1 + 1e-12))[np.nonzero(fin)[0]])


def test_f64_rounding_edges(gpz, oracle):
    """Values on the fp32 rounding ties, at the top of the fp32 range (one
    rounds to infinity: refused), fp32-subnormal magnitudes and zeros take
    the same path as the oracle."""
    import struct
    rng = np.random.default_rng(12)
    f32 = rng.standard_normal(4096).astype(np.float32)
    ties = np.array([struct.unpack("<d", struct.pack("<Q", struct.unpack("<Q", struct.pack("<d", float(v)))[0]
                                                    | 0x10000000))[0] for v in f32])
    x = np.stack([ties, np.concatenate([rng.standard_normal(4000) * 1e-40, np.zeros(96)]),
                  rng.uniform(-1.0, 1.0, 4096) * 3.3e38])
    s, p, used = gpz.compress_f64(torch.from_numpy(x).cuda(), 1e32)
    rs, rp, rused = oracle.compress_f64(x, 1e32)
    assert np.array_equal(np.array(used), rused) and np.array_equal(s.cpu().numpy(), rs)
    y = x.copy()
    y[2, 7] = 3.4028235677973366e38  # rounds to +inf in fp32: the fp32 form cannot hold it
    assert oracle.compress_f64_status(y, 1e32) == oracle.ERR_UNSUPPORTED
    s, p, used = gpz.compress_f64(torch.from_numpy(y).cuda(), 1e32, want_perm=True)
    rs, rp, rused = oracle.compress_wide(y, 1e32)  # the 64-bit form instead
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(p.cpu().numpy().astype(np.uint32), rp)
    assert np.array_equal(np.array(used), rused)
    out = gpz.decompress_f64(s, 3, x.shape[1]).cpu().numpy()
    assert np.array_equal(out.view(np.uint64), oracle.decompress_wide(rs, 3, x.shape[1]).view(np.uint64))


@pytest.mark.parametrize("mode", [0, 1])
def test_f64_falls_back_to_64_bit_intermediates(gpz, oracle, mode):
    """A bound finer than fp32 can hold: the fp32 form refuses, and
    gpz_compress_f64 writes the 64-bit form's stream (version 2) with the
    full bounds; gpz_decompress_f64 reads it back through the version word."""
    x = np.full((2, 2048), 12345.678901234)
    x[0, 1::2] = 1.0
    x[1] = np.linspace(-3.0, 7.0, 2048)
    eb = 1e-9 if mode == 0 else 1e-13
    assert oracle.compress_f64_status(x, eb, mode) == oracle.ERR_UNSUPPORTED
    s, p, used = gpz.compress_f64(torch.from_numpy(x).cuda(), eb, mode, want_perm=True)
    rs, rp, rused = oracle.compress_wide(x, eb, mode)
    assert s.cpu().numpy().view(np.uint32)[1] == 2
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(p.cpu().numpy().astype(np.uint32), rp)
    assert np.array_equal(np.array(used), rused)
    out = gpz.decompress_f64(s, 2, 2048).cpu().numpy()
    ref = oracle.decompress_wide(rs, 2, 2048)
    assert np.array_equal(out.view(np.uint64), ref.view(np.uint64))
    assert np.all(np.abs(x[:, rp] - out) <= np.array(used)[:, None])


def test_f64_full_snapshot(gpz, oracle):
    """The 2^26 x 6 cosmology snapshot in fp64 (relative bound 1e-4): the
    stream is the fp32 path's stream for the rounded values and reduced
    bounds, and sampled decoded values are within eb of the fp64 input."""
    from paper_2508_10305_gb300 import synth
    x32 = synth.cosmology(1 << 26, seed=2, device="cuda")
    F, n = x32.shape
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    x = x32.double() + (torch.rand(x32.shape, generator=g, device="cuda", dtype=torch.float64) - 0.5) * 1e-5
    stream, perm, used = gpz.compress_f64(x, 1e-4, gpz.EB_REL, 3, want_perm=True)
    r = x.float()
    ref, _ = gpz.compress(r, used, gpz.EB_ABS, 3)
    assert torch.equal(stream, ref)
    out = gpz.decompress_f64(stream, F, n)
    idx = torch.randint(0, n, (1 << 20,), device="cuda", generator=g)
    xs = x[:, perm.long()[idx]]
    delta = (x - r.double()).abs().amax(dim=1)
    err = (xs - out[:, idx]).abs()
    bound = (torch.tensor(used, device="cuda", dtype=torch.float64) + delta) * (1 + 1e-12)
    assert torch.all(err <= bound[:, None])
