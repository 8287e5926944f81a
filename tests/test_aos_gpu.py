"""Interleaved (array-of-structures) input and output through the C ABI
(gpz_compress_aos / gpz_decompress_aos) against the oracle on the same values
in structure-of-arrays form: the stream and permutation bit for bit, and the
decompressed records equal to the oracle's values interleaved."""
import numpy as np
import pytest
import torch

from tests.test_parity_gpu import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


@pytest.mark.parametrize("F,n,mode,kind,offset", [
    (3, 300_000, 0, "lidar", 0),     # LAS-style x, y, z records
    (3, 4097, 1, "clustered", 1),    # ragged last tile, 4-byte aligned base
    (1, 1, 0, "uniform", 0),
    (6, 100_000, 1, "clustered", 0),
    (8, 5000, 0, "mixed", 3),
    (2, 1023, 0, "uniform", 2),
    (8, 3_000_000, 1, "mixed", 0),   # relative bound: more tiles than CTAs in the fused range pass
    (5, 70_001, 1, "uniform", 0),    # ragged last tile, aligned base
])
def test_aos_matches_oracle(gpz, oracle, F, n, mode, kind, offset):
    rng = np.random.default_rng(F * 1000 + n % 997)
    x = gen(kind, F, n, rng)
    eb = 1e-3 if mode == 0 else 1e-4
    buf = torch.zeros(offset + n * F + 4, dtype=torch.float32, device="cuda")
    buf[offset:offset + n * F] = torch.from_numpy(np.ascontiguousarray(x.T).reshape(-1)).cuda()
    stream, perm = gpz.compress_aos(buf[offset:offset + n * F], F, eb, mode, 3, want_perm=True)
    rs, rp = oracle.compress(x, eb, mode, 3)
    assert stream.numel() == rs.size and np.array_equal(stream.cpu().numpy(), rs)
    assert np.array_equal(perm.cpu().numpy().astype(np.uint32), rp)
    out = gpz.decompress_aos(stream, F, n)
    ro = oracle.decompress(rs, F, n)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), np.ascontiguousarray(ro.T).view(np.uint32))


@pytest.mark.parametrize("own_ws", [False, True])
def test_aos_relative_bound_with_non_finite_values(gpz, oracle, own_ws):
    """The transpose that also does the range pass: blocks with NaN or an
    infinity go raw, the range of a field is taken over its non-NaN values
    (an infinity makes it infinite, so eb = rel), and a field holding only
    NaN keeps eb = rel -- the stream is the oracle's either way."""
    import ctypes as C
    rng = np.random.default_rng(17)
    F, n = 4, 9000
    x = gen("clustered", F, n, rng)
    x[0, 5] = np.nan
    x[1, 4000] = np.inf
    x[2, :] = np.nan
    x[3, 8999] = -np.inf
    xa = torch.from_numpy(np.ascontiguousarray(x.T).reshape(-1)).cuda()
    params = gpz.make_params(F, 1e-3, gpz.EB_REL)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    h = C.c_uint64(0)
    need = gpz.gpz_compress_aos_workspace_size(n, F)
    ws = None if own_ws else torch.empty(need, dtype=torch.uint8, device="cuda")
    st = gpz.lib.gpz_compress_aos(xa.data_ptr(), n, C.byref(params), out.data_ptr(), cap, None, C.byref(h), None,
                                  ws.data_ptr() if ws is not None else None, need if ws is not None else 0, None)
    assert st == gpz.OK
    rs, _ = oracle.compress(x, 1e-3, 1, 3)
    assert h.value == rs.size and np.array_equal(out[:h.value].cpu().numpy(), rs)


def test_aos_workspace_checks(gpz):
    n, F = 10_000, 3
    x = torch.zeros(n * F, dtype=torch.float32, device="cuda")
    params = gpz.make_params(F, 1e-2)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    need = gpz.gpz_compress_aos_workspace_size(n, F)
    assert need >= gpz.gpz_compress_workspace_size(n, F) + 4 * n * F
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    import ctypes as C
    st = gpz.lib.gpz_compress_aos(x.data_ptr(), n, C.byref(params), out.data_ptr(), cap, None, None, None,
                                  ws.data_ptr(), need - 1, None)
    assert st == gpz.ERR_CAPACITY
    st = gpz.lib.gpz_compress_aos(x.data_ptr() + 2, n, C.byref(params), out.data_ptr(), cap, None, None, None,
                                  ws.data_ptr(), need, None)
    assert st == gpz.ERR_INVALID_ARG  # records must be 4-byte aligned
    assert gpz.gpz_decompress_aos_workspace_size(n, 9) == 0


def test_aos_without_workspace(gpz, oracle):
    """d_ws = NULL: the library allocates, synchronises and returns the status."""
    import ctypes as C
    rng = np.random.default_rng(5)
    F, n = 3, 20_000
    x = gen("clustered", F, n, rng)
    xa = torch.from_numpy(np.ascontiguousarray(x.T).reshape(-1)).cuda()
    params = gpz.make_params(F, 1e-3)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    h = C.c_uint64(0)
    st = gpz.lib.gpz_compress_aos(xa.data_ptr(), n, C.byref(params), out.data_ptr(), cap, None, C.byref(h), None,
                                  None, 0, None)
    assert st == gpz.OK
    rs, _ = oracle.compress(x, 1e-3, 0, 3)
    assert h.value == rs.size and np.array_equal(out[:h.value].cpu().numpy(), rs)
    rec = torch.empty(n * F, dtype=torch.float32, device="cuda")
    st = gpz.lib.gpz_decompress_aos(out.data_ptr(), h.value, rec.data_ptr(), F, n, None, 0, None)
    assert st == gpz.OK
    ro = oracle.decompress(rs, F, n)
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), np.ascontiguousarray(ro.T).reshape(-1).view(np.uint32))
    # a damaged stream: the status comes back from the call itself
    bad = out[:h.value].clone()
    bad[0] ^= 1
    st = gpz.lib.gpz_decompress_aos(bad.data_ptr(), h.value, rec.data_ptr(), F, n, None, 0, None)
    assert st == gpz.ERR_CORRUPT


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_aos_forms_and_general_path(gpz, oracle, offset, flags, mode):
    """Both routes of gpz_compress_aos give the oracle's stream: 16-byte
    aligned records read by the tile kernel itself, and (4-byte aligned
    records, or fused compaction) records transposed first.  The array mixes
    blocks of every path: encoded, raw (NaN) and general (codes of 2^23 or
    more, from one block spanning a much wider range)."""
    import ctypes as C
    rng = np.random.default_rng(31 + offset + 2 * flags + 4 * mode)
    F, n = 4, 6 * 1024 + 77
    x = gen("clustered", F, n, rng)
    x[:, 1024:2048] = (rng.random((F, 1024)) * 4e4).astype(np.float32)  # wide block
    x[2, 3000] = np.nan                                                # raw block
    eb = 1e-3 if mode == 0 else 1e-7
    buf = torch.zeros(offset + n * F + 4, dtype=torch.float32, device="cuda")
    buf[offset:offset + n * F] = torch.from_numpy(np.ascontiguousarray(x.T).reshape(-1)).cuda()
    xa = buf[offset:offset + n * F]
    params = gpz.make_params(F, eb, mode, 3, flags)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    h = C.c_uint64(0)
    need = gpz.gpz_compress_aos_workspace_size(n, F)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = gpz.lib.gpz_compress_aos(xa.data_ptr(), n, C.byref(params), out.data_ptr(), cap, None, C.byref(h),
                                  perm.data_ptr(), ws.data_ptr(), need, None)
    assert st == gpz.OK
    rs, rp = oracle.compress(x, eb, mode, 3)
    assert h.value == rs.size and np.array_equal(out[:h.value].cpu().numpy(), rs)
    assert np.array_equal(perm.cpu().numpy().astype(np.uint32), rp)
    w = rs.view(np.uint32)
    nb = (n + 1023) // 1024
    table = w[16 + 2 * F:16 + 2 * F + nb + 1]
    modes = [int(w[16 + 2 * F + nb + 1 + table[b]]) for b in range(nb)]
    assert any(m & 1 for m in modes)  # a raw block is among them
    rec = torch.empty(n * F + 1, dtype=torch.float32, device="cuda")[offset:offset + n * F]
    dws = gpz.gpz_decompress_aos_workspace_size(n, F)
    dw = torch.zeros(dws, dtype=torch.uint8, device="cuda")
    assert gpz.lib.gpz_decompress_aos(out.data_ptr(), h.value, rec.data_ptr(), F, n, dw.data_ptr(), dws, None) == gpz.OK
    assert gpz.gpz_sync_status(dw) == gpz.OK
    ro = oracle.decompress(rs, F, n)
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), np.ascontiguousarray(ro.T).reshape(-1).view(np.uint32))


def test_aos_records_wider_than_128_bits(gpz, oracle):
    """Eight fields of 19-bit codes: records of 143 bits, decoded field by
    field from the stream, written straight into the records."""
    rng = np.random.default_rng(77)
    F, n = 8, 3 * 1024 + 5
    x = (rng.random((F, n)) * 1000).astype(np.float32)
    xa = torch.from_numpy(np.ascontiguousarray(x.T).reshape(-1)).cuda()
    stream, _ = gpz.compress_aos(xa, F, 1e-3, 0, 3, want_perm=True)
    rs, _ = oracle.compress(x, 1e-3, 0, 3)
    assert np.array_equal(stream.cpu().numpy(), rs)
    w = rs.view(np.uint32)
    widths = [(int(w[16 + 2 * F + 4 + 1 + 1 + F + k // 4]) >> (8 * (k % 4))) & 0xff for k in range(F)]
    assert sum(widths) - 9 > 128
    out = gpz.decompress_aos(stream, F, n)
    ro = oracle.decompress(rs, F, n)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), np.ascontiguousarray(ro.T).view(np.uint32))
