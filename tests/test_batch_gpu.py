"""The batched entry points (include/gpz_batch.h) on the GPU, through the C
ABI: every chunk of a batch must give exactly the stream the CPU oracle
writes for it alone (and the single-array GPU call writes), every decompressed
chunk exactly the oracle's values, whatever the launch shape, with the
CUDA graph or without, and a failing chunk must not disturb the others."""
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


def make_chunks(seed, count, sizes=None):
    """Mixed chunks: every field count, segment width and bound mode, the
    edge sizes (0, 1, one block, one block + 1), NaN and constant chunks."""
    rng = np.random.default_rng(seed)
    edge = [0, 1, 5, 1023, 1024, 1025, 2048, 3000, 4097, 9000, 20000]
    out = []
    for c in range(count):
        n = int(sizes[c]) if sizes is not None else int(edge[c] if c < len(edge) else rng.integers(1, 40000))
        F = int(rng.choice([1, 2, 3, 4, 5, 6, 7, 8]))
        G = int(rng.integers(0, 4))
        mode = int(rng.integers(0, 2))
        kind = str(rng.choice(["uniform", "clustered", "lidar", "mixed"]))
        eb = [float(rng.choice([1e-1, 1e-2, 1e-3, 1e-4])) for _ in range(F)]
        x = gen(kind, F, n, rng) if n else np.zeros((F, 0), np.float32)
        if c == count - 2 and n > 10:
            x[0, n // 2] = np.nan  # a block stored raw
        if c == count - 3 and n > 0:
            x[:] = 7.25            # constant fields
        out.append(dict(x=x, F=F, G=G, mode=mode, eb=eb, n=n))
    return out


def device_fields(x, offset=0):
    F, n = x.shape
    buf = torch.zeros((F, n + 8), dtype=torch.float32, device="cuda")
    if n:
        buf[:, offset:offset + n] = torch.from_numpy(x).cuda()
    return buf, [buf[f, offset:offset + n] for f in range(F)]


def compress_batch(gpz, chunks, use_graph, cfg=None, want_perm=True, offsets=None):
    items, keep = [], []
    for k, ch in enumerate(chunks):
        buf, fields = device_fields(ch["x"], offsets[k] if offsets else 0)
        perm = torch.zeros(max(ch["n"], 1), dtype=torch.int32, device="cuda") if want_perm else None
        keep.append((buf, perm))
        items.append((fields, gpz.make_params(ch["F"], ch["eb"], ch["mode"], ch["G"]), perm))
    bc = gpz.BatchCompressor(items, use_graph=use_graph)
    if cfg is not None:
        assert gpz.gpz_batch_set_config(bc.plan, cfg) == gpz.OK
    bc()
    st, per = bc.status()
    assert st == gpz.OK and per == [0] * len(chunks)
    streams = [s.cpu().numpy() for s in bc.streams()]
    perms = [p[:ch["n"]].cpu().numpy().astype(np.uint32) if p is not None else None
             for (_, p), ch in zip(keep, chunks)]
    return bc, streams, perms, keep


def assert_oracle(oracle, chunks, streams, perms):
    for c, (ch, s) in enumerate(zip(chunks, streams)):
        rs, rp = oracle.compress(ch["x"], ch["eb"], ch["mode"], ch["G"])
        assert s.size == rs.size and np.array_equal(s, rs), "chunk %d: stream differs from the oracle's" % c
        if perms[c] is not None:
            assert np.array_equal(perms[c], rp), "chunk %d: permutation differs" % c


def test_batch_compress_matches_oracle(gpz, oracle):
    chunks = make_chunks(11, 40)
    bc, streams, perms, _ = compress_batch(gpz, chunks, use_graph=False)
    assert_oracle(oracle, chunks, streams, perms)
    bc.close()


def test_batch_matches_single_call(gpz):
    """The batch and one gpz_compress call per chunk write the same bytes."""
    chunks = make_chunks(12, 24)
    bc, streams, _, keep = compress_batch(gpz, chunks, use_graph=True, want_perm=False)
    for c, ch in enumerate(chunks):
        _, fields = device_fields(ch["x"])
        comp = gpz.Compressor(ch["n"], ch["F"], ch["eb"], ch["mode"], ch["G"])
        size = comp(fields)
        assert np.array_equal(comp.out[:size].cpu().numpy(), streams[c]), "chunk %d" % c
    bc.close()


def test_batch_unaligned_fields(gpz, oracle):
    chunks = make_chunks(13, 12)
    offs = [k % 4 for k in range(12)]
    bc, streams, perms, _ = compress_batch(gpz, chunks, use_graph=False, offsets=offs)
    assert_oracle(oracle, chunks, streams, perms)
    bc.close()


@pytest.mark.parametrize("slice_,compact,general,form", [(1024, 1, 1, 1), (4096, 4, 4, 2), (1 << 20, 32, 2, 0),
                                                         (65536, 16, 2, 2)])
def test_batch_launch_shapes_and_graph(gpz, oracle, slice_, compact, general, form):
    """Any launch shape -- either per-block compression body included -- (and
    the graph replays of it) gives the same bytes; small slices split every
    relative-bound field into many range items."""
    chunks = make_chunks(14, 20)
    cfg = gpz.gpz_batch_config(slice_, compact, general, form)
    bc, streams, perms, _ = compress_batch(gpz, chunks, use_graph=True, cfg=cfg)
    assert_oracle(oracle, chunks, streams, perms)
    for _ in range(2):  # replays of the captured graph
        bc.sizes.zero_()
        bc()
        assert bc.status()[0] == gpz.OK
        again = [s.cpu().numpy() for s in bc.streams()]
        assert all(np.array_equal(a, b) for a, b in zip(again, streams))
    bc.close()


def test_batch_decompress_matches_oracle(gpz, oracle):
    chunks = make_chunks(15, 40)
    bc, streams, _, _ = compress_batch(gpz, chunks, use_graph=False, want_perm=False)
    dev = [torch.from_numpy(s).cuda() if s.size else torch.zeros(64, dtype=torch.uint8, device="cuda")
           for s in streams]
    items = [(d, s.size, ch["F"], ch["n"]) for d, s, ch in zip(dev, streams, chunks)]
    for use_graph in (False, True):
        bd = gpz.BatchDecompressor(items, use_graph=use_graph)
        bd()
        st, per = bd.status()
        assert st == gpz.OK and per == [0] * len(chunks)
        for c, ch in enumerate(chunks):
            ref = oracle.decompress(streams[c], ch["F"], ch["n"])
            got = bd.outs[c][:, :ch["n"]].cpu().numpy()
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), "chunk %d" % c
        bd.close()
    bc.close()


def test_batch_decompress_isolates_a_bad_chunk(gpz, oracle):
    """A chunk whose descriptor disagrees with its stream header (wrong n) is
    reported GPZ_ERR_CORRUPT in its own status; the others decode exactly."""
    chunks = make_chunks(16, 8, sizes=[5000, 3000, 7000, 1025, 2048, 9000, 100, 4096])
    bc, streams, _, _ = compress_batch(gpz, chunks, use_graph=False, want_perm=False)
    dev = [torch.from_numpy(s).cuda() for s in streams]
    items = [(d, s.size, ch["F"], ch["n"]) for d, s, ch in zip(dev, streams, chunks)]
    bad = 2
    items[bad] = (dev[bad], streams[bad].size, chunks[bad]["F"], chunks[bad]["n"] - 1)
    bd = gpz.BatchDecompressor(items, use_graph=False)
    bd()
    st, per = bd.status()
    assert st == gpz.ERR_CORRUPT
    assert per == [gpz.ERR_CORRUPT if c == bad else 0 for c in range(len(chunks))]
    for c, ch in enumerate(chunks):
        if c == bad:
            continue
        ref = oracle.decompress(streams[c], ch["F"], ch["n"])
        assert np.array_equal(bd.outs[c][:, :ch["n"]].cpu().numpy().view(np.uint32), ref.view(np.uint32))
    bd.close()
    bc.close()


def test_batch_tune_keeps_the_bytes(gpz, oracle):
    chunks = make_chunks(17, 16)
    bc, streams, perms, _ = compress_batch(gpz, chunks, use_graph=False)
    cfg, ms = bc.tune(reps=1)
    assert ms > 0 and cfg.range_slice % 1024 == 0 and 1 <= cfg.compact_ctas <= 32
    bc.sizes.zero_()
    bc()
    assert bc.status()[0] == gpz.OK
    assert all(np.array_equal(a.cpu().numpy(), b) for a, b in zip(bc.streams(), streams))
    bc.close()


def test_batched_workload_sampled(gpz, oracle):
    """512 chunks of the batched workload's kind (log-uniform sizes, 3 or 6
    fields, relative bounds 1e-3 / 1e-4; sizes scaled down 10x): every chunk
    equals its single-call stream on the GPU; sampled small chunks equal the
    oracle's; the decompressed values are within each field's bound."""
    from paper_2508_10305_gb300 import synth
    wl = synth.batched_workload(n_chunks=512, lo=1_000, hi=400_000, seed=4, device="cuda")
    items = [(wl.fields(c), gpz.make_params(wl.F[c], [wl.rel[c]] * wl.F[c], gpz.EB_REL, 3))
             for c in range(wl.count)]
    bc = gpz.BatchCompressor(items, use_graph=True)
    bc()
    assert bc.status()[0] == gpz.OK
    streams = bc.streams()
    rng = np.random.default_rng(0)
    small = [c for c in range(wl.count) if wl.n[c] <= 20000]
    for c in rng.choice(small, size=min(6, len(small)), replace=False):
        x = torch.stack(wl.fields(c)).cpu().numpy()
        rs, _ = oracle.compress(x, [wl.rel[c]] * wl.F[c], 1, 3)
        assert np.array_equal(streams[c].cpu().numpy(), rs), "chunk %d" % c
    for c in range(wl.count):
        comp = gpz.Compressor(wl.n[c], wl.F[c], [wl.rel[c]] * wl.F[c], gpz.EB_REL, 3)
        size = comp(wl.fields(c))
        assert torch.equal(comp.out[:size], streams[c]), "chunk %d" % c
    items = [(streams[c], streams[c].numel(), wl.F[c], wl.n[c]) for c in range(wl.count)]
    bd = gpz.BatchDecompressor(items, use_graph=True)
    bd()
    assert bd.status()[0] == gpz.OK
    for c in range(0, wl.count, 7):
        x = torch.stack(wl.fields(c))
        for f in range(wl.F[c]):
            eb = float(np.frombuffer(streams[c][64 + 8 * f:68 + 8 * f].cpu().numpy().tobytes(), np.float32)[0])
            # values come back permuted within each block; if every value is
            # within eb of its original, so is the k-th smallest of the block
            got = bd.outs[c][f, :wl.n[c]]
            nb = (wl.n[c] + 1023) // 1024
            for b in (0, nb - 1):
                lo, hi = b * 1024, min(wl.n[c], (b + 1) * 1024)
                gs = torch.sort(got[lo:hi]).values
                xs = torch.sort(x[f, lo:hi]).values
                assert float((gs - xs).abs().max()) <= eb * 1.0000001
    bd.close()
    bc.close()
