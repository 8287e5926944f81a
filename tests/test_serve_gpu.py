"""The serving engine (include/gpz_serve.h) on the GPU: every result of a
mixed stream of compress and decompress requests, run in continuous batches
over several lanes, equals the single call's result for that request alone
(and the CPU oracle's); the plain one-request-per-launch mode gives the same
bytes; admission keeps the arena within its budget; a bad request fails
alone."""
import ctypes as C

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


def make_requests(gpz, seed, count):
    """(kind, payload) pairs: compress requests of random shapes and bounds;
    decompress requests of streams compressed beforehand by the single call."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(count):
        n = int(rng.choice([0, 1, 1000, 1024, 1025, 5000, int(rng.integers(1, 60000))]))
        F = int(rng.choice([1, 3, 4, 6, 8]))
        G = int(rng.integers(0, 4))
        mode = int(rng.integers(0, 2))
        eb = [float(rng.choice([1e-2, 1e-3, 1e-4])) for _ in range(F)]
        x = gen(str(rng.choice(["uniform", "clustered", "lidar", "mixed"])), F, n, rng) if n else np.zeros((F, 0), np.float32)
        xd = torch.from_numpy(x).cuda() if n else torch.zeros((F, 1), device="cuda")[:, :0]
        p = gpz.make_params(F, eb, mode, G)
        comp = gpz.Compressor(n, F, eb, mode, G)
        size = comp([xd[f] for f in range(F)])
        stream = comp.out[:size].clone()
        if rng.random() < 0.5:
            reqs.append(dict(kind=0, x=x, xd=xd, params=p, F=F, n=n, eb=eb, mode=mode, G=G, ref=stream))
        else:
            ref = gpz.Decompressor(n, F)(stream, size).clone()
            reqs.append(dict(kind=1, stream=stream, size=size, F=F, n=n, ref=ref))
    return reqs


def serve(gpz, reqs, **cfg):
    srv = gpz.Server(**cfg)
    ids = {}
    for k, r in enumerate(reqs):
        if r["kind"] == 0:
            ids[srv.submit_compress([r["xd"][f] for f in range(r["F"])], r["params"])] = k
        else:
            ids[srv.submit_decompress(r["stream"], r["size"], r["F"], r["n"])] = k
    got = {}
    while len(got) < len(reqs):
        for res in srv.poll(timeout_ms=2000):
            k = ids[res["id"]]
            r = reqs[k]
            assert res["status"] == gpz.OK, (k, res["status"])
            if r["kind"] == 0:
                got[k] = (res, srv.stream_of(res).clone())
            else:
                got[k] = (res, srv.fields_of(res, r["F"], r["n"]).clone())
            torch.cuda.current_stream().synchronize()  # the copy is done before the memory is reused
            srv.release(res["id"])
    stats = srv.stats()
    srv.close()
    return got, stats


def test_served_results_equal_single_calls(gpz, oracle):
    reqs = make_requests(gpz, 3, 60)
    got, stats = serve(gpz, reqs, budget_bytes=1 << 30, lanes=2, max_batch=16)
    assert stats["completed"] == len(reqs) and stats["batches"] < len(reqs)  # some requests shared a batch
    assert max(res["batch_size"] for res, _ in got.values()) > 1
    for k, r in enumerate(reqs):
        res, out = got[k]
        if r["kind"] == 0:
            assert torch.equal(out, r["ref"]), "request %d: stream differs from the single call" % k
            if k % 5 == 0:
                rs, _ = oracle.compress(r["x"], r["eb"], r["mode"], r["G"])
                assert np.array_equal(out.cpu().numpy(), rs), "request %d: stream differs from the oracle" % k
        else:
            assert torch.equal(out[:, :r["n"]].view(torch.int32), r["ref"][:, :r["n"]].view(torch.int32)), \
                "request %d: values differ from the single call" % k
            assert res["out_bytes"] == 4 * r["n"] * r["F"]


def test_plain_mode_gives_the_same_results(gpz):
    reqs = make_requests(gpz, 4, 24)
    got, stats = serve(gpz, reqs, budget_bytes=1 << 30, lanes=1, max_batch=1)
    assert stats["batches"] == len(reqs)
    for k, r in enumerate(reqs):
        res, out = got[k]
        assert res["batch_size"] == 1
        if r["kind"] == 0:
            assert torch.equal(out, r["ref"])
        else:
            assert torch.equal(out[:, :r["n"]].view(torch.int32), r["ref"][:, :r["n"]].view(torch.int32))


def test_admission_respects_the_budget(gpz):
    """With a budget that holds only a few requests at once, every request
    still completes (admitted as memory comes back) and the arena never
    exceeds the budget; a request larger than the budget is refused."""
    budget = 48 << 20
    rng = np.random.default_rng(5)
    xs = [torch.from_numpy((rng.random((3, 400_000)) * 100).astype(np.float32)).cuda() for _ in range(12)]
    srv = gpz.Server(budget_bytes=budget, lanes=2, max_batch=8)
    p = gpz.make_params(3, 1e-3, gpz.EB_ABS, 3)
    ids = [srv.submit_compress([x[f] for f in range(3)], p) for x in xs]
    done = 0
    peak = 0
    while done < len(ids):
        for res in srv.poll(timeout_ms=2000):
            assert res["status"] == gpz.OK
            done += 1
            peak = max(peak, srv.stats()["arena_in_use"])
            srv.release(res["id"])
    st = srv.stats()
    assert st["arena_peak"] <= budget and st["completed"] == len(ids)
    big = torch.zeros((3, 4_000_000), device="cuda")
    with pytest.raises(gpz.GpzError) as e:
        srv.submit_compress([big[f] for f in range(3)], p)
    assert e.value.status == gpz.ERR_CAPACITY
    srv.close()


def test_a_bad_request_fails_alone(gpz):
    reqs = make_requests(gpz, 6, 12)
    reqs = [r for r in reqs if r["n"] > 2]
    srv = gpz.Server(budget_bytes=1 << 30, lanes=1, max_batch=32)
    ids = {}
    bad = None
    for k, r in enumerate(reqs):
        if r["kind"] == 1 and bad is None:
            bad = k
            ids[srv.submit_decompress(r["stream"], r["size"], r["F"], r["n"] - 1)] = k  # n disagrees with the header
        elif r["kind"] == 1:
            ids[srv.submit_decompress(r["stream"], r["size"], r["F"], r["n"])] = k
        else:
            ids[srv.submit_compress([r["xd"][f] for f in range(r["F"])], r["params"])] = k
    seen = 0
    while seen < len(reqs):
        for res in srv.poll(timeout_ms=2000):
            k = ids[res["id"]]
            assert res["status"] == (gpz.ERR_CORRUPT if k == bad else gpz.OK)
            seen += 1
            srv.release(res["id"])
    srv.close()
