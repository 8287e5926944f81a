"""gpz_compress_noalloc, the compression entry point that allocates no device
memory (for callers whose device memory is fully reserved by their own pool
allocator, or that cannot afford an allocation's stall), checked through the
C ABI against the ordinary gpz_compress on the same inputs, twice in a row:
the streams and permutations must be identical, byte for byte.  This file is
collected last on purpose."""
import ctypes as C

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


def _reference(gpz, x, eb, mode, G):
    F, n = x.shape
    c = gpz.Compressor(n, F, eb, mode, G, want_perm=True)
    size = c([x[f] for f in range(F)])
    return c.out[:size].cpu().numpy(), c.perm[:n].cpu().numpy()


def _noalloc(gpz, x, eb, mode, G):
    F, n = x.shape
    params = gpz.make_params(F, eb, mode, G)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    size = C.c_uint64(0)
    st = gpz.gpz_compress_noalloc([x[f] for f in range(F)], n, params, out, cap, None, size, perm)
    assert st == gpz.OK, gpz.gpz_status_str(st)
    return out[:size.value].cpu().numpy(), perm.cpu().numpy()


def test_noalloc_matches_gpz_compress_twice():
    pytest.importorskip("torch")
    from paper_2508_10305_gb300 import build, synth
    build.build()
    from paper_2508_10305_gb300 import gpz
    cases = [
        (torch.from_numpy(synth.uniform_box(200_000 + 77, seed=11)).cuda(), 1e-2, gpz.EB_ABS, 3),
        (synth.cosmology(1 << 20, seed=12, device="cuda"), 1e-4, gpz.EB_REL, 3),
    ]
    for x, eb, mode, G in cases:  # two calls in a row, different sizes and field counts
        ref_stream, ref_perm = _reference(gpz, x, eb, mode, G)
        got_stream, got_perm = _noalloc(gpz, x, eb, mode, G)
        assert got_stream.size == ref_stream.size and np.array_equal(got_stream, ref_stream)
        assert np.array_equal(got_perm, ref_perm)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz
    F, n = 6, 4 << 20  # 24M values: more than the 32 MiB scratch array holds
    assert gpz.gpz_compress_workspace_size(n, F) > 32 << 20
    params = gpz.make_params(F, 1e-3)
    dummy = [torch.empty(16, device="cuda") for _ in range(F)]
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    st = gpz.gpz_compress_noalloc(dummy, n, params, out, gpz.gpz_bound_size(n, F))
    assert st == gpz.ERR_CAPACITY
