"""The library's workspace pool: calls given no workspace allocate it from a
pool that keeps freed memory for the next call (no new pages after the
first), give the same streams as calls given a workspace, and hand the memory
back on gpz_release_pooled_memory."""
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


def test_pool_reuses_and_releases(gpz, oracle):
    from paper_2508_10305_gb300 import synth
    x = torch.from_numpy(synth.uniform_box(300_000, seed=9)).cuda()
    F, n = x.shape
    params = gpz.make_params(F, 1e-2)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    dec = torch.empty((F, n), dtype=torch.float32, device="cuda")
    assert gpz.gpz_release_pooled_memory() == gpz.OK
    assert gpz.gpz_pooled_bytes() == 0
    size = C.c_uint64(0)
    assert gpz.gpz_compress(x, n, params, out, cap, h_out_size=size) == gpz.OK
    held = gpz.gpz_pooled_bytes()
    assert held >= gpz.gpz_compress_workspace_size(n, F)
    ref, _ = oracle.compress(x.cpu().numpy(), 1e-2, 0, 3)
    assert np.array_equal(out[:size.value].cpu().numpy(), ref)
    for _ in range(3):  # the same and smaller workspaces come from what the pool holds
        assert gpz.gpz_compress(x, n, params, out, cap, h_out_size=size) == gpz.OK
        assert gpz.gpz_compress(x[:, :1000].contiguous(), 1000, params, out, cap) == gpz.OK
        assert gpz.gpz_decompress(out, cap, dec, F, 1000) == gpz.OK
        assert gpz.gpz_pooled_bytes() == held
    assert gpz.gpz_compress(x, n, params, out, cap, h_out_size=size) == gpz.OK
    assert np.array_equal(out[:size.value].cpu().numpy(), ref)
    assert gpz.gpz_decompress(out, size.value, dec, F, n) == gpz.OK
    assert np.array_equal(dec.cpu().numpy().view(np.uint32), oracle.decompress(ref, F, n).view(np.uint32))
    assert gpz.gpz_release_pooled_memory() == gpz.OK
    assert gpz.gpz_pooled_bytes() == 0
