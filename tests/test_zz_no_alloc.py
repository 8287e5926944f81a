"""gpz_compress_noalloc, the compression entry point that allocates no device
memory, for callers that cannot allocate when they compress: an in-situ
hook inside a simulation whose own pool allocator holds all device memory,
or a loop that cannot afford an allocation's stall.  It is checked through
the C ABI against the ordinary gpz_compress on the same inputs, on several
calls in a row: the streams and permutations must be identical, byte for
byte, whether the size is returned to the host (the call synchronises) or
only written on the device; and once its scratch array has been taken,
further calls must not lower the device's free memory.  This file is
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


def _cases(gpz):
    from paper_2508_10305_gb300 import synth
    return [
        (torch.from_numpy(synth.uniform_box(200_000 + 77, seed=11)).cuda(), 1e-2, gpz.EB_ABS, 3),
        (synth.cosmology(1 << 20, seed=12, device="cuda"), 1e-4, gpz.EB_REL, 3),
    ]


def _reference(gpz, x, eb, mode, G):
    F, n = x.shape
    c = gpz.Compressor(n, F, eb, mode, G, want_perm=True)
    size = c([x[f] for f in range(F)])
    return c.out[:size].cpu().numpy(), c.perm[:n].cpu().numpy()


def _buffers(gpz, x):
    F, n = x.shape
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    d_size = torch.zeros(1, dtype=torch.int64, device="cuda")
    return cap, out, perm, d_size


def test_noalloc_matches_gpz_compress_twice(gpz):
    for x, eb, mode, G in _cases(gpz):  # two calls in a row, different sizes and field counts
        F, n = x.shape
        ref_stream, ref_perm = _reference(gpz, x, eb, mode, G)
        cap, out, perm, _ = _buffers(gpz, x)
        size = C.c_uint64(0)
        st = gpz.gpz_compress_noalloc(x, n, gpz.make_params(F, eb, mode, G), out, cap, None, size, perm)
        assert st == gpz.OK, gpz.gpz_status_str(st)
        assert size.value == ref_stream.size and np.array_equal(out[:size.value].cpu().numpy(), ref_stream)
        assert np.array_equal(perm.cpu().numpy(), ref_perm)


def test_noalloc_device_size_only(gpz):
    """Without h_out_size the call enqueues and returns; the size is written
    on the device and the status is read with gpz_noalloc_sync_status."""
    for x, eb, mode, G in _cases(gpz):
        F, n = x.shape
        ref_stream, ref_perm = _reference(gpz, x, eb, mode, G)
        cap, out, perm, d_size = _buffers(gpz, x)
        st = gpz.gpz_compress_noalloc(x, n, gpz.make_params(F, eb, mode, G), out, cap, d_size, None, perm)
        assert st == gpz.OK
        assert gpz.gpz_noalloc_sync_status() == gpz.OK
        size = int(d_size.item())
        assert size == ref_stream.size and np.array_equal(out[:size].cpu().numpy(), ref_stream)
        assert np.array_equal(perm.cpu().numpy(), ref_perm)


def test_noalloc_takes_no_device_memory(gpz):
    """After gpz_noalloc_prepare (which takes the scratch array) and one
    warm-up call, calls of different sizes leave the free device memory
    where it was."""
    assert gpz.gpz_noalloc_prepare() == gpz.OK
    cases = _cases(gpz)
    bufs = [_buffers(gpz, x) for x, _, _, _ in cases]
    params = [gpz.make_params(x.shape[0], eb, mode, G) for x, eb, mode, G in cases]
    x0 = cases[0][0]
    assert gpz.gpz_compress_noalloc(x0, x0.shape[1], params[0], bufs[0][1], bufs[0][0], bufs[0][3]) == gpz.OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for (x, _, _, _), p, (cap, out, perm, d_size) in zip(cases, params, bufs):
            assert gpz.gpz_compress_noalloc(x, x.shape[1], p, out, cap, d_size, None, perm) == gpz.OK
    assert gpz.gpz_noalloc_sync_status() == gpz.OK
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after >= free_before - (1 << 20), (free_before, free_after)


def test_noalloc_rejects_inputs_beyond_its_scratch(gpz):
    F, n = 6, 4 << 20  # 24M values: more than the 32 MiB scratch array holds
    assert gpz.gpz_compress_workspace_size(n, F) > 32 << 20
    params = gpz.make_params(F, 1e-3)
    dummy = [torch.empty(16, device="cuda") for _ in range(F)]
    out = torch.empty(16, dtype=torch.uint8, device="cuda")
    st = gpz.gpz_compress_noalloc(dummy, n, params, out, gpz.gpz_bound_size(n, F))
    assert st == gpz.ERR_CAPACITY
