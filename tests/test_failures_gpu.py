"""Failure detection without a GPU fault: the bounded device-side waits run
out and report, and an exhausted device shows up as GPZ_ERR_OOM.

The waits are the look-backs of the compaction's prefix sum (Section 4.4,
step 2) and of fused compaction.  The hooks of include/gpz_test.h launch the
product kernels with a predecessor that never publishes and a limit of a few
thousand SM cycles; the kernels must give up, record their status and
return, after which the GPU must still run an ordinary round trip."""
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


def _round_trip_still_works(gpz, oracle):
    from paper_2508_10305_gb300 import synth
    x = synth.uniform_box(3000, seed=5)
    stream, perm = gpz.compress(torch.from_numpy(x).cuda(), 1e-2, gpz.EB_ABS, 3, want_perm=True)
    ref, ref_perm = oracle.compress(x, 1e-2, 0, 3)
    assert np.array_equal(stream.cpu().numpy(), ref)
    assert np.array_equal(perm.cpu().numpy().astype(np.uint32), ref_perm)


@pytest.mark.parametrize("batched", [0, 1])
def test_scan_wait_runs_out(gpz, oracle, batched):
    ws = torch.zeros(gpz.lib.gpz_test_scan_workspace_size(), dtype=torch.uint8, device="cuda")
    st = gpz.gpz_test_scan_timeout(batched, 20_000, ws)
    assert st == gpz.ERR_TIMEOUT, gpz.gpz_status_str(st)
    # both CTAs finished: tiles 1 and 2 published their (partial) prefixes
    states = ws[256:256 + 24].view(torch.int64).cpu().numpy().view(np.uint64)
    shift = 62 if batched else 32  # the flag above a 62-bit (batched) or 32-bit value; 2 = prefix
    assert states[0] == 0
    assert all(int(v) >> shift == 2 for v in states[1:]), states
    torch.cuda.synchronize()
    _round_trip_still_works(gpz, oracle)


def test_block_lookback_gives_up(gpz, oracle):
    ws = torch.zeros(8 * 64, dtype=torch.uint8, device="cuda")
    st, placed = gpz.gpz_test_block_lookback_timeout(40, 20_000, ws)
    assert st == gpz.OK and placed == 0
    _round_trip_still_works(gpz, oracle)


def test_injected_allocation_failures(gpz, oracle):
    from paper_2508_10305_gb300 import synth
    x = torch.from_numpy(synth.uniform_box(5000, seed=6)).cuda()
    F, n = x.shape
    params = gpz.make_params(F, 1e-2)
    cap = gpz.gpz_bound_size(n, F)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    gpz.gpz_test_fail_next_allocations(1)
    try:
        st = gpz.gpz_compress(x, n, params, out, cap)  # no workspace: the library allocates
        assert st == gpz.ERR_OOM
        assert gpz.gpz_test_fail_next_allocations(0) == 0  # the one failure was used
        size = C.c_uint64(0)
        assert gpz.gpz_compress(x, n, params, out, cap, h_out_size=size) == gpz.OK
        dec = torch.empty((F, n), dtype=torch.float32, device="cuda")
        gpz.gpz_test_fail_next_allocations(1)
        assert gpz.gpz_decompress(out, size.value, dec, F, n) == gpz.ERR_OOM
        assert gpz.gpz_decompress(out, size.value, dec, F, n) == gpz.OK
        ref, _ = oracle.compress(x.cpu().numpy(), 1e-2, 0, 3)
        assert np.array_equal(out[:size.value].cpu().numpy(), ref)
        # a batch plan and the serving engine's arena
        gpz.gpz_test_fail_next_allocations(1)
        ch = gpz.gpz_compress_chunk()
        for f in range(F):
            ch.fields[f] = x[f].data_ptr()
        ch.n, ch.params, ch.out, ch.out_capacity = n, params, out.data_ptr(), cap
        st, plan = gpz.gpz_batch_create_compress([ch])
        assert st == gpz.ERR_OOM
        st, plan = gpz.gpz_batch_create_compress([ch])
        assert st == gpz.OK
        gpz.gpz_batch_destroy(plan)
        gpz.gpz_test_fail_next_allocations(1)
        cfg = gpz.gpz_server_config()
        cfg.budget_bytes, cfg.lanes, cfg.max_batch, cfg.max_batch_bytes, cfg.lane_bytes = 64 << 20, 1, 4, 0, 0
        used = gpz.gpz_server_config()
        h = C.c_void_p()
        st = gpz.lib.gpz_server_create(C.byref(cfg), C.byref(used), C.byref(h))
        assert st == gpz.ERR_OOM and not h.value
    finally:
        gpz.gpz_test_fail_next_allocations(0)
    _round_trip_still_works(gpz, oracle)
