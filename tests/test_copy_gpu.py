"""gpz_copy_stream: a copy sized by a word in device memory, between device
memory and pinned host memory, with no host round trip; a compressed stream
moved to the host and back this way decompresses to the same values when
gpz_decompress is given the buffer's capacity as in_size."""
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


@pytest.mark.parametrize("nbytes,cap,off", [(0, 64, 0), (4, 64, 0), (4096, 4096, 0), (4100, 8192, 0),
                                            (1_000_004, 2_000_000, 0), (12, 8, 0), (1_000_004, 2_000_000, 1)])
def test_copy_sized(gpz, nbytes, cap, off):
    rng = np.random.default_rng(nbytes + off)
    src = torch.from_numpy(rng.integers(0, 2**31, size=max(cap // 4, 1) + 4, dtype=np.int64).astype(np.int32)).cuda()
    h = torch.full((cap // 4 + 8,), -1, dtype=torch.int32, pin_memory=True)
    d_size = torch.tensor([nbytes], dtype=torch.int64, device="cuda")
    dst_view, src_view = h[off:], src[off:]  # off = 1: 4-byte aligned only
    assert gpz.gpz_copy_stream(dst_view, src_view, d_size, cap) == gpz.OK
    torch.cuda.synchronize()
    k = min(nbytes, cap) // 4
    got, want = dst_view.numpy(), src_view.cpu().numpy()
    assert np.array_equal(got[:k], want[:k])
    assert np.all(got[k:cap // 4] == -1)  # nothing beyond the size


def test_stream_round_trip_through_host(gpz):
    from paper_2508_10305_gb300 import synth
    x = synth.cosmology(1 << 20, seed=4, device="cuda")
    F, n = x.shape
    c = gpz.Compressor(n, F, 1e-4, gpz.EB_REL, 3)
    c([x[f] for f in range(F)], sync=False)  # the size stays on the device
    h_stream = torch.empty(c.capacity, dtype=torch.uint8, pin_memory=True)
    d_back = torch.empty(c.capacity, dtype=torch.uint8, device="cuda")
    assert gpz.gpz_copy_stream(h_stream, c.out, c.d_size, c.capacity) == gpz.OK
    assert gpz.gpz_copy_stream(d_back, h_stream, c.d_size, c.capacity) == gpz.OK
    d = gpz.Decompressor(n, F)
    out = d(d_back, c.capacity)  # in_size = the capacity: the header bounds the reads
    ref = gpz.Decompressor(n, F)(c.out, int(c.d_size.item()))
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    size = int(c.d_size.item())
    assert torch.equal(h_stream[:size], c.out[:size].cpu())
