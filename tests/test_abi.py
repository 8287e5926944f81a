"""The C ABI library loads and exports every entry point include/gpz.h
declares; host-side entry points behave without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpz.h")


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpz_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gpz_bound_size", "gpz_compress", "gpz_decompress", "gpz_compress_workspace_size",
                     "gpz_decompress_workspace_size", "gpz_sync_status", "gpz_inspect", "gpz_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(gpz):
    lib = C.CDLL(gpz.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_bound_and_workspace_sizes(gpz):
    assert gpz.gpz_bound_size(0, 3) == 4 * (16 + 6 + 1)
    n, F = 1_000_000, 3
    nb = (n + 1023) // 1024
    assert gpz.gpz_bound_size(n, F) == 4 * (16 + 2 * F + (nb + 1) + nb + F * n)
    assert gpz.gpz_bound_size(10, 0) == 0 and gpz.gpz_bound_size(10, 9) == 0
    assert gpz.gpz_compress_workspace_size(n, F) >= 4 * F * n
    assert gpz.gpz_decompress_workspace_size() >= 4


def test_bound_matches_oracle(gpz, oracle):
    for n in (0, 1, 1023, 1024, 1025, 10**6):
        for F in (1, 3, 6, 8):
            assert gpz.gpz_bound_size(n, F) == oracle.bound_size(n, F)


def test_status_strings(gpz):
    assert gpz.gpz_status_str(gpz.OK) == "ok"
    assert gpz.gpz_status_str(gpz.ERR_CORRUPT) == "corrupt stream"
    assert gpz.gpz_status_str(99) == "unknown status"


def test_inspect_host_header(gpz, oracle):
    x = (np.random.default_rng(1).random((4, 3000)) * 9).astype(np.float32)
    stream, _ = oracle.compress(x, 1e-3, 1, 2)
    info = gpz.gpz_inspect(stream[:64].tobytes())
    assert info == dict(n=3000, n_fields=4, seg_bits=2, mode=1)
    bad = bytearray(stream[:64].tobytes())
    bad[0] ^= 1
    with pytest.raises(gpz.GpzError):
        gpz.gpz_inspect(bytes(bad))


def test_argument_errors_need_no_device(gpz):
    """Invalid arguments are rejected before anything is enqueued."""
    L = gpz.lib
    p = gpz.make_params(3, 1e-3)
    fields = (C.c_void_p * 3)(16, 32, 48)
    dummy = C.c_void_p(4096)
    assert L.gpz_compress(fields, 10, None, dummy, 1 << 20, None, None, None, None, 0, None) == gpz.ERR_INVALID_ARG
    bad = gpz.make_params(3, 1e-3)
    bad.eb[1] = 0.0
    assert L.gpz_compress(fields, 10, C.byref(bad), dummy, 1 << 20, None, None, None, None, 0, None) == gpz.ERR_INVALID_ARG
    bad = gpz.make_params(3, 1e-3, seg_bits=4)
    assert L.gpz_compress(fields, 10, C.byref(bad), dummy, 1 << 20, None, None, None, None, 0, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_compress(fields, 10, C.byref(p), dummy, 8, None, None, None, None, 0, None) == gpz.ERR_CAPACITY
    assert L.gpz_compress(fields, 10, C.byref(p), C.c_void_p(4098), 1 << 20, None, None, None, None, 0, None) == gpz.ERR_INVALID_ARG
    big = gpz.make_params(8, 1e-3)
    fields8 = (C.c_void_p * 8)(*([16] * 8))
    assert L.gpz_compress(fields8, 1 << 29, C.byref(big), dummy, 1 << 62, None, None, None, None, 0, None) == gpz.ERR_UNSUPPORTED
    outs = (C.c_void_p * 3)(16, 32, 48)
    assert L.gpz_decompress(dummy, 8, outs, 3, 10, None, 0, None) == gpz.ERR_CORRUPT
    assert L.gpz_decompress(dummy, 1024, outs, 0, 10, None, 0, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_decompress(None, 1024, outs, 3, 10, None, 0, None) == gpz.ERR_INVALID_ARG
