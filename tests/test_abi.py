"""The C ABI library loads and exports every entry point the headers under
include/ declare (gpz.h, gpz_batch.h, gpz_serve.h, gpz_test.h); host-side
entry points behave without touching a GPU."""
import ctypes as C
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
                 if h.endswith(".h"))


@pytest.fixture(scope="module")
def gpz():
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz as g
    return g


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(gpz_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gpz_bound_size", "gpz_compress", "gpz_decompress", "gpz_compress_workspace_size",
                     "gpz_decompress_workspace_size", "gpz_sync_status", "gpz_inspect", "gpz_status_str"):
        assert required in names


def test_header_declares_the_test_hooks():
    names = declared_functions()
    for required in ("gpz_test_fail_next_allocations", "gpz_test_scan_workspace_size", "gpz_test_scan_timeout",
                     "gpz_test_block_lookback_timeout"):
        assert required in names


def test_header_declares_the_batch_boundary():
    names = declared_functions()
    for required in ("gpz_batch_create_compress", "gpz_batch_create_decompress", "gpz_batch_run",
                     "gpz_batch_tune", "gpz_batch_sync_status", "gpz_batch_destroy", "gpz_batch_workspace_size"):
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


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_batch_struct_layout_matches_the_header(gpz, tmp_path):
    """The binding's ctypes structures have the headers' sizes and offsets."""
    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gpz_batch.h"
#include "gpz_serve.h"
int main(void) {
    printf("%zu %zu %zu ", sizeof(gpz_params), offsetof(gpz_params, flags), offsetof(gpz_params, eb));
    printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu ", sizeof(gpz_compress_chunk), offsetof(gpz_compress_chunk, n),
           offsetof(gpz_compress_chunk, params), offsetof(gpz_compress_chunk, out),
           offsetof(gpz_compress_chunk, perm), sizeof(gpz_decompress_chunk),
           offsetof(gpz_decompress_chunk, n_fields), offsetof(gpz_decompress_chunk, n), sizeof(gpz_batch_config));
    printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gpz_server_config), offsetof(gpz_server_config, max_batch_bytes),
           offsetof(gpz_server_config, lane_bytes),
           sizeof(gpz_request_result), offsetof(gpz_request_result, out), offsetof(gpz_request_result, batch),
           sizeof(gpz_server_stats));
    return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    cc, dc = gpz.gpz_compress_chunk, gpz.gpz_decompress_chunk
    sc, rr = gpz.gpz_server_config, gpz.gpz_request_result
    gp = gpz.gpz_params
    want = [C.sizeof(gp), gp.flags.offset, gp.eb.offset, C.sizeof(cc), cc.n.offset, cc.params.offset, cc.out.offset, cc.perm.offset, C.sizeof(dc),
            dc.n_fields.offset, dc.n.offset, C.sizeof(gpz.gpz_batch_config),
            C.sizeof(sc), sc.max_batch_bytes.offset, sc.lane_bytes.offset, C.sizeof(rr), rr.out.offset, rr.batch.offset,
            C.sizeof(gpz.gpz_server_stats)]
    assert got == want


def test_batch_argument_errors_need_no_device(gpz):
    """Descriptor errors are found before any CUDA call; NULL plans are refused."""
    L = gpz.lib

    def chunk(n=1000, F=3, eb=1e-3, cap=None, out=4096, mode=0, G=3):
        d = gpz.gpz_compress_chunk()
        for f in range(F):
            d.fields[f] = 16 * (f + 1)
        d.n, d.params = n, gpz.make_params(F, eb, mode, G)
        d.out = out
        d.out_capacity = gpz.gpz_bound_size(n, F) if cap is None else cap
        return d

    def create(chunks):
        arr = (gpz.gpz_compress_chunk * len(chunks))(*chunks)
        h = C.c_void_p()
        st = L.gpz_batch_create_compress(arr, len(chunks), C.byref(h))
        assert not h.value
        return st

    assert create([chunk(), chunk(eb=0.0)]) == gpz.ERR_INVALID_ARG
    assert create([chunk(), chunk(cap=100)]) == gpz.ERR_CAPACITY
    assert create([chunk(out=4098)]) == gpz.ERR_INVALID_ARG
    assert create([chunk(G=4)]) == gpz.ERR_INVALID_ARG
    bad = chunk()
    bad.params.n_fields = 9
    assert create([bad]) == gpz.ERR_INVALID_ARG
    bad = chunk()
    bad.fields[1] = None
    assert create([bad]) == gpz.ERR_INVALID_ARG
    assert create([chunk(n=1 << 29, F=8, cap=1 << 62)]) == gpz.ERR_UNSUPPORTED
    h = C.c_void_p()
    assert L.gpz_batch_create_compress(None, 1, C.byref(h)) == gpz.ERR_INVALID_ARG
    assert L.gpz_batch_create_compress((gpz.gpz_compress_chunk * 1)(chunk()), 0, C.byref(h)) == gpz.ERR_INVALID_ARG
    assert L.gpz_batch_create_compress((gpz.gpz_compress_chunk * 1)(chunk()), 1, None) == gpz.ERR_INVALID_ARG

    d = gpz.gpz_decompress_chunk()
    d.in_, d.in_size, d.n_fields, d.n = 4096, 8, 3, 10
    for f in range(3):
        d.fields[f] = 16 * (f + 1)
    assert L.gpz_batch_create_decompress((gpz.gpz_decompress_chunk * 1)(d), 1, C.byref(h)) == gpz.ERR_CORRUPT
    d.in_size, d.n_fields = 1024, 0
    assert L.gpz_batch_create_decompress((gpz.gpz_decompress_chunk * 1)(d), 1, C.byref(h)) == gpz.ERR_INVALID_ARG

    assert L.gpz_batch_workspace_size(None) == 0
    assert L.gpz_batch_launches(None) == 0
    assert L.gpz_batch_run(None, C.c_void_p(256), 1 << 20, None, 0, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_batch_sync_status(None, C.c_void_p(256), None, None) == gpz.ERR_INVALID_ARG
    cfg = gpz.gpz_batch_config()
    assert L.gpz_batch_set_config(None, C.byref(cfg)) == gpz.ERR_INVALID_ARG
    assert L.gpz_batch_get_config(None, C.byref(cfg)) == gpz.ERR_INVALID_ARG
    assert L.gpz_batch_tune(None, C.c_void_p(256), 1 << 20, None, 1, None, None, None) == gpz.ERR_INVALID_ARG
    L.gpz_batch_destroy(None)


def test_server_argument_errors_need_no_device(gpz):
    L = gpz.lib
    h = C.c_void_p()
    bad = [gpz.gpz_server_config(1 << 30, 0, 8, 0, 0), gpz.gpz_server_config(1 << 30, 9, 8, 0, 0),
           gpz.gpz_server_config(1 << 30, 2, 0, 0, 0), gpz.gpz_server_config(1000, 2, 8, 0, 0)]
    for cfg in bad:
        assert L.gpz_server_create(C.byref(cfg), None, C.byref(h)) == gpz.ERR_INVALID_ARG
        assert not h.value
    assert L.gpz_server_create(None, None, C.byref(h)) == gpz.ERR_INVALID_ARG
    rid = C.c_uint64()
    p = gpz.make_params(3, 1e-3)
    fields = (C.c_void_p * 3)(16, 32, 48)
    assert L.gpz_server_submit_compress(None, fields, 10, C.byref(p), C.byref(rid)) == gpz.ERR_INVALID_ARG
    assert L.gpz_server_submit_decompress(None, C.c_void_p(4096), 1024, 3, 10, C.byref(rid)) == gpz.ERR_INVALID_ARG
    out = (gpz.gpz_request_result * 4)()
    assert L.gpz_server_poll(None, out, 4, 0) == 0
    assert L.gpz_server_release(None, 1) == gpz.ERR_INVALID_ARG
    assert L.gpz_server_stats_get(None, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_server_now_ns(None) == 0
    L.gpz_server_destroy(None)


def test_wide_sizes_match_oracle(gpz, oracle):
    """The 64-bit form's bound: 4 (16 + 4F + 2 nblocks + 1 + 2 F n) bytes."""
    for n in (0, 1, 1023, 1025, 10**6):
        for F in (1, 3, 6, 8):
            nb = (n + 1023) // 1024
            assert gpz.gpz_bound_size_wide(n, F) == oracle.bound_size_wide(n, F) == 4 * (16 + 4 * F + 2 * nb + 1 + 2 * F * n)
            assert gpz.lib.gpz_compress_wide_workspace_size(n, F) >= 8 * F * n
    assert gpz.gpz_bound_size_wide(10, 0) == 0 and gpz.gpz_bound_size_wide(10, 9) == 0
    # gpz_compress_f64 may fall back to the 64-bit form: its workspace covers that form's
    for n, F in ((1000, 3), (1 << 20, 6)):
        assert gpz.lib.gpz_compress_f64_workspace_size(n, F) >= gpz.lib.gpz_compress_wide_workspace_size(n, F)


def test_wide_argument_errors_need_no_device(gpz):
    """Invalid arguments to the 64-bit entry points are rejected before anything is enqueued."""
    L = gpz.lib
    p = gpz.make_params(3, 1e-9)
    fields = (C.c_void_p * 3)(4096, 8192, 12288)
    out = C.c_void_p(1 << 20)
    ws = C.c_void_p(1 << 24)
    n = 1000
    need = int(L.gpz_compress_wide_workspace_size(n, 3))
    cap = gpz.gpz_bound_size_wide(n, 3)

    def comp(params, flds=fields, o=out, c=cap, w=ws, wsz=need):
        return L.gpz_compress_wide(flds, n, params, o, c, None, None, None, w, wsz, None, None)

    assert comp(None) == gpz.ERR_INVALID_ARG
    bad = gpz.make_params(3, 1e-9)
    bad.eb[2] = -1.0
    assert comp(C.byref(bad)) == gpz.ERR_INVALID_ARG
    assert comp(C.byref(gpz.make_params(3, 1e-9, seg_bits=4))) == gpz.ERR_INVALID_ARG
    assert comp(C.byref(p), flds=(C.c_void_p * 3)(4096, 8196, 12288)) == gpz.ERR_INVALID_ARG  # field not 8-byte aligned
    assert comp(C.byref(p), w=None) == gpz.ERR_INVALID_ARG                                     # workspace required
    assert comp(C.byref(p), w=C.c_void_p((1 << 24) + 64)) == gpz.ERR_INVALID_ARG              # not 256-byte aligned
    assert comp(C.byref(p), wsz=need - 1) == gpz.ERR_CAPACITY
    assert comp(C.byref(p), c=cap - 4) == gpz.ERR_CAPACITY                                     # absolute bound: no range pass first
    assert comp(C.byref(p), o=C.c_void_p((1 << 20) + 2)) == gpz.ERR_INVALID_ARG
    outs = (C.c_void_p * 3)(4096, 8192, 12288)
    assert L.gpz_decompress_wide(None, 1024, outs, 3, n, ws, 256, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_decompress_wide(out, 1024, outs, 0, n, ws, 256, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_decompress_wide(out, 1024, outs, 3, n, None, 256, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_decompress_wide(out, 1024, outs, 3, n, ws, 8, None) == gpz.ERR_CAPACITY
    assert L.gpz_decompress_wide(out, 1024, (C.c_void_p * 3)(4096, 8196, 12288), 3, n, ws, 256, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_decompress_wide(out, 60, outs, 3, n, ws, 256, None) == gpz.ERR_CORRUPT       # shorter than the header


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """The product path has no fallback: a copy of the binding with no
    libgpz.so beside it must fail at import, naming the missing library."""
    shutil.copy(os.path.join(ROOT, "paper_2508_10305_gb300", "gpz.py"), tmp_path / "gpz.py")
    code = ("import importlib.util, sys\n"
            "spec = importlib.util.spec_from_file_location('gpz_copy', sys.argv[1])\n"
            "m = importlib.util.module_from_spec(spec)\n"
            "try:\n"
            "    spec.loader.exec_module(m)\n"
            "except ImportError as e:\n"
            "    print('refused:', e); sys.exit(3)\n"
            "sys.exit(0)\n")
    r = subprocess.run(["python", "-c", code, str(tmp_path / "gpz.py")], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 3, r.stdout + r.stderr
    assert "libgpz.so is not built" in r.stdout


def test_package_never_reaches_the_oracle():
    """Only the tests, the smoke check and the benchmark's CPU leg may use the
    oracle; no source file of the package (Python or CUDA) imports it, links
    its library or calls one of its functions."""
    pkg = os.path.join(ROOT, "paper_2508_10305_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                if re.search(r"(from|import)\s+oracle\b|gpz_oracle|gpzo_|oracle[/\\]", text):
                    offenders.append(f)
    assert not offenders, offenders


def test_failure_hooks_need_no_device(gpz):
    """The hooks refuse bad arguments before any device call, and an armed
    allocation failure makes a call without a workspace return
    GPZ_ERR_OOM before it touches the device (its arguments are checked
    first, and the allocation is the call's first device operation)."""
    L = gpz.lib
    assert L.gpz_test_scan_timeout(0, 1000, None, 0, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_test_scan_timeout(1, 0, 256, 1 << 20, None) == gpz.ERR_INVALID_ARG
    placed = C.c_int(0)
    assert L.gpz_test_block_lookback_timeout(0, 1000, 256, 4096, C.byref(placed), None) == gpz.ERR_INVALID_ARG
    assert L.gpz_test_block_lookback_timeout(5, 1000, None, 4096, C.byref(placed), None) == gpz.ERR_INVALID_ARG
    assert L.gpz_test_scan_workspace_size() > 8 * 8193
    assert gpz.gpz_test_fail_next_allocations(2) == 0
    try:
        params = gpz.make_params(3, 1e-2)
        fake = (C.c_void_p * 3)(4096, 8192, 12288)  # never dereferenced: the call stops at the allocation
        cap = gpz.gpz_bound_size(100, 3)
        assert L.gpz_compress(fake, 100, C.byref(params), 65536, cap, None, None, None, None, 0, None) == gpz.ERR_OOM
        assert L.gpz_decompress(65536, 4 * 64, fake, 3, 100, None, 0, None) == gpz.ERR_OOM
        assert gpz.gpz_test_fail_next_allocations(0) == 0
    finally:
        gpz.gpz_test_fail_next_allocations(0)


def test_copy_stream_argument_errors_need_no_device(gpz):
    L = gpz.lib
    assert L.gpz_copy_stream(None, 256, 256, 64, None) == gpz.ERR_INVALID_ARG
    assert L.gpz_copy_stream(256, 258, 256, 64, None) == gpz.ERR_INVALID_ARG  # src not 4-byte aligned
    assert L.gpz_copy_stream(256, 512, 260, 64, None) == gpz.ERR_INVALID_ARG  # size word not 8-byte aligned
