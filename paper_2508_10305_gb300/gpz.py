"""Python binding of libgpz (include/gpz.h): the same entry points, argument
marshalling only.  Every step of compression and decompression runs in the
library's CUDA kernels; this module only turns torch tensors into pointers
and streams into handles.

There is no fallback: if libgpz.so has not been built, importing this module
raises.  Build it with ``python -c "import __graft_entry__ as g; g.build()"``
or ``python paper_2508_10305_gb300/build.py``.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpz.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED = range(8)
EB_ABS, EB_REL = 0, 1
FLAG_FUSED_COMPACTION = 1
MAX_FIELDS = 8
BLOCK = 1024


class gpz_params(C.Structure):
    _fields_ = [("mode", C.c_int), ("n_fields", C.c_int), ("seg_bits", C.c_int), ("flags", C.c_uint),
                ("eb", C.c_double * MAX_FIELDS)]


class gpz_compress_chunk(C.Structure):
    _fields_ = [("fields", C.c_void_p * MAX_FIELDS), ("n", C.c_uint64), ("params", gpz_params),
                ("out", C.c_void_p), ("out_capacity", C.c_uint64), ("perm", C.c_void_p)]


class gpz_decompress_chunk(C.Structure):
    _fields_ = [("in_", C.c_void_p), ("in_size", C.c_uint64), ("fields", C.c_void_p * MAX_FIELDS),
                ("n_fields", C.c_int), ("n", C.c_uint64)]


class gpz_batch_config(C.Structure):
    _fields_ = [("range_slice", C.c_uint32), ("compact_ctas", C.c_uint32), ("general_ctas", C.c_uint32),
                ("qse_form", C.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class gpz_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("lanes", C.c_uint32), ("max_batch", C.c_uint32),
                ("max_batch_bytes", C.c_uint64), ("lane_bytes", C.c_uint64)]


class gpz_request_result(C.Structure):
    _fields_ = [("id", C.c_uint64), ("kind", C.c_int), ("status", C.c_int), ("out", C.c_void_p),
                ("out_bytes", C.c_uint64), ("field_stride", C.c_uint64), ("in_bytes", C.c_uint64),
                ("t_submit_ns", C.c_uint64), ("t_start_ns", C.c_uint64), ("t_done_ns", C.c_uint64),
                ("batch", C.c_uint32), ("batch_size", C.c_uint32)]


class gpz_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("in_bytes", C.c_uint64), ("arena_peak", C.c_uint64), ("arena_in_use", C.c_uint64),
                ("queued", C.c_uint64)]


class GpzError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, gpz_status_str(status), status))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgpz.so is not built (%s); run paper_2508_10305_gb300/build.py" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P, u64, vp = C.POINTER, C.c_uint64, C.c_void_p
    L.gpz_bound_size.argtypes = [u64, C.c_int]
    L.gpz_bound_size.restype = u64
    L.gpz_compress_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_compress_workspace_size.restype = u64
    L.gpz_decompress_workspace_size.argtypes = []
    L.gpz_decompress_workspace_size.restype = u64
    L.gpz_compress.argtypes = [P(vp), u64, P(gpz_params), vp, u64, vp, P(u64), vp, vp, u64, vp]
    L.gpz_compress.restype = C.c_int
    L.gpz_compress_noalloc.argtypes = [P(vp), u64, P(gpz_params), vp, u64, vp, P(u64), vp, vp]
    L.gpz_compress_noalloc.restype = C.c_int
    L.gpz_noalloc_prepare.argtypes = []
    L.gpz_noalloc_prepare.restype = C.c_int
    L.gpz_noalloc_sync_status.argtypes = [vp]
    L.gpz_noalloc_sync_status.restype = C.c_int
    L.gpz_decompress.argtypes = [vp, u64, P(vp), C.c_int, u64, vp, u64, vp]
    L.gpz_decompress.restype = C.c_int
    L.gpz_copy_stream.argtypes = [vp, vp, vp, u64, vp]
    L.gpz_copy_stream.restype = C.c_int
    L.gpz_sync_status.argtypes = [vp, vp]
    L.gpz_sync_status.restype = C.c_int
    L.gpz_inspect.argtypes = [vp, u64, P(u64), P(C.c_int), P(C.c_int), P(C.c_int)]
    L.gpz_inspect.restype = C.c_int
    L.gpz_status_str.argtypes = [C.c_int]
    L.gpz_status_str.restype = C.c_char_p
    L.gpz_set_stage_timing.argtypes = [vp, C.c_int]
    L.gpz_set_stage_timing.restype = None
    L.gpz_compress_f64_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_compress_f64_workspace_size.restype = u64
    L.gpz_decompress_f64_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_decompress_f64_workspace_size.restype = u64
    L.gpz_compress_f64.argtypes = [vp, u64, P(gpz_params), vp, u64, vp, P(u64), vp, vp, u64, P(C.c_double), vp]
    L.gpz_compress_f64.restype = C.c_int
    L.gpz_decompress_f64.argtypes = [vp, u64, vp, C.c_int, u64, vp, u64, vp]
    L.gpz_decompress_f64.restype = C.c_int
    L.gpz_bound_size_wide.argtypes = [u64, C.c_int]
    L.gpz_bound_size_wide.restype = u64
    L.gpz_compress_wide_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_compress_wide_workspace_size.restype = u64
    L.gpz_compress_wide.argtypes = [vp, u64, P(gpz_params), vp, u64, vp, P(u64), vp, vp, u64, P(C.c_double), vp]
    L.gpz_compress_wide.restype = C.c_int
    L.gpz_decompress_wide.argtypes = [vp, u64, vp, C.c_int, u64, vp, u64, vp]
    L.gpz_decompress_wide.restype = C.c_int
    L.gpz_compress_aos_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_compress_aos_workspace_size.restype = u64
    L.gpz_decompress_aos_workspace_size.argtypes = [u64, C.c_int]
    L.gpz_decompress_aos_workspace_size.restype = u64
    L.gpz_compress_aos.argtypes = [vp, u64, P(gpz_params), vp, u64, vp, P(u64), vp, vp, u64, vp]
    L.gpz_compress_aos.restype = C.c_int
    L.gpz_decompress_aos.argtypes = [vp, u64, vp, C.c_int, u64, vp, u64, vp]
    L.gpz_decompress_aos.restype = C.c_int
    L.gpz_stage_times.argtypes = [P(C.c_char_p), P(C.c_float), P(C.c_int), C.c_int]
    L.gpz_stage_times.restype = C.c_int
    L.gpz_launch_count.argtypes = [C.c_int]
    L.gpz_launch_count.restype = u64
    L.gpz_pooled_bytes.argtypes = []
    L.gpz_pooled_bytes.restype = u64
    L.gpz_release_pooled_memory.argtypes = []
    L.gpz_release_pooled_memory.restype = C.c_int
    # failure-injection hooks (include/gpz_test.h)
    L.gpz_test_fail_next_allocations.argtypes = [C.c_int]
    L.gpz_test_fail_next_allocations.restype = C.c_int
    L.gpz_test_scan_workspace_size.argtypes = []
    L.gpz_test_scan_workspace_size.restype = u64
    L.gpz_test_scan_timeout.argtypes = [C.c_int, C.c_uint32, vp, u64, vp]
    L.gpz_test_scan_timeout.restype = C.c_int
    L.gpz_test_block_lookback_timeout.argtypes = [C.c_uint32, C.c_uint32, vp, u64, P(C.c_int), vp]
    L.gpz_test_block_lookback_timeout.restype = C.c_int
    # batched entry points (include/gpz_batch.h)
    L.gpz_batch_create_compress.argtypes = [P(gpz_compress_chunk), C.c_uint32, P(vp)]
    L.gpz_batch_create_compress.restype = C.c_int
    L.gpz_batch_create_decompress.argtypes = [P(gpz_decompress_chunk), C.c_uint32, P(vp)]
    L.gpz_batch_create_decompress.restype = C.c_int
    L.gpz_batch_destroy.argtypes = [vp]
    L.gpz_batch_destroy.restype = None
    L.gpz_batch_workspace_size.argtypes = [vp]
    L.gpz_batch_workspace_size.restype = u64
    L.gpz_batch_set_config.argtypes = [vp, P(gpz_batch_config)]
    L.gpz_batch_set_config.restype = C.c_int
    L.gpz_batch_get_config.argtypes = [vp, P(gpz_batch_config)]
    L.gpz_batch_get_config.restype = C.c_int
    L.gpz_batch_run.argtypes = [vp, vp, u64, vp, C.c_int, vp]
    L.gpz_batch_run.restype = C.c_int
    L.gpz_batch_sync_status.argtypes = [vp, vp, P(C.c_uint32), vp]
    L.gpz_batch_sync_status.restype = C.c_int
    L.gpz_batch_tune.argtypes = [vp, vp, u64, vp, C.c_int, vp, P(gpz_batch_config), P(C.c_float)]
    L.gpz_batch_tune.restype = C.c_int
    L.gpz_batch_launches.argtypes = [vp]
    L.gpz_batch_launches.restype = C.c_uint32
    # serving engine (include/gpz_serve.h)
    L.gpz_server_create.argtypes = [P(gpz_server_config), P(gpz_server_config), P(vp)]
    L.gpz_server_create.restype = C.c_int
    L.gpz_server_submit_compress.argtypes = [vp, P(vp), u64, P(gpz_params), P(u64)]
    L.gpz_server_submit_compress.restype = C.c_int
    L.gpz_server_submit_decompress.argtypes = [vp, vp, u64, C.c_int, u64, P(u64)]
    L.gpz_server_submit_decompress.restype = C.c_int
    L.gpz_server_poll.argtypes = [vp, P(gpz_request_result), C.c_int, C.c_int]
    L.gpz_server_poll.restype = C.c_int
    L.gpz_server_release.argtypes = [vp, u64]
    L.gpz_server_release.restype = C.c_int
    L.gpz_server_stats_get.argtypes = [vp, P(gpz_server_stats)]
    L.gpz_server_stats_get.restype = C.c_int
    L.gpz_server_now_ns.argtypes = [vp]
    L.gpz_server_now_ns.restype = u64
    L.gpz_server_destroy.argtypes = [vp]
    L.gpz_server_destroy.restype = None
    return L


lib = _load()


# ----------------------------------------------------------------------------- raw entry points

def gpz_bound_size(n, n_fields):
    return int(lib.gpz_bound_size(n, n_fields))


def gpz_compress_workspace_size(n, n_fields):
    return int(lib.gpz_compress_workspace_size(n, n_fields))


def gpz_decompress_workspace_size():
    return int(lib.gpz_decompress_workspace_size())


def gpz_status_str(status):
    return lib.gpz_status_str(status).decode()


def gpz_set_stage_timing(enable, stream=None):
    """Time the later calls enqueued on `stream` (the current stream when None)."""
    lib.gpz_set_stage_timing(_stream_handle(stream), 1 if enable else 0)


def gpz_compress_aos_workspace_size(n, n_fields):
    return int(lib.gpz_compress_aos_workspace_size(n, n_fields))


def gpz_decompress_aos_workspace_size(n, n_fields):
    return int(lib.gpz_decompress_aos_workspace_size(n, n_fields))


def compress_aos(x_aos, n_fields, eb, mode=EB_ABS, seg_bits=3, want_perm=False, stream=None):
    """x_aos: CUDA float32 tensor of n * n_fields values, particle-major.
    Returns (stream bytes as a CUDA uint8 tensor of the exact size, perm or None)."""
    n = x_aos.numel() // n_fields
    dev = x_aos.device
    params = make_params(n_fields, eb, mode, seg_bits)
    cap = gpz_bound_size(n, n_fields)
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=dev)
    ws_size = gpz_compress_aos_workspace_size(n, n_fields)
    ws = torch.empty(max(ws_size, 256), dtype=torch.uint8, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if want_perm else None
    h = C.c_uint64(0)
    st = lib.gpz_compress_aos(x_aos.data_ptr() if n else None, n, C.byref(params), out.data_ptr(), cap, None,
                              C.byref(h), perm.data_ptr() if want_perm else None, ws.data_ptr(), ws_size,
                              _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_compress_aos")
    return out[:h.value], (perm[:n] if want_perm else None)


def decompress_aos(stream_buf, n_fields, n, size=None, stream=None):
    """The inverse: a CUDA float32 tensor [n, n_fields] in block-sorted order."""
    size = stream_buf.numel() if size is None else size
    dev = stream_buf.device
    out = torch.empty((max(n, 1), n_fields), dtype=torch.float32, device=dev)
    ws_size = gpz_decompress_aos_workspace_size(n, n_fields)
    ws = torch.zeros(max(ws_size, 256), dtype=torch.uint8, device=dev)
    st = lib.gpz_decompress_aos(stream_buf.data_ptr(), size, out.data_ptr(), n_fields, n, ws.data_ptr(), ws_size,
                                _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_decompress_aos")
    st = gpz_sync_status(ws, stream)
    if st != OK:
        raise GpzError(st, "gpz_decompress_aos (device)")
    return out[:n]


def compress_f64(x, eb, mode=EB_ABS, seg_bits=3, want_perm=False, stream=None):
    """x: CUDA float64 tensor [F, n].  Returns (stream bytes as a CUDA uint8
    tensor of the exact size, perm or None, the reduced bounds eb'_f)."""
    F, n = x.shape
    dev = x.device
    params = make_params(F, eb, mode, seg_bits)
    cap = gpz_bound_size_wide(n, F)  # room for the 64-bit form, which it falls back to
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=dev)
    ws_size = int(lib.gpz_compress_f64_workspace_size(n, F))
    ws = torch.empty(max(ws_size, 256), dtype=torch.uint8, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if want_perm else None
    used = (C.c_double * F)()
    h = C.c_uint64(0)
    st = lib.gpz_compress_f64(_ptr_array([x[f] for f in range(F)]), n, C.byref(params), out.data_ptr(), cap, None,
                              C.byref(h), perm.data_ptr() if want_perm else None, ws.data_ptr(), ws_size, used,
                              _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_compress_f64")
    return out[:h.value], (perm[:n] if want_perm else None), [used[f] for f in range(F)]


def decompress_f64(stream_buf, n_fields, n, size=None, stream=None):
    """The inverse: a CUDA float64 tensor [F, n] in block-sorted order."""
    size = stream_buf.numel() if size is None else size
    dev = stream_buf.device
    out = torch.empty((n_fields, max(n, 1)), dtype=torch.float64, device=dev)
    ws_size = int(lib.gpz_decompress_f64_workspace_size(n, n_fields))
    ws = torch.zeros(max(ws_size, 256), dtype=torch.uint8, device=dev)
    st = lib.gpz_decompress_f64(stream_buf.data_ptr(), size, _ptr_array([out[f] for f in range(n_fields)]),
                                n_fields, n, ws.data_ptr(), ws_size, _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_decompress_f64")
    st = gpz_sync_status(ws, stream)
    if st != OK:
        raise GpzError(st, "gpz_decompress_f64 (device)")
    return out[:, :n]


def gpz_bound_size_wide(n, n_fields):
    return int(lib.gpz_bound_size_wide(n, n_fields))


def compress_wide(x, eb, mode=EB_ABS, seg_bits=3, want_perm=False, stream=None):
    """64-bit intermediates: x is a CUDA float64 tensor [F, n].  Returns
    (stream bytes as a CUDA uint8 tensor of the exact size, perm or None, the
    absolute bounds eb_f used)."""
    F, n = x.shape
    dev = x.device
    params = make_params(F, eb, mode, seg_bits)
    cap = gpz_bound_size_wide(n, F)
    out = torch.empty(max(cap, 16), dtype=torch.uint8, device=dev)
    ws_size = int(lib.gpz_compress_wide_workspace_size(n, F))
    ws = torch.empty(max(ws_size, 256), dtype=torch.uint8, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if want_perm else None
    used = (C.c_double * F)()
    h = C.c_uint64(0)
    st = lib.gpz_compress_wide(_ptr_array([x[f] for f in range(F)]), n, C.byref(params), out.data_ptr(), cap, None,
                               C.byref(h), perm.data_ptr() if want_perm else None, ws.data_ptr(), ws_size, used,
                               _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_compress_wide")
    return out[:h.value], (perm[:n] if want_perm else None), [used[f] for f in range(F)]


def decompress_wide(stream_buf, n_fields, n, size=None, stream=None):
    """The inverse of compress_wide: a CUDA float64 tensor [F, n] in block-sorted order."""
    size = stream_buf.numel() if size is None else size
    dev = stream_buf.device
    out = torch.empty((n_fields, max(n, 1)), dtype=torch.float64, device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    st = lib.gpz_decompress_wide(stream_buf.data_ptr(), size, _ptr_array([out[f] for f in range(n_fields)]),
                                 n_fields, n, ws.data_ptr(), ws.numel(), _stream_handle(stream))
    if st != OK:
        raise GpzError(st, "gpz_decompress_wide")
    st = gpz_sync_status(ws, stream)
    if st != OK:
        raise GpzError(st, "gpz_decompress_wide (device)")
    return out[:, :n]


def compress_deferred_blocks(ws):
    """After a fused-compaction call: the blocks the copy kernel moved."""
    return int(ws[32:36].view(torch.int32).item())


def gpz_stage_times(max_stages=8):
    """{stage: (total_ms, launches)} since the previous read (clears the log)."""
    names = (C.c_char_p * max_stages)()
    ms = (C.c_float * max_stages)()
    cnt = (C.c_int * max_stages)()
    k = lib.gpz_stage_times(names, ms, cnt, max_stages)
    return {names[i].decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}


def gpz_launch_count(reset=False):
    return int(lib.gpz_launch_count(1 if reset else 0))


def gpz_pooled_bytes():
    """Bytes held by the library's workspace pool on the current device."""
    return int(lib.gpz_pooled_bytes())


def gpz_release_pooled_memory():
    """Synchronise the current device and return the pool's unused memory."""
    return int(lib.gpz_release_pooled_memory())


def gpz_test_fail_next_allocations(count):
    """Arm `count` injected device-allocation failures; returns how many were armed before."""
    return int(lib.gpz_test_fail_next_allocations(count))


def gpz_test_scan_timeout(batched, wait_cycles, ws, stream=None):
    """Run a look-back scan whose first tile never publishes; returns the device status."""
    return lib.gpz_test_scan_timeout(1 if batched else 0, wait_cycles, ws.data_ptr() if ws is not None else None,
                                     ws.numel() if ws is not None else 0, _stream_handle(stream))


def gpz_test_block_lookback_timeout(block, wait_cycles, ws, stream=None):
    """One block's look-back with no predecessor published: (status, placed)."""
    placed = C.c_int(-1)
    st = lib.gpz_test_block_lookback_timeout(block, wait_cycles, ws.data_ptr() if ws is not None else None,
                                             ws.numel() if ws is not None else 0, C.byref(placed),
                                             _stream_handle(stream))
    return st, placed.value


def gpz_inspect(header_bytes):
    """Parse a stream header held in host memory (bytes-like, >= 64 bytes)."""
    buf = (C.c_uint8 * len(header_bytes)).from_buffer_copy(bytes(header_bytes))
    n, F, G, mode = C.c_uint64(), C.c_int(), C.c_int(), C.c_int()
    st = lib.gpz_inspect(C.cast(buf, C.c_void_p), len(header_bytes), C.byref(n), C.byref(F), C.byref(G),
                         C.byref(mode))
    if st != OK:
        raise GpzError(st, "gpz_inspect")
    return dict(n=n.value, n_fields=F.value, seg_bits=G.value, mode=mode.value)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr()
    return arr


def make_params(n_fields, eb, mode=EB_ABS, seg_bits=3, flags=0):
    p = gpz_params()
    p.mode, p.n_fields, p.seg_bits, p.flags = mode, n_fields, seg_bits, flags
    ebs = list(eb) if hasattr(eb, "__len__") else [eb] * n_fields
    if len(ebs) != n_fields:
        raise ValueError("need one error bound per field")
    for f, e in enumerate(ebs):
        p.eb[f] = float(e)
    return p


def gpz_compress(fields, n, params, out, out_capacity, d_out_size=None, h_out_size=None, perm=None, ws=None,
                 ws_size=0, stream=None):
    """Mirror of the C entry point.  fields: list of CUDA float32 tensors (or a
    2-D [F, n] tensor); out/d_out_size/perm/ws: CUDA tensors or None;
    h_out_size: a ctypes.c_uint64 or None.  Returns the status code."""
    if isinstance(fields, torch.Tensor):
        fields = [fields[f] for f in range(fields.shape[0])]
    return lib.gpz_compress(_ptr_array(fields), n, C.byref(params), out.data_ptr(), out_capacity,
                            d_out_size.data_ptr() if d_out_size is not None else None,
                            C.byref(h_out_size) if h_out_size is not None else None,
                            perm.data_ptr() if perm is not None else None,
                            ws.data_ptr() if ws is not None else None, ws_size, _stream_handle(stream))


def gpz_compress_noalloc(fields, n, params, out, out_capacity, d_out_size=None, h_out_size=None, perm=None,
                         stream=None):
    """Mirror of the C entry point that allocates nothing (its scratch space is
    a fixed array inside the library; see include/gpz.h for the limit)."""
    if isinstance(fields, torch.Tensor):
        fields = [fields[f] for f in range(fields.shape[0])]
    return lib.gpz_compress_noalloc(_ptr_array(fields), n, C.byref(params), out.data_ptr(), out_capacity,
                                    d_out_size.data_ptr() if d_out_size is not None else None,
                                    C.byref(h_out_size) if h_out_size is not None else None,
                                    perm.data_ptr() if perm is not None else None, _stream_handle(stream))


def gpz_noalloc_prepare():
    """Take gpz_compress_noalloc's scratch array on the current device now."""
    return lib.gpz_noalloc_prepare()


def gpz_noalloc_sync_status(stream=None):
    """Read and clear the device-side status of earlier gpz_compress_noalloc calls."""
    return lib.gpz_noalloc_sync_status(_stream_handle(stream))


def gpz_decompress(stream_buf, in_size, fields, n_fields, n, ws=None, ws_size=0, stream=None):
    """Mirror of the C entry point; fields: list of CUDA float32 tensors or a 2-D tensor."""
    if isinstance(fields, torch.Tensor):
        fields = [fields[f] for f in range(fields.shape[0])]
    return lib.gpz_decompress(stream_buf.data_ptr(), in_size, _ptr_array(fields), n_fields, n,
                              ws.data_ptr() if ws is not None else None, ws_size, _stream_handle(stream))


def gpz_copy_stream(dst, src, d_size, capacity, stream=None):
    """Mirror of the C entry point: dst/src/d_size are tensors (device, or
    pinned host memory); the byte count is read from d_size on the device."""
    return lib.gpz_copy_stream(dst.data_ptr(), src.data_ptr(), d_size.data_ptr(), capacity, _stream_handle(stream))


def gpz_sync_status(ws, stream=None):
    return lib.gpz_sync_status(ws.data_ptr(), _stream_handle(stream))


def gpz_batch_create_compress(chunks):
    """chunks: sequence of gpz_compress_chunk.  Returns (status, plan handle)."""
    arr = (gpz_compress_chunk * len(chunks))(*chunks)
    h = C.c_void_p()
    st = lib.gpz_batch_create_compress(arr, len(chunks), C.byref(h))
    return st, h


def gpz_batch_create_decompress(chunks):
    arr = (gpz_decompress_chunk * len(chunks))(*chunks)
    h = C.c_void_p()
    st = lib.gpz_batch_create_decompress(arr, len(chunks), C.byref(h))
    return st, h


def gpz_batch_destroy(plan):
    lib.gpz_batch_destroy(plan)


def gpz_batch_workspace_size(plan):
    return int(lib.gpz_batch_workspace_size(plan))


def gpz_batch_set_config(plan, cfg):
    return lib.gpz_batch_set_config(plan, C.byref(cfg))


def gpz_batch_get_config(plan):
    cfg = gpz_batch_config()
    st = lib.gpz_batch_get_config(plan, C.byref(cfg))
    if st != OK:
        raise GpzError(st, "gpz_batch_get_config")
    return cfg


def gpz_batch_run(plan, ws, ws_size, d_out_sizes=None, use_graph=False, stream=None):
    return lib.gpz_batch_run(plan, ws.data_ptr(), ws_size,
                             d_out_sizes.data_ptr() if d_out_sizes is not None else None,
                             1 if use_graph else 0, _stream_handle(stream))


def gpz_batch_sync_status(plan, ws, count, stream=None):
    """Returns (first status, per-chunk status list)."""
    arr = (C.c_uint32 * count)()
    st = lib.gpz_batch_sync_status(plan, ws.data_ptr(), arr, _stream_handle(stream))
    return st, [int(v) for v in arr]


def gpz_batch_tune(plan, ws, ws_size, d_out_sizes=None, reps=2, stream=None):
    """Returns (status, chosen gpz_batch_config, ms per run)."""
    cfg = gpz_batch_config()
    ms = C.c_float(0.0)
    st = lib.gpz_batch_tune(plan, ws.data_ptr(), ws_size,
                            d_out_sizes.data_ptr() if d_out_sizes is not None else None, reps,
                            _stream_handle(stream), C.byref(cfg), C.byref(ms))
    return st, cfg, float(ms.value)


def gpz_batch_launches(plan):
    return int(lib.gpz_batch_launches(plan))


# ----------------------------------------------------------------------------- convenience wrappers

class Compressor:
    """Holds the device buffers for one (n, F) shape so that repeated calls
    allocate nothing: out (bound size), workspace, size word and optional
    permutation."""

    def __init__(self, n, n_fields, eb, mode=EB_ABS, seg_bits=3, want_perm=False, device=None, flags=0):
        device = device or torch.device("cuda")
        self.n, self.F = n, n_fields
        self.params = make_params(n_fields, eb, mode, seg_bits, flags)
        self.capacity = gpz_bound_size(n, n_fields)
        self.out = torch.empty(max(self.capacity, 16), dtype=torch.uint8, device=device)
        self.ws_size = gpz_compress_workspace_size(n, n_fields)
        self.ws = torch.empty(max(self.ws_size, 256), dtype=torch.uint8, device=device)
        self.d_size = torch.zeros(1, dtype=torch.int64, device=device)
        self.perm = torch.empty(max(n, 1), dtype=torch.int32, device=device) if want_perm else None

    def __call__(self, fields, stream=None, sync=True):
        """Compress; returns the stream size in bytes (sync=True) or None."""
        h = C.c_uint64(0) if sync else None
        st = gpz_compress(fields, self.n, self.params, self.out, self.capacity, self.d_size, h,
                          self.perm, self.ws, self.ws_size, stream)
        if st != OK:
            raise GpzError(st, "gpz_compress")
        return h.value if sync else None


class Decompressor:
    def __init__(self, n, n_fields, device=None):
        device = device or torch.device("cuda")
        self.n, self.F = n, n_fields
        self.out = torch.empty((n_fields, max(n, 1)), dtype=torch.float32, device=device)
        self.ws = torch.zeros(gpz_decompress_workspace_size(), dtype=torch.uint8, device=device)

    def __call__(self, stream_buf, size, stream=None, check=True):
        st = gpz_decompress(stream_buf, size, [self.out[f] for f in range(self.F)], self.F, self.n, self.ws,
                            self.ws.numel(), stream)
        if st != OK:
            raise GpzError(st, "gpz_decompress")
        if check:
            st = gpz_sync_status(self.ws, stream)
            if st != OK:
                raise GpzError(st, "gpz_decompress (device)")
        return self.out[:, :self.n]


def compress(x, eb, mode=EB_ABS, seg_bits=3, want_perm=False, stream=None):
    """One-shot: x is a CUDA float32 tensor [F, n].  Returns (stream bytes as a
    CUDA uint8 tensor of the exact size, perm or None)."""
    if x.dim() == 1:
        x = x.unsqueeze(0)
    F, n = x.shape
    c = Compressor(n, F, eb, mode, seg_bits, want_perm, x.device)
    size = c([x[f] for f in range(F)], stream)
    return c.out[:size], (c.perm[:n] if want_perm else None)


def decompress(stream_buf, n_fields, n, stream=None):
    d = Decompressor(n, n_fields, stream_buf.device)
    return d(stream_buf, stream_buf.numel(), stream).clone()


def _fields_list(x):
    if isinstance(x, torch.Tensor):
        return [x[f] for f in range(x.shape[0])] if x.dim() == 2 else [x]
    return list(x)


class BatchCompressor:
    """A compression plan over many arrays (include/gpz_batch.h), with its
    output buffers (one of gpz_bound_size bytes per chunk), the per-chunk size
    array and the workspace.  chunks: list of (fields, params[, perm]) with
    fields a [F, n] CUDA float32 tensor or a list of F 1-D tensors."""

    def __init__(self, chunks, device=None, use_graph=True):
        device = device or torch.device("cuda")
        self.use_graph = use_graph
        self.count = len(chunks)
        self._keep = []
        descs, self.outs, self.n = [], [], []
        for ch in chunks:
            fields, params = _fields_list(ch[0]), ch[1]
            perm = ch[2] if len(ch) > 2 else None
            n = fields[0].numel() if fields else 0
            cap = gpz_bound_size(n, params.n_fields)
            out = torch.empty(max(cap, 64), dtype=torch.uint8, device=device)
            d = gpz_compress_chunk()
            for f in range(params.n_fields):
                d.fields[f] = fields[f].data_ptr() if n else None
            d.n, d.params, d.out, d.out_capacity = n, params, out.data_ptr(), cap
            d.perm = perm.data_ptr() if perm is not None else None
            descs.append(d)
            self.outs.append(out)
            self.n.append(n)
            self._keep.append((fields, perm))
        st, self.plan = gpz_batch_create_compress(descs)
        if st != OK:
            raise GpzError(st, "gpz_batch_create_compress")
        self.ws_size = gpz_batch_workspace_size(self.plan)
        self.ws = torch.empty(max(self.ws_size, 256), dtype=torch.uint8, device=device)
        self.sizes = torch.zeros(self.count, dtype=torch.int64, device=device)

    def __call__(self, stream=None):
        st = gpz_batch_run(self.plan, self.ws, self.ws_size, self.sizes, self.use_graph, stream)
        if st != OK:
            raise GpzError(st, "gpz_batch_run")

    def status(self, stream=None):
        return gpz_batch_sync_status(self.plan, self.ws, self.count, stream)

    def streams(self):
        """The chunks' streams (CUDA uint8 views of the exact sizes)."""
        sizes = self.sizes.tolist()
        return [self.outs[c][:sizes[c]] for c in range(self.count)]

    def tune(self, reps=2, stream=None):
        st, cfg, ms = gpz_batch_tune(self.plan, self.ws, self.ws_size, self.sizes, reps, stream)
        if st != OK:
            raise GpzError(st, "gpz_batch_tune")
        return cfg, ms

    def close(self):
        if self.plan:
            gpz_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchDecompressor:
    """A decompression plan: chunks is a list of (stream tensor, size in bytes,
    n_fields, n); the outputs are allocated here, one [F, n] tensor per chunk."""

    def __init__(self, chunks, device=None, use_graph=True, outs=None):
        device = device or torch.device("cuda")
        self.use_graph = use_graph
        self.count = len(chunks)
        descs = []
        self.outs = outs if outs is not None else [
            torch.empty((F, max(n, 1)), dtype=torch.float32, device=device) for (_, _, F, n) in chunks]
        self._keep = [c[0] for c in chunks]
        for (buf, size, F, n), out in zip(chunks, self.outs):
            d = gpz_decompress_chunk()
            d.in_, d.in_size, d.n_fields, d.n = buf.data_ptr(), size, F, n
            for f in range(F):
                d.fields[f] = out[f].data_ptr() if n else None
            descs.append(d)
        st, self.plan = gpz_batch_create_decompress(descs)
        if st != OK:
            raise GpzError(st, "gpz_batch_create_decompress")
        self.ws_size = gpz_batch_workspace_size(self.plan)
        self.ws = torch.empty(max(self.ws_size, 256), dtype=torch.uint8, device=device)

    def __call__(self, stream=None):
        st = gpz_batch_run(self.plan, self.ws, self.ws_size, None, self.use_graph, stream)
        if st != OK:
            raise GpzError(st, "gpz_batch_run")

    def status(self, stream=None):
        return gpz_batch_sync_status(self.plan, self.ws, self.count, stream)

    def tune(self, reps=2, stream=None):
        st, cfg, ms = gpz_batch_tune(self.plan, self.ws, self.ws_size, None, reps, stream)
        if st != OK:
            raise GpzError(st, "gpz_batch_tune")
        return cfg, ms

    def close(self):
        if self.plan:
            gpz_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A view of device memory for torch.as_tensor (no copy)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False), "version": 3}


def device_bytes(ptr, nbytes, device=None):
    """A uint8 CUDA tensor viewing nbytes of device memory at ptr (no copy)."""
    if nbytes == 0:
        return torch.empty(0, dtype=torch.uint8, device=device or "cuda")
    return torch.as_tensor(_DeviceArray(ptr, nbytes), device=device or "cuda")


class Server:
    """The serving engine (include/gpz_serve.h): submit compress / decompress
    requests, poll results, release their memory.  Keeps the inputs of each
    request alive until its result is polled."""

    def __init__(self, budget_bytes, lanes=2, max_batch=64, max_batch_bytes=0, lane_bytes=0):
        cfg = gpz_server_config(budget_bytes, lanes, max_batch, max_batch_bytes, lane_bytes)
        used = gpz_server_config()
        h = C.c_void_p()
        st = lib.gpz_server_create(C.byref(cfg), C.byref(used), C.byref(h))
        if st != OK:
            raise GpzError(st, "gpz_server_create")
        self.handle, self.config = h, used
        self._inputs = {}
        self._buf = (gpz_request_result * 256)()

    def submit_compress(self, fields, params):
        fields = _fields_list(fields)
        n = fields[0].numel() if fields else 0
        rid = C.c_uint64()
        st = lib.gpz_server_submit_compress(self.handle, _ptr_array(fields), n, C.byref(params), C.byref(rid))
        if st != OK:
            raise GpzError(st, "gpz_server_submit_compress")
        self._inputs[rid.value] = fields
        return rid.value

    def submit_decompress(self, stream_buf, size, n_fields, n):
        rid = C.c_uint64()
        st = lib.gpz_server_submit_decompress(self.handle, stream_buf.data_ptr(), size, n_fields, n, C.byref(rid))
        if st != OK:
            raise GpzError(st, "gpz_server_submit_decompress")
        self._inputs[rid.value] = stream_buf
        return rid.value

    def poll(self, max_results=256, timeout_ms=100):
        """Completed results as dicts (oldest first); their outputs stay valid until release()."""
        k = lib.gpz_server_poll(self.handle, self._buf, min(max_results, len(self._buf)), timeout_ms)
        out = []
        for i in range(k):
            r = self._buf[i]
            self._inputs.pop(r.id, None)
            out.append({name: getattr(r, name) for name, _ in gpz_request_result._fields_})
        return out

    def stream_of(self, result):
        """A polled compress result's stream as a CUDA uint8 view (valid until
        release).  A copy of it runs on the caller's current stream, which the
        engine's lanes do not wait for: synchronise that stream before
        releasing the result, or a later request may overwrite the memory
        first."""
        return device_bytes(result["out"], result["out_bytes"])

    def fields_of(self, result, n_fields, n):
        """Decompressed fields of a polled result as a [F, n] float32 CUDA
        tensor (a copy, enqueued on the caller's current stream: synchronise
        it before releasing the result)."""
        stride = result["field_stride"]
        raw = device_bytes(result["out"], stride * n_fields)
        return torch.stack([raw[f * stride:f * stride + 4 * n].view(torch.float32) for f in range(n_fields)])

    def release(self, rid):
        st = lib.gpz_server_release(self.handle, rid)
        if st != OK:
            raise GpzError(st, "gpz_server_release")

    def stats(self):
        s = gpz_server_stats()
        lib.gpz_server_stats_get(self.handle, C.byref(s))
        return {name: int(getattr(s, name)) for name, _ in gpz_server_stats._fields_}

    def now_ns(self):
        return int(lib.gpz_server_now_ns(self.handle))

    def close(self):
        if self.handle:
            lib.gpz_server_destroy(self.handle)
            self.handle = None
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
