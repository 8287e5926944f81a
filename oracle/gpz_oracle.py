"""ctypes wrapper of the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain numpy marshalling around oracle/libgpz_oracle.so (built by
oracle/build.py).  Only tests/, the smoke check and the benchmark's CPU
baseline import this module; the product path must never reach it.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_UNSUPPORTED = 0, 1, 2, 3, 7
BLOCK = 1024


class FieldParams(C.Structure):
    _fields_ = [("eb", C.c_float), ("s", C.c_float), ("inv", C.c_float), ("ebchk", C.c_float)]

    def as_tuple(self):
        return (self.eb, self.s, self.inv, self.ebchk)


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        u32p, f32p, u8p = P(C.c_uint32), P(C.c_float), P(C.c_uint8)
        L.gpzo_params_abs.argtypes = [C.c_double, P(FieldParams)]
        L.gpzo_params_rel.argtypes = [C.c_double, f32p, C.c_uint64, P(FieldParams)]
        L.gpzo_bound_size.argtypes = [C.c_uint64, C.c_int]
        L.gpzo_bound_size.restype = C.c_uint64
        L.gpzo_bound_size_b.argtypes = [C.c_uint64, C.c_int, C.c_uint32]
        L.gpzo_bound_size_b.restype = C.c_uint64
        L.gpzo_encode_block.argtypes = [P(f32p), C.c_int, C.c_int, C.c_int, P(FieldParams), u32p,
                                        C.c_uint32, u32p, u32p]
        L.gpzo_decode_block.argtypes = [u32p, C.c_uint32, C.c_int, C.c_int, C.c_int, f32p, P(f32p)]
        L.gpzo_block_stages.argtypes = [P(f32p), C.c_int, C.c_int, C.c_int, P(FieldParams),
                                        P(C.c_int), f32p, u32p, u32p, u32p, u32p, u32p, u32p, u32p,
                                        u32p, u32p]
        L.gpzo_pack_fixed.argtypes = [u32p, C.c_uint32, C.c_uint32, u32p]
        L.gpzo_pack_fixed.restype = C.c_uint32
        L.gpzo_unpack_fixed.argtypes = [u32p, C.c_uint32, C.c_uint32, u32p]
        L.gpzo_compress.argtypes = [P(f32p), C.c_uint64, C.c_int, C.c_int, P(C.c_double), C.c_int,
                                    u8p, C.c_uint64, P(C.c_uint64), u32p]
        L.gpzo_compress_b.argtypes = [P(f32p), C.c_uint64, C.c_int, C.c_int, P(C.c_double), C.c_int,
                                      C.c_uint32, u8p, C.c_uint64, P(C.c_uint64), u32p]
        L.gpzo_decompress.argtypes = [u8p, C.c_uint64, P(f32p), C.c_int, C.c_uint64]
        L.gpzo_decompress_b.argtypes = [u8p, C.c_uint64, P(f32p), C.c_int, C.c_uint64, C.c_int]
        L.gpzo_compress_f64.argtypes = [P(C.c_void_p), C.c_uint64, C.c_int, C.c_int, P(C.c_double), C.c_int,
                                        u8p, C.c_uint64, P(C.c_uint64), u32p, P(C.c_double)]
        dp = P(C.c_double)
        L.gpzo_params_wide.argtypes = [C.c_double, dp, dp, dp]
        L.gpzo_bound_size_wide.argtypes = [C.c_uint64, C.c_int]
        L.gpzo_bound_size_wide.restype = C.c_uint64
        L.gpzo_compress_wide.argtypes = [P(C.c_void_p), C.c_uint64, C.c_int, C.c_int, dp, C.c_int, u8p, C.c_uint64,
                                         P(C.c_uint64), u32p, dp]
        L.gpzo_decompress_wide.argtypes = [u8p, C.c_uint64, P(C.c_void_p), C.c_int, C.c_uint64]
        L.gpzo_wide_first_candidate_failures.argtypes = [dp, C.c_uint64, C.c_double, C.c_double, P(C.c_uint64)]
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _field_ptrs(fields):
    """fields: 2-D float32 C-contiguous array [F, n] -> (F-array of float*, keepalive)."""
    arr = (C.POINTER(C.c_float) * fields.shape[0])()
    for f in range(fields.shape[0]):
        arr[f] = _ptr(fields[f], C.c_float)
    return arr


def _as_fields(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x[None, :]
    return x


def params_abs(eb):
    p = FieldParams()
    rc = lib().gpzo_params_abs(float(eb), C.byref(p))
    if rc != OK:
        raise ValueError("gpzo_params_abs failed: %d" % rc)
    return p


def params_rel(rel, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    p = FieldParams()
    rc = lib().gpzo_params_rel(float(rel), _ptr(x, C.c_float), x.size, C.byref(p))
    if rc != OK:
        raise ValueError("gpzo_params_rel failed: %d" % rc)
    return p


def bound_size(n, n_fields, block=1024):
    return int(lib().gpzo_bound_size_b(n, n_fields, block))


def _params_array(params):
    arr = (FieldParams * len(params))()
    for i, p in enumerate(params):
        arr[i] = p
    return arr


def encode_block(fields, seg_bits, params, want_perm=True):
    """Encode one block: fields [F, n_b] float32; params: list of FieldParams."""
    x = _as_fields(fields)
    F, n_b = x.shape
    cap = 1 + F * n_b + 64
    out = np.zeros(cap, dtype=np.uint32)
    nw = C.c_uint32(0)
    perm = np.zeros(n_b, dtype=np.uint32) if want_perm else None
    rc = lib().gpzo_encode_block(_field_ptrs(x), F, n_b, seg_bits, _params_array(params),
                                 _ptr(out, C.c_uint32), cap, C.byref(nw),
                                 _ptr(perm, C.c_uint32) if want_perm else None)
    if rc != OK:
        raise ValueError("gpzo_encode_block failed: %d" % rc)
    return out[:nw.value].copy(), perm


def decode_block(words, n_fields, n_b, seg_bits, steps):
    """One block's words -> [F, n_b] float32 (block-sorted order)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    s = np.ascontiguousarray(steps, dtype=np.float32)
    out = np.zeros((n_fields, n_b), dtype=np.float32)
    rc = lib().gpzo_decode_block(_ptr(w, C.c_uint32), w.size, n_fields, n_b, seg_bits,
                                 _ptr(s, C.c_float), _field_ptrs(out))
    if rc != OK:
        raise RuntimeError("gpzo_decode_block failed: %d" % rc)
    return out


def block_stages(fields, seg_bits, params):
    """All intermediate results of one block, as a dict of numpy arrays."""
    x = _as_fields(fields)
    F, n_b = x.shape
    is_raw = C.c_int(0)
    mins = np.zeros(F, np.float32)
    bits = np.zeros(F, np.uint32)
    q = np.zeros((F, n_b), np.uint32)
    seg_id = np.zeros((F, n_b), np.uint32)
    seg_off = np.zeros((F, n_b), np.uint32)
    key = np.zeros(n_b, np.uint32)
    perm = np.zeros(n_b, np.uint32)
    nu = C.c_uint32(0)
    uniq = np.zeros(n_b, np.uint32)
    counts = np.zeros(n_b, np.uint32)
    u32 = C.c_uint32
    rc = lib().gpzo_block_stages(_field_ptrs(x), F, n_b, seg_bits, _params_array(params),
                                 C.byref(is_raw), _ptr(mins, C.c_float), _ptr(bits, u32),
                                 _ptr(q, u32), _ptr(seg_id, u32), _ptr(seg_off, u32),
                                 _ptr(key, u32), _ptr(perm, u32), C.byref(nu), _ptr(uniq, u32),
                                 _ptr(counts, u32))
    if rc != OK:
        raise ValueError("gpzo_block_stages failed: %d" % rc)
    U = nu.value
    return dict(raw=bool(is_raw.value), mins=mins, bits=bits, q=q, seg_id=seg_id,
                seg_off=seg_off, key=key, perm=perm, uniq=uniq[:U].copy(),
                counts=counts[:U].copy())


def pack_fixed(values, w):
    v = np.ascontiguousarray(values, dtype=np.uint32)
    out = np.zeros((v.size * w + 31) // 32 + 1, dtype=np.uint32)
    nw = lib().gpzo_pack_fixed(_ptr(v, C.c_uint32), v.size, w, _ptr(out, C.c_uint32))
    return out[:nw].copy()


def unpack_fixed(words, length, w):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros(length, dtype=np.uint32)
    lib().gpzo_unpack_fixed(_ptr(words, C.c_uint32), length, w, _ptr(out, C.c_uint32))
    return out


def compress(fields, eb, mode=0, seg_bits=3, want_perm=True, block=1024):
    """Compress [F, n] float32 -> (stream bytes as np.uint8, perm or None);
    block: the block size (256, 512, 1024 -- the paper's -- or 2048)."""
    x = _as_fields(fields)
    F, n = x.shape
    ebs = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (F,)))
    cap = bound_size(n, F, block)
    out = np.zeros(max(cap, 4), dtype=np.uint8)
    size = C.c_uint64(0)
    perm = np.zeros(n, dtype=np.uint32) if want_perm else None
    rc = lib().gpzo_compress_b(_field_ptrs(x), n, F, mode, _ptr(ebs, C.c_double), seg_bits, block,
                               _ptr(out, C.c_uint8), cap, C.byref(size),
                               _ptr(perm, C.c_uint32) if want_perm else None)
    if rc != OK:
        raise RuntimeError("gpzo_compress failed: %d" % rc)
    return out[:size.value].copy(), perm


def compress_status(fields, eb, mode=0, seg_bits=3, cap=None):
    """Return only the status code (for argument-error tests)."""
    x = _as_fields(fields)
    F, n = x.shape
    ebs = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (F,)))
    cap = bound_size(n, F) if cap is None else cap
    out = np.zeros(max(cap, 4), dtype=np.uint8)
    size = C.c_uint64(0)
    return lib().gpzo_compress(_field_ptrs(x), n, F, mode, _ptr(ebs, C.c_double), seg_bits,
                               _ptr(out, C.c_uint8), cap, C.byref(size), None)


def compress_f64(fields, eb, mode=0, seg_bits=3, want_perm=True):
    """fp64 [F, n] -> (stream bytes, perm or None, the reduced absolute bounds eb'_f)."""
    x = np.ascontiguousarray(fields, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    F, n = x.shape
    ebs = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (F,)))
    cap = bound_size(n, F)
    out = np.zeros(max(cap, 4), dtype=np.uint8)
    size = C.c_uint64(0)
    perm = np.zeros(n, dtype=np.uint32) if want_perm else None
    used = np.zeros(F, dtype=np.float64)
    ptrs = (C.c_void_p * F)(*[x[f].ctypes.data for f in range(F)])
    rc = lib().gpzo_compress_f64(ptrs, n, F, mode, _ptr(ebs, C.c_double), seg_bits, _ptr(out, C.c_uint8), cap,
                                 C.byref(size), _ptr(perm, C.c_uint32) if want_perm else None,
                                 _ptr(used, C.c_double))
    if rc != OK:
        raise RuntimeError("gpzo_compress_f64 failed: %d" % rc)
    return out[:size.value].copy(), perm, used


def compress_f64_status(fields, eb, mode=0, seg_bits=3):
    """Only the status code of gpzo_compress_f64."""
    x = np.ascontiguousarray(fields, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    F, n = x.shape
    ebs = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (F,)))
    cap = bound_size(n, F)
    out = np.zeros(max(cap, 4), dtype=np.uint8)
    size = C.c_uint64(0)
    ptrs = (C.c_void_p * F)(*[x[f].ctypes.data for f in range(F)])
    return lib().gpzo_compress_f64(ptrs, n, F, mode, _ptr(ebs, C.c_double), seg_bits, _ptr(out, C.c_uint8), cap,
                                   C.byref(size), None, None)


def decompress(stream, n_fields, n, any_block=False):
    """Stream bytes -> [F, n] float32 in block-sorted order (any_block: also
    streams of a block size other than 1024, which gpzo_compress_b writes)."""
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros((n_fields, n), dtype=np.float32)
    rc = lib().gpzo_decompress_b(_ptr(s, C.c_uint8), s.size, _field_ptrs(out), n_fields, n, 1 if any_block else 0)
    if rc != OK:
        raise RuntimeError("gpzo_decompress failed: %d" % rc)
    return out


def decompress_status(stream, n_fields, n):
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros((n_fields, n), dtype=np.float32)
    return lib().gpzo_decompress(_ptr(s, C.c_uint8), s.size, _field_ptrs(out), n_fields, n)


# ---------------------------------------------------------------- 64-bit intermediates

def params_wide(eb):
    """(s, inv, ebchk) of the 64-bit form for an absolute bound eb."""
    s, inv, chk = C.c_double(0), C.c_double(0), C.c_double(0)
    rc = lib().gpzo_params_wide(float(eb), C.byref(s), C.byref(inv), C.byref(chk))
    if rc != OK:
        raise ValueError("gpzo_params_wide failed: %d" % rc)
    return s.value, inv.value, chk.value


def bound_size_wide(n, n_fields):
    return int(lib().gpzo_bound_size_wide(n, n_fields))


def _f64_fields(fields):
    x = np.ascontiguousarray(fields, dtype=np.float64)
    if x.ndim == 1:
        x = x[None, :]
    return x


def compress_wide_status(fields, eb, mode=0, seg_bits=3, want_perm=True):
    """fp64 [F, n] -> (status, stream bytes, perm or None, absolute bounds used)."""
    x = _f64_fields(fields)
    F, n = x.shape
    ebs = np.ascontiguousarray(np.broadcast_to(np.asarray(eb, dtype=np.float64), (F,)))
    cap = bound_size_wide(n, F)
    out = np.zeros(max(cap, 4), dtype=np.uint8)
    size = C.c_uint64(0)
    perm = np.zeros(n, dtype=np.uint32) if want_perm else None
    used = np.zeros(F, dtype=np.float64)
    ptrs = (C.c_void_p * F)(*[x[f].ctypes.data for f in range(F)])
    rc = lib().gpzo_compress_wide(ptrs, n, F, mode, _ptr(ebs, C.c_double), seg_bits, _ptr(out, C.c_uint8), cap,
                                  C.byref(size), _ptr(perm, C.c_uint32) if want_perm else None,
                                  _ptr(used, C.c_double))
    return rc, out[:size.value].copy(), perm, used


def compress_wide(fields, eb, mode=0, seg_bits=3, want_perm=True):
    rc, s, perm, used = compress_wide_status(fields, eb, mode, seg_bits, want_perm)
    if rc != OK:
        raise RuntimeError("gpzo_compress_wide failed: %d" % rc)
    return s, perm, used


def decompress_wide_status(stream, n_fields, n):
    """Stream bytes -> (status, [F, n] float64 in block-sorted order)."""
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros((n_fields, n), dtype=np.float64)
    ptrs = (C.c_void_p * n_fields)(*[out[f].ctypes.data for f in range(n_fields)])
    rc = lib().gpzo_decompress_wide(_ptr(s, C.c_uint8), s.size, ptrs, n_fields, n)
    return rc, out


def decompress_wide(stream, n_fields, n):
    rc, out = decompress_wide_status(stream, n_fields, n)
    if rc != OK:
        raise RuntimeError("gpzo_decompress_wide failed: %d" % rc)
    return out


def wide_first_candidate_failures(x, boundary_min, eb):
    """Values of x whose first candidate fails the 64-bit form's check."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = C.c_uint64(0)
    rc = lib().gpzo_wide_first_candidate_failures(_ptr(x, C.c_double), x.size, float(boundary_min), float(eb),
                                                  C.byref(out))
    if rc != OK:
        raise ValueError("gpzo_wide_first_candidate_failures failed: %d" % rc)
    return int(out.value)
