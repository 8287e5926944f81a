"""Readers for the hand-worked fixtures under tests/golden/ and two exact
rounding helpers (rational -> nearest fp32) used to pin fp32 results without
going through the code under test."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok):
    if tok.lower().startswith("0x"):
        return int(tok, 16)
    if tok.lower() == "nan":
        return float("nan")
    if any(c in tok for c in ".eE") or tok.lower() in ("inf", "-inf"):
        return float(tok)
    return int(tok)


def load(name):
    d = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(":")
            d[key.strip()] = [_num(t) for t in rest.split()]
    out = {"n_fields": d["n_fields"][0], "seg_bits": d["seg_bits"][0], "mode": d["mode"][0],
           "eb": float(d["eb"][0])}
    F = out["n_fields"]
    if "fill" in d:
        n, v = d["fill"]
        out["fields"] = np.full((F, int(n)), v, dtype=np.float32)
    else:
        out["fields"] = np.array([d["field%d" % f] for f in range(F)], dtype=np.float32)
    if "q0" in d:
        out["codes"] = np.array([d["q%d" % f] for f in range(F)], dtype=np.uint64).astype(np.uint32)
    for k in ("block_words", "stream_words", "perm"):
        if k in d:
            out[k] = np.array(d[k], dtype=np.uint64).astype(np.uint32)
    if "out0" in d:
        out["out"] = np.array([d["out%d" % f] for f in range(F)], dtype=np.float32)
    return out


def all_names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


def rn32(fr):
    """Round a rational to the nearest float32, ties to even (finite range)."""
    fr = Fraction(fr)
    # beyond FLT_MAX + half an ulp (2^128 - 2^103) the nearest is infinity
    if abs(fr) >= Fraction(2 ** 128 - 2 ** 103):
        return np.float32(np.inf if fr > 0 else -np.inf)
    c = np.float32(float(fr))
    lo = np.nextafter(c, np.float32(-np.inf))
    hi = np.nextafter(c, np.float32(np.inf))
    best = None
    for v in (lo, c, hi):
        if not np.isfinite(v):
            continue
        err = abs(Fraction(float(v)) - fr)
        even = (int(np.float32(v).view(np.uint32)) & 1) == 0
        key = (err, not even)
        if best is None or key < best[0]:
            best = (key, v)
    return np.float32(best[1])


def rd32(fr):
    """Largest float32 <= the rational fr."""
    fr = Fraction(fr)
    c = np.float32(float(fr))
    while Fraction(float(c)) > fr:
        c = np.nextafter(c, np.float32(-np.inf))
    while True:
        up = np.nextafter(c, np.float32(np.inf))
        if np.isfinite(up) and Fraction(float(up)) <= fr:
            c = up
        else:
            return np.float32(c)
