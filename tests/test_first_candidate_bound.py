"""The fast compression path skips the check of a block's first candidates
when first_candidate_exact() holds (csrc/gpz_qse_block.cuh): every code of the
block below 2^15 and ulp(max |x|) <= eb/512.  That is only sound if, under the
condition, the format's check (Section 4.1 quantisation with the step and
rounding used here: q = floor(RN(fma(RN(x - min), 1/s, 1/2))), then
|RN(x - RN(fma(q, s, min)))| <= ebchk) can never fail.

This test checks the claim with exact arithmetic over adversarial blocks that
satisfy the condition: values on and a few ulps around the midpoints between
lattice points, at the largest codes and magnitudes the condition allows.  A
control shows the test can fail: with the condition loosened (codes below
2^18, ulp(max |x|) <= eb/64), failures appear.  No GPU is involved; the CUDA path's parity tests then
compare whole streams with the oracle, which always checks."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def params(eb):
    """eb (double) -> RN32(eb), s = RN32(eb * 63/32), inv = RN32(1/s), ebchk = RD32(eb (1 - 2^-22))."""
    s = F32(eb * 1.96875)
    inv = F32(1.0 / float(s))
    t = eb * (1.0 - 2.0 ** -22)
    c = F32(t)
    if float(c) > t:
        c = np.nextafter(c, F32(-np.inf))
    return F32(eb), s, inv, c


def rn32_exact(a, b):
    """RN32(a + b) for float64 arrays a, b whose sum may not be exact in float64."""
    s = a + b
    bb = s - a
    err = (a - (s - bb)) + (b - bb)  # TwoSum: a + b == s + err exactly
    out = s.astype(np.float32)
    for i in np.nonzero(err != 0)[0]:  # rare: round the exact sum directly
        exact = Fraction(float(a[i])) + Fraction(float(b[i]))
        lo = np.float32(float(exact))
        cand = [lo, np.nextafter(lo, F32(-np.inf)), np.nextafter(lo, F32(np.inf))]
        out[i] = min(cand, key=lambda c: (abs(Fraction(float(c)) - exact), int(np.float32(c).view(np.uint32)) & 1))
    return out


def first_candidates_pass(x, mn, s, inv, ebchk):
    d = (x.astype(np.float64) - np.float64(mn)).astype(np.float32)  # exact difference, one rounding
    t = rn32_exact(d.astype(np.float64) * np.float64(inv), np.full(x.shape, 0.5))  # fma: exact product
    q = np.floor(t.astype(np.float64))
    xh = rn32_exact(q * np.float64(s), np.full(x.shape, np.float64(mn)))  # fma(q, s, min)
    diff = (x.astype(np.float64) - xh.astype(np.float64)).astype(np.float32)
    return np.abs(diff) <= ebchk


def ulp_of(M):
    """ulp of the float32 magnitude M as the CUDA predicate takes it: 2^(exponent - 23),
    at least the smallest subnormal."""
    if M == 0:
        return 2.0 ** -149
    return max(2.0 ** (int(np.frexp(F32(M))[1]) - 24), 2.0 ** -149)


def condition(x, mn, inv, eb32, max_bits=15, ulp_div=512):
    """The CUDA predicate, from the block's minimum and maximum."""
    mx = x.max()
    d = np.array([np.float64(F32(np.float64(mx) - np.float64(mn)))])
    tq = rn32_exact(d * np.float64(inv), np.array([0.5]))[0]
    bits = int(np.floor(float(tq))).bit_length()
    M = max(abs(float(mn)), abs(float(mx)))
    return bits <= max_bits and ulp_of(M) * ulp_div <= float(eb32)


def adversarial_block(rng, eb, k, ulp_div):
    eb32, s, inv, ebchk = params(eb)
    # the largest magnitude whose ulp the condition allows
    E = int(np.floor(np.log2(float(eb32) / ulp_div))) + 23
    M = 2.0 ** E * rng.uniform(1.0, 1.999)
    Q = min(2 ** k - 1, int(2 * M / float(s)) - 2)
    if Q < 2:
        return None
    lo = -M if rng.random() < 0.5 else rng.uniform(-M, M - Q * float(s))
    mn = F32(lo)
    j = rng.integers(0, Q, 1024)
    mid = np.float64(mn) + (j + 0.5) * np.float64(s)  # midpoints between lattice points
    x = mid.astype(np.float32).astype(np.float64)
    x = (x + rng.integers(-3, 4, 1024) * np.spacing(x.astype(np.float32)).astype(np.float64)).astype(np.float32)
    x[0] = mn
    x = np.clip(x, mn, F32(M))
    return x, mn, eb32, s, inv, ebchk


def run(trials, k_range, ulp_div, check_ulp_div, check_bits, seed):
    rng = np.random.default_rng(seed)
    tested = failed = 0
    for _ in range(trials):
        eb = 10.0 ** rng.uniform(-6, 2)
        k = int(rng.integers(*k_range))
        blk = adversarial_block(rng, eb, k, ulp_div)
        if blk is None:
            continue
        x, mn, eb32, s, inv, ebchk = blk
        if not condition(x, mn, inv, eb32, check_bits, check_ulp_div):
            continue
        tested += 1
        failed += int(not first_candidates_pass(x, mn, s, inv, ebchk).all())
    return tested, failed


def test_first_candidates_never_fail_under_the_condition():
    tested, failed = run(trials=1500, k_range=(10, 16), ulp_div=512, check_ulp_div=512, check_bits=15, seed=1)
    assert tested > 500
    assert failed == 0


def test_control_loosened_condition_fails():
    """With the condition loosened to codes below 2^18 and ulp(max |x|) <=
    eb/64, the first candidate does fail in some blocks (so the test above
    would notice a wrong bound)."""
    tested, failed = run(trials=400, k_range=(14, 18), ulp_div=64, check_ulp_div=64, check_bits=18, seed=2)
    assert tested > 100
    assert failed > 0
