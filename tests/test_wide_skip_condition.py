"""The 64-bit block kernel skips the check of first candidates for a field of
a block when eb >= 2^-1000, the block's value range is at most 2^40 steps
(rounded up) and max |x| <= 2^45 eb.  The stream stays the oracle's only if
no first candidate can fail under that condition.  This stress test draws
adversarial blocks inside the condition -- values on and around the
half-steps between lattice points, magnitudes up to the limit, bounds from
2^-1000 to 2^900 -- and counts failing first candidates with the oracle's own
arithmetic: there must be none.  Blocks far outside the condition do fail,
which shows the probe can see a failure."""
import numpy as np

STEP_PER_EB = 1.96875


def condition(lo, hi, eb):
    """The kernel's test, with the range rounded up conservatively."""
    s = eb * STEP_PER_EB
    rng_up = np.nextafter(hi - lo, np.inf)
    return eb >= 2.0 ** -1000 and rng_up <= s * 2.0 ** 40 and max(abs(lo), abs(hi)) <= eb * 2.0 ** 45


def adversarial_block(rng, eb, n=1024):
    s = eb * STEP_PER_EB
    limit = eb * 2.0 ** 45
    width = s * 2.0 ** 40 * rng.uniform(0.5, 1.0)  # up to the range limit
    kind = rng.integers(0, 3)
    if kind == 0:  # near the magnitude limit
        lo = (limit - width) * rng.choice([-1.0, 1.0]) if rng.random() < 0.5 else limit - width
        lo = min(lo, limit - width)
    elif kind == 1:  # straddling zero
        lo = -width * rng.uniform(0.0, 1.0)
    else:
        lo = rng.uniform(-limit, limit - width)
    k = np.floor(rng.random(n) * (width / s - 1.0))
    x = lo + (k + 0.5) * s  # half-steps (rounded to the nearest double)
    # a few ulps either side of them
    for _ in range(3):
        m = rng.random(n) < 0.3
        x[m] = np.nextafter(x[m], np.where(rng.random(m.sum()) < 0.5, -np.inf, np.inf))
    x[0] = lo
    return x


def test_first_candidates_pass_inside_the_condition(oracle):
    rng = np.random.default_rng(2025)
    tested = 0
    for _ in range(3000):
        eb = 2.0 ** rng.uniform(-1000, 900)
        x = adversarial_block(rng, eb)
        lo, hi = float(x.min()), float(x.max())
        if not (np.all(np.isfinite(x)) and condition(lo, hi, eb)):
            continue
        mn = 0.0 if lo == 0.0 else lo
        assert oracle.wide_first_candidate_failures(x, mn, eb) == 0, (eb, lo, hi)
        tested += 1
    assert tested > 2000


def test_probe_sees_failures_outside_the_condition(oracle):
    """At |x| near 2^53 eb (256 times the limit) an ulp of x is about eb, and
    half-steps start to fail: the margin of the condition is wide."""
    rng = np.random.default_rng(7)
    eb = 3e-6
    s = eb * STEP_PER_EB
    lo = eb * 2.0 ** 53
    x = lo + (np.floor(rng.random(4096) * 100000) + 0.5) * s
    assert not condition(float(x.min()), float(x.max()), eb)
    assert oracle.wide_first_candidate_failures(x, float(x.min()), eb) > 0
