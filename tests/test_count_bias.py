"""What a -1 bias on the run-length code would save (Section 4.3).

Section 4.3 stores each run's id difference and its particle count without
saying whether they are biased.  The stream keeps them literal (delta_0 = u_0,
delta_k = u_k - u_(k-1), counts c_k >= 1).  Every delta after the first and
every count is at least 1, so storing delta_k - 1 and c_k - 1 could narrow
the fixed-length widths by one bit in some blocks.  These tests measure,
from the oracle's per-block stages alone, how many bits that would save on
the synthetic workloads, and pin that the literal form costs well under
half a percent of the stream.  Run as a script, the module prints the table
of savings."""
import numpy as np
import pytest

from oracle import gpz_oracle as O
from paper_2508_10305_gb300 import synth

B = 1024


def _bitwidth(v):
    return int(v).bit_length()


def bias_saving(x, eb, mode, G, max_blocks=None):
    """(bits saved by the bias over the sampled blocks scaled to the whole
    array, stream bits, sampled blocks whose widths shrink)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    F, n = x.shape
    stream, _ = O.compress(x, eb, mode, G, want_perm=False)
    params = [O.params_rel(eb, x[f]) for f in range(F)] if mode == 1 else [O.params_abs(eb)] * F
    nblocks = (n + B - 1) // B
    blocks = np.arange(nblocks) if max_blocks is None else np.unique(
        np.linspace(0, nblocks - 1, max_blocks).astype(int))
    saved = shrunk = 0
    for b in blocks:
        st = O.block_stages(x[:, b * B:min(n, b * B + B)], G, params)
        if st["raw"]:
            continue
        u = st["uniq"].astype(np.int64)
        c = st["counts"].astype(np.int64)
        d = np.diff(u, prepend=0)
        # the run-length code's invariants, which make the bias lossless
        assert c.min() >= 1 and c.sum() == min(B, n - b * B)
        assert (d[1:] >= 1).all()
        d_biased = d.copy()
        d_biased[1:] -= 1
        wd, wc = _bitwidth(d.max()), _bitwidth(c.max())
        wd_b, wc_b = _bitwidth(d_biased.max()), _bitwidth((c - 1).max())
        assert wd_b <= wd and wc_b <= wc and wd - wd_b <= 1 and wc - wc_b <= 1
        saved += len(u) * ((wd - wd_b) + (wc - wc_b))
        shrunk += (wd_b < wd) or (wc_b < wc)
    return saved * nblocks / len(blocks), 8 * stream.size, shrunk


CASES = [
    # name, generator, bound, mode, G, sampled blocks (None: all)
    ("uniform 1e6 x 3", lambda: synth.uniform_box(1_000_000, seed=0), 1e-2, 0, 3, None),
    ("uniform 1e6 x 3", lambda: synth.uniform_box(1_000_000, seed=0), 1e-2, 0, 2, 200),
    ("cosmology 2^20 x 6", lambda: np.asarray(synth.cosmology(1 << 20, seed=2)), 1e-4, 1, 3, 300),
    ("LiDAR 2^20 x 3", lambda: np.asarray(synth.lidar(1 << 20, seed=3)), 1e-3, 0, 3, 300),
    ("LiDAR 2^20 x 3", lambda: np.asarray(synth.lidar(1 << 20, seed=3)), 1e-3, 0, 0, 300),
]


@pytest.mark.parametrize("name,gen,eb,mode,G,sample", CASES)
def test_literal_run_code_costs_under_half_a_percent(name, gen, eb, mode, G, sample):
    saved, stream_bits, _ = bias_saving(gen(), eb, mode, G, sample)
    assert 0 <= saved < 0.005 * stream_bits


def test_bias_saves_one_count_bit_in_single_run_blocks():
    """G = 0: one run per block holding all 1,024 particles, count 1024 needs
    11 bits and 1023 needs 10, so exactly one bit per full block."""
    x = synth.uniform_box(8 * B, seed=1)
    saved, _, shrunk = bias_saving(x, 1e-2, 0, 0)
    assert saved == 8 and shrunk == 8


if __name__ == "__main__":
    for name, gen, eb, mode, G, sample in CASES:
        saved, stream_bits, shrunk = bias_saving(gen(), eb, mode, G, sample)
        print("%-20s eb %-7g G %d: saves %8.0f bytes of %9d (%.3f%%), widths shrink in %d sampled blocks"
              % (name, eb, G, saved / 8, stream_bits // 8, 100 * saved / stream_bits, shrunk))
