"""The block-size sweep (Section 4.2's trade-off, on the three single-array
workloads) -- TEST INFRASTRUCTURE: it runs only the oracle, on the seeded
synthetic inputs of paper_2508_10305_gb300.synth, and prints a markdown
table of, per workload and block size B in {256, 512, 1024, 2048}: the
compression ratio, bits per value, PSNR, max |error| / eb and the oracle's
own throughput (compress + decompress over all host threads by ranges of
whole blocks; a CPU figure, not the GPU library's, which writes B = 1024).

    python oracle/block_size_sweep.py [--quick]

Relative bounds are taken over the whole array once and passed as absolute
bounds, so that every block is encoded as in one call on the whole array.
"""
import argparse
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import gpz_oracle  # noqa: E402

SIZES = (256, 512, 1024, 2048)


def absolute_bounds(x, eb, rel):
    if not rel:
        return [eb] * x.shape[0]
    out = []
    for f in range(x.shape[0]):
        v = x[f][~np.isnan(x[f])]
        rng = float(v.max()) - float(v.min()) if v.size else 0.0
        e = eb * rng
        out.append(e if (0.0 < rng < float("inf") and 0.0 < e < float("inf")) else eb)
    return out


def run(x, ebs, G, B, threads):
    """Whole-array stream size, PSNR, max error / eb, and the seconds of the
    oracle's compress + decompress (the checks are not timed)."""
    F, n = x.shape
    nb = (n + B - 1) // B
    cuts = sorted(set(min(n, (nb * k // threads) * B) for k in range(threads + 1)))
    parts = [np.ascontiguousarray(x[:, cuts[k]:cuts[k + 1]]) for k in range(len(cuts) - 1)]

    def work(part):
        s, p = gpz_oracle.compress(part, ebs, 0, G, want_perm=True, block=B)
        out = gpz_oracle.decompress(s, F, part.shape[1], any_block=True)
        return s, p, out

    t0 = time.perf_counter()
    with ThreadPoolExecutor(len(parts)) as ex:
        res = list(ex.map(work, parts))
    dt = time.perf_counter() - t0
    payload, sq, worst = 0, np.zeros(F), 0.0
    for part, (s, p, out) in zip(parts, res):
        nbk = (part.shape[1] + B - 1) // B
        payload += s.size // 4 - (16 + 2 * F + nbk + 1)
        d = part[:, p].astype(np.float64) - out.astype(np.float64)
        sq += (d * d).sum(axis=1)
        worst = max(worst, float((np.abs(d).max(axis=1) / np.asarray(ebs)).max()))
    size = 4 * (16 + 2 * F + nb + 1 + payload)
    rmse = np.sqrt(sq / n)
    rng = x.max(axis=1).astype(np.float64) - x.min(axis=1).astype(np.float64)
    nrmse = np.sqrt(np.mean((rmse / rng) ** 2))
    return size, -20.0 * np.log10(nrmse), worst, dt


def workloads(quick):
    """The generators run where the benchmark runs them (on the GPU when there
    is one: the CPU and CUDA random streams differ), so that at B = 1024 the
    ratios equal the benchmark's."""
    import torch
    from paper_2508_10305_gb300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    n2 = (1 << 22) if quick else (1 << 26)
    n3 = 20_000_000 if quick else 200_000_000
    return [
        ("uniform 1e6 x 3, abs 1e-2", lambda: synth.uniform_box(1_000_000, seed=0), 1e-2, False),
        ("cosmology %s x 6, rel 1e-4" % ("2^22" if quick else "2^26"),
         lambda: synth.cosmology(n2, seed=2, device=dev).cpu().numpy(), 1e-4, True),
        ("LiDAR %.0e x 3, abs 1e-3 m" % n3, lambda: synth.lidar(n3, seed=3, device=dev).cpu().numpy(), 1e-3, False),
    ]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="smaller cosmology and LiDAR arrays")
    ap.add_argument("--G", type=int, default=3)
    args = ap.parse_args()
    gpz_oracle.lib()
    threads = os.cpu_count() or 1
    print("| workload | B | ratio | bits/value | PSNR dB | max err / eb | oracle GB/s (%d host threads) |" % threads)
    print("|---|---|---|---|---|---|---|")
    for name, make, eb, rel in workloads(args.quick):
        x = make()
        x = np.ascontiguousarray(x, dtype=np.float32)
        ebs = absolute_bounds(x, eb, rel)
        for B in SIZES:
            size, psnr, worst, dt = run(x, ebs, args.G, B, threads)
            print("| %s | %d | %.3f | %.3f | %.1f | %.4f | %.3f |" % (
                name, B, x.nbytes / size, 8.0 * size / x.size, psnr, worst, x.nbytes / dt / 1e9), flush=True)
        del x


if __name__ == "__main__":
    main()
