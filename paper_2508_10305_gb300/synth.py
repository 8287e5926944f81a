"""Seeded synthetic particle data shaped like the paper's workloads.

The paper evaluates on six real datasets (Section 6, dataset table) that are
not available here; these generators stand in for them.  They hold no part
of the compression method: they only draw inputs, which the CUDA path and the
CPU oracle then both receive unchanged.

  uniform_box       -- n particles uniform in [0, 256)^3 (numpy, seed given)
  cosmology         -- halo mixture + uniform background, positions and
                       velocities (OuterRim / NewWorlds / LAMMPS-sized)
  lidar             -- airborne-LiDAR-like scan-order point cloud (USGS 3DEP-like)
  uniform_box_torch -- the same distribution drawn with torch (GPU or CPU)
  chunk_sizes       -- particle counts of the batched workload
  batched_workload  -- the batched workload: many chunks of 3 or 6 fields
  request_trace     -- the served workload's Poisson arrivals

The large generators use torch so that they can run on the GPU (fast) or
the CPU; for a given seed and device the output is deterministic.
"""
import math

import numpy as np
import torch

BOX = 256.0


def _below(x, hi):
    """Clamp float32 values into [.., hi) (rounding to float32 may reach hi)."""
    top = float(np.nextafter(np.float32(hi), np.float32(0)))
    return torch.clamp(x, max=top) if isinstance(x, torch.Tensor) else np.minimum(x, np.float32(top))


def uniform_box(n, seed=0, box=BOX):
    """[3, n] float32, uniform in [0, box)^3 (the small configuration)."""
    rng = np.random.default_rng(seed)
    x = (rng.random((3, n)) * box).astype(np.float32)
    return _below(x, box)


def cosmology(n, seed=2, n_halos=20000, halo_frac=0.7, device="cpu", box=BOX, sigma_v=300.0):
    """[6, n] float32: x, y, z, vx, vy, vz.

    20,000 Gaussian halos with centres uniform in the box, sigma log-uniform
    in [0.05, 2.0], masses from a power law dN/dM ~ M^-1.9 on [1, 1e5]; 70% of
    the particles are split among halos in proportion to mass (largest
    remainder), 30% are a uniform background.  Positions wrap periodically.
    Velocities are N(0, 300^2) per component plus the halo's bulk velocity
    (also N(0, 300^2) per component; 0 for the background).  Storage order:
    halos one after another in random order, then the background.
    """
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dev = torch.device(device)
    f64 = torch.float64
    u = torch.rand(n_halos, generator=g, device=dev, dtype=f64)
    a = 1.0 - 1.9
    m = (1.0 + u * (1e5 ** a - 1.0)) ** (1.0 / a)
    n_halo_total = int(round(halo_frac * n))
    share = m / m.sum() * n_halo_total
    counts = torch.floor(share).to(torch.int64)
    rest = n_halo_total - int(counts.sum())
    if rest > 0:
        order = torch.argsort(share - counts.to(f64), descending=True)
        counts[order[:rest]] += 1
    perm = torch.randperm(n_halos, generator=g, device=dev)
    counts = counts[perm]
    centres = torch.rand((n_halos, 3), generator=g, device=dev, dtype=f64) * box
    sig = torch.exp(torch.empty(n_halos, device=dev, dtype=f64).uniform_(math.log(0.05), math.log(2.0), generator=g))
    bulk = torch.randn((n_halos, 3), generator=g, device=dev, dtype=f64) * sigma_v
    hid = torch.repeat_interleave(torch.arange(n_halos, device=dev), counts)
    nh = hid.numel()
    out = torch.empty((6, n), dtype=torch.float32, device=dev)
    pos = centres[hid] + torch.randn((nh, 3), generator=g, device=dev, dtype=f64) * sig[hid, None]
    pos = torch.remainder(pos, box)
    out[:3, :nh] = _below(pos.t().to(torch.float32), box)
    vel = bulk[hid] + torch.randn((nh, 3), generator=g, device=dev, dtype=f64) * sigma_v
    out[3:, :nh] = vel.t().to(torch.float32)
    nb = n - nh
    out[:3, nh:] = _below((torch.rand((3, nb), generator=g, device=dev, dtype=f64) * box).to(torch.float32), box)
    out[3:, nh:] = (torch.randn((3, nb), generator=g, device=dev, dtype=f64) * sigma_v).to(torch.float32)
    return out


def lidar(n, seed=3, device="cpu", pts_per_line=20000, tile=10000.0):
    """[3, n] float32: x, y, z of an airborne scan in acquisition order.

    Boustrophedon lines along x, 1 m apart, 0.5 m point spacing along the line
    with U(-0.1, 0.1) m jitter on x and y; ground height z = sum of 8 random
    sinusoids (amplitude U[1, 50] m, wavelength U[500, 5000] m, random
    direction and phase) + N(0, 0.05^2) m; 5% of the points are vegetation
    returns raised by U[0, 30] m.
    """
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dev = torch.device(device)
    f64 = torch.float64
    amp = torch.empty(8, device=dev, dtype=f64).uniform_(1.0, 50.0, generator=g)
    lam = torch.empty(8, device=dev, dtype=f64).uniform_(500.0, 5000.0, generator=g)
    ang = torch.rand(8, generator=g, device=dev, dtype=f64) * (2 * math.pi)
    phase = torch.rand(8, generator=g, device=dev, dtype=f64) * (2 * math.pi)
    kx = 2 * math.pi * torch.cos(ang) / lam
    ky = 2 * math.pi * torch.sin(ang) / lam
    out = torch.empty((3, n), dtype=torch.float32, device=dev)
    step = 1 << 24
    for s in range(0, n, step):
        e = min(n, s + step)
        i = torch.arange(s, e, device=dev, dtype=torch.int64)
        line = i // pts_per_line
        k = i % pts_per_line
        k = torch.where(line % 2 == 0, k, pts_per_line - 1 - k)
        x = k.to(f64) * 0.5 + torch.empty(e - s, device=dev, dtype=f64).uniform_(-0.1, 0.1, generator=g)
        y = (line % int(tile)).to(f64) * 1.0 + torch.empty(e - s, device=dev, dtype=f64).uniform_(-0.1, 0.1, generator=g)
        z = torch.zeros(e - s, device=dev, dtype=f64)
        for q in range(8):
            z += amp[q] * torch.sin(kx[q] * x + ky[q] * y + phase[q])
        z += torch.randn(e - s, generator=g, device=dev, dtype=f64) * 0.05
        veg = torch.rand(e - s, generator=g, device=dev, dtype=f64) < 0.05
        z += torch.where(veg, torch.rand(e - s, generator=g, device=dev, dtype=f64) * 30.0, torch.zeros_like(z))
        out[0, s:e] = x.to(torch.float32)
        out[1, s:e] = y.to(torch.float32)
        out[2, s:e] = z.to(torch.float32)
    return out


def uniform_box_torch(n, seed=0, device="cpu", box=BOX):
    """[3, n] float32 uniform in [0, box)^3, drawn with torch (fast on a GPU)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.rand((3, n), generator=g, device=torch.device(device), dtype=torch.float64) * box
    return _below(x.to(torch.float32), box)


def chunk_sizes(n_chunks=4096, lo=10_000, hi=4_000_000, seed=4):
    """Particle counts log-uniform in [lo, hi] (the batched workload)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n_chunks)).astype(np.int64)


class BatchedWorkload:
    """Chunks held in two pools (one per field count), each chunk's fields
    starting on a 128-byte boundary."""

    def __init__(self, n, F, rel, pools, offsets):
        self.n, self.F, self.rel = [int(v) for v in n], [int(v) for v in F], [float(v) for v in rel]
        self.pools, self.offsets = pools, [int(v) for v in offsets]
        self.count = len(self.n)

    def fields(self, c):
        pool, o, n = self.pools[self.F[c]], self.offsets[c], self.n[c]
        return [pool[f, o:o + n] for f in range(self.F[c])]

    def input_bytes(self):
        return sum(4 * n * F for n, F in zip(self.n, self.F))


def batched_workload(n_chunks=4096, lo=10_000, hi=4_000_000, seed=4, device="cpu"):
    """The batched workload: n_chunks chunks with log-uniform particle counts
    in [lo, hi]; each has 3 fields drawn like the small configuration (uniform
    box) or 6 drawn like the cosmology snapshot (its halo count scaled to keep
    the snapshot's particles per halo), with equal odds, and a relative error
    bound 1e-3 or 1e-4, with equal odds.  Chunk c is seeded 1000 + c."""
    n = chunk_sizes(n_chunks, lo, hi, seed)
    rng = np.random.default_rng(seed + 1)
    F = rng.choice([3, 6], n_chunks)
    rel = rng.choice([1e-3, 1e-4], n_chunks)
    pad = [int(-(-int(v) // 32) * 32) for v in n]
    offsets = np.zeros(n_chunks, dtype=np.int64)
    pools = {}
    for ff in (3, 6):
        idx = [c for c in range(n_chunks) if F[c] == ff]
        total = sum(pad[c] for c in idx)
        pool = torch.empty((ff, max(total, 32)), dtype=torch.float32, device=torch.device(device))
        o = 0
        for c in idx:
            offsets[c] = o
            if ff == 3:
                pool[:, o:o + n[c]] = uniform_box_torch(int(n[c]), seed=1000 + c, device=device)
            else:
                halos = max(4, int(round(20000 * int(n[c]) / 2 ** 26)))
                pool[:, o:o + n[c]] = cosmology(int(n[c]), seed=1000 + c, n_halos=halos, device=device)
            o += pad[c]
        pools[ff] = pool
    return BatchedWorkload(n, F, rel, pools, offsets)


def request_trace(n_requests=20000, rate=2000.0, lo=100_000, hi=64_000_000, seed=5):
    """Poisson arrivals (seconds), sizes log-uniform in [lo, hi], generator id
    in {0: uniform box, 1: cosmology, 2: lidar}, op in {0: compress, 1: decompress}."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    size = np.exp(rng.uniform(np.log(lo), np.log(hi), n_requests)).astype(np.int64)
    gen = rng.integers(0, 3, n_requests)
    op = rng.integers(0, 2, n_requests)
    return t, size, gen, op
