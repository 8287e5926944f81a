"""GPZ on GB300: compress + decompress throughput on the cosmology-like
snapshot (2^26 particles x 6 fp32 fields, relative error bound 1e-4 of each
field's range, segment bits G = 3).

A step is one round trip through the whole hot path: gpz_compress (range
pass, fused quantise/sort/encode, look-back scan, compaction) then
gpz_decompress, with the input already resident in HBM.  The metric is GB/s
of input per round trip: 4*n*F bytes / (compress time + decompress time),
summed over ranks (weak scaling: every rank compresses its own snapshot; no
collective touches the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line on rank 0.  Besides the headline it carries, each measured in
the same run on the same GPU:
  - compress_roofline / decompress_roofline: the algorithmic bytes of each
    direction (input read by the range pass and by the fused kernel, stream
    written; stream read, output written) over its time, against the measured
    copy bandwidth and the nominal 8 TB/s;
  - e2e: the same round trip through the C ABI with the input and output in
    pinned host memory (uploads, downloads and the stream's trip to the host
    and back inside the timed region), pipelined over two buffer sets with no
    host synchronisation, plus the sequential form and the form in which each
    call allocates its workspace (the paper's end-to-end accounting);
  - small / lidar: the 1e6 x 3 uniform and 2e8 x 3 LiDAR-like workloads;
  - batched: 4,096 uneven chunks through the batched plans (graphs, tuned
    shapes) against one call per chunk;
  - served: Poisson request traces against the serving engine and the plain
    path, at 2,000 requests/s and at a rate neither keeps up with;
  - variants: fused compaction, interleaved records, fp64 input, 64-bit
    intermediates.
The reference arm (--impl reference) times the plain CPU oracle on the
box's host cores on bounded samples of the same workload.

    python bench.py --workload batched|served|sweep

measures one of those forms alone, with its own options (see --help).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Compress+decompress GB/s (% HBM roofline) and ratio; served p50/p99 vs plain"
N_PARTICLES = 1 << 26
N_FIELDS = 6
REL_EB = 1e-4
SEG_BITS = 3
SEED = 2
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal
WORKLOAD = "cosmology-like snapshot: 2^26 particles x 6 fp32 (x,y,z,vx,vy,vz), 20,000 halos + 30% background, relative eb 1e-4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpz", choices=["gpz", "reference"])
    ap.add_argument("--n", type=int, default=N_PARTICLES, help="particles (profiling runs only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused-compaction comparison")
    ap.add_argument("--no-aos", action="store_true", help="skip the interleaved-records round trip")
    ap.add_argument("--no-f64", action="store_true", help="skip the fp64 round trip")
    ap.add_argument("--no-wide", action="store_true", help="skip the 64-bit-intermediate round trip")
    ap.add_argument("--no-small", action="store_true", help="skip the 1e6 x 3 uniform workload")
    ap.add_argument("--no-lidar", action="store_true", help="skip the 2e8 x 3 LiDAR-like workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-served", action="store_true", help="skip the served workload")
    ap.add_argument("--workload", default="cosmology", choices=["cosmology", "batched", "served", "sweep"])
    ap.add_argument("--requests", type=int, default=4000, help="served workload: requests per arm")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="served workload: admission budget")
    ap.add_argument("--rate", type=float, default=2000.0, help="served workload: requests per second")
    ap.add_argument("--sat-rate", type=float, default=20000.0,
                    help="served workload: the rate of the saturating comparison (above either arm's capacity)")
    ap.add_argument("--sat-requests", type=int, default=2000, help="served workload: requests of the saturating runs")
    ap.add_argument("--serve-arms", default="batched:2:64:256:64,plain:1:1:0:0",
                    help="served workload: arms name:lanes:max_batch:max_batch_MB:express_lane_MB; the first is "
                         "the served arm, 'plain' the comparison")
    ap.add_argument("--chunks", type=int, default=4096, help="batched workload: number of chunks")
    ap.add_argument("--chunk-lo", type=int, default=10_000)
    ap.add_argument("--chunk-hi", type=int, default=4_000_000)
    ap.add_argument("--batched-steps", type=int, default=10, help="batched workload in the default run: timed steps")
    ap.add_argument("--batched-only", action="store_true",
                    help="batched workload: time the plans with their default shapes only (profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- measurement helpers

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel):
    """Per-launch DRAM bytes from the committed ncu summary of `kernel`, or
    None when any source the kernel is built from changed since the counters
    were taken (the summary lists the files and their sha256)."""
    path = os.path.join(ROOT, "profiles", "traffic_%s.txt" % kernel)
    if not os.path.exists(path):
        return None
    info, hashes = {}, {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k.startswith("sha256 "):
                hashes[k[len("sha256 "):]] = v
            else:
                info[k] = v
    if not hashes:
        return None
    for name, digest in hashes.items():
        src = os.path.join(ROOT, "paper_2508_10305_gb300", "csrc", name)
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != digest:
            return None
    try:
        return float(info["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.lines = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            ident = ["-i", "GPU-" + uuid if not uuid.startswith("GPU-") else uuid]
        except Exception:
            ident = []
        self.cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"] + ident

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ranks

def ranks_max(values, device):
    """Element-wise max of a list of floats over the ranks of the default
    process group; the values themselves when there is one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_gbs(world, bytes_per_rank_step, steps, seconds):
    """Whole-job GB/s of input: each rank processes its own snapshot every step
    (replicas, weak scaling) and the job lasts as long as the slowest rank."""
    return world * bytes_per_rank_step * steps / seconds / 1e9


def r4(v):
    """Round for the JSON line (keeps it short enough for the driver's record)."""
    return None if v is None else float("%.4g" % v)


# ----------------------------------------------------------------------------- workload

def make_workload(n, rank, device):
    from paper_2508_10305_gb300 import synth
    return synth.cosmology(n, seed=SEED + rank, device=device)


def psnr_and_error(x, out, perm, ebs):
    """Aggregate PSNR (Section 3.1: NRMSE per field, then -20 log10 of the
    root mean square) and max |x - x_hat| / eb, on the device in double."""
    import torch
    nrmse2, worst = [], 0.0
    for f in range(x.shape[0]):
        xs = x[f][perm].double()
        d = xs - out[f].double()
        rng = (xs.max() - xs.min()).item()
        rmse = torch.sqrt(torch.mean(d * d)).item()
        nrmse2.append((rmse / rng) ** 2 if rng > 0 else 0.0)
        worst = max(worst, d.abs().max().item() / ebs[f])
    psnr = -20.0 * np.log10(np.sqrt(np.mean(nrmse2))) if np.mean(nrmse2) > 0 else float("inf")
    return psnr, worst


def absolute_bounds(x_host, rel):
    """Each field's absolute bound for a relative bound over the whole array,
    exactly as the oracle's relative mode computes it (rel times the double
    range of the non-NaN values; rel itself when that is not a finite
    positive number)."""
    out = []
    for f in range(x_host.shape[0]):
        v = x_host[f][~np.isnan(x_host[f])]
        rng = float(v.max()) - float(v.min()) if v.size else 0.0
        e = rel * rng
        out.append(e if (0.0 < rng < float("inf") and 0.0 < e < float("inf")) else rel)
    return out


def cpu_oracle_sample(x_host_blocks, n_fields, ebs):
    """Time the CPU oracle (single thread) on a host sample with absolute
    bounds ebs; returns GB/s of input per round trip and the two times."""
    from oracle import gpz_oracle
    gpz_oracle.lib()
    t0 = time.perf_counter()
    stream, _ = gpz_oracle.compress(x_host_blocks, ebs, 0, SEG_BITS, want_perm=False)
    t1 = time.perf_counter()
    gpz_oracle.decompress(stream, n_fields, x_host_blocks.shape[1])
    t2 = time.perf_counter()
    return x_host_blocks.nbytes / (t2 - t0) / 1e9, t1 - t0, t2 - t1


def cpu_oracle_threads(x_host, n_fields, threads, ebs):
    """The oracle, unchanged, over `threads` host threads: each compresses and
    then decompresses a contiguous range of whole blocks (blocks are
    independent) with the absolute bounds ebs, so that every block is
    encoded as in one call on the whole array.  ctypes releases the
    interpreter lock during the C calls.  Returns (GB/s of input per round
    trip, wall seconds, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import gpz_oracle
    gpz_oracle.lib()
    F, n = x_host.shape
    nb = (n + 1023) // 1024
    cuts = [min(n, (nb * k // threads) * 1024) for k in range(threads + 1)]
    parts = [np.ascontiguousarray(x_host[:, cuts[k]:cuts[k + 1]]) for k in range(threads) if cuts[k + 1] > cuts[k]]

    def work(part):
        stream, _ = gpz_oracle.compress(part, ebs, 0, SEG_BITS, want_perm=False)
        gpz_oracle.decompress(stream, n_fields, part.shape[1])

    with ThreadPoolExecutor(len(parts)) as ex:
        t0 = time.perf_counter()
        list(ex.map(work, parts))
        dt = time.perf_counter() - t0
    return x_host.nbytes / dt / 1e9, dt, len(parts)


def host_blocks(x_dev, blocks):
    """The given 1024-particle blocks of the device workload, on the host."""
    import torch
    idx = torch.as_tensor(blocks, device=x_dev.device)
    sel = (idx[:, None] * 1024 + torch.arange(1024, device=x_dev.device)[None, :]).reshape(-1)
    return x_dev[:, sel].cpu().numpy()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host's cores (one thread per core,
    each on a contiguous range of whole blocks), on the GPU arm's workload,
    metric, unit and config.  The relative bound is turned into each field's
    absolute bound over the whole snapshot once, so that every sampled block
    is encoded exactly as in the GPU arm's stream.  Each step is a bounded
    sample of whole 1024-particle blocks spread over the snapshot (rotating
    offset), sized so that all steps together take about 90 s of single-core
    work per core."""
    if rank != 0:
        return
    import torch
    from paper_2508_10305_gb300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    x = synth.cosmology(args.n, seed=SEED, device=dev)
    ebs = absolute_bounds(x.cpu().numpy(), REL_EB)
    nb = args.n // 1024
    nthreads = os.cpu_count() or 1
    per_step = int(max(8 * nthreads, min(nb, nthreads * 90.0 * 1.4e6 / max(1, args.steps) / 1024)))
    stride = max(1, nb // per_step)

    def sample(i):
        return host_blocks(x, np.arange(i % stride, nb, stride)[:per_step])

    for i in range(args.warmup):
        cpu_oracle_threads(sample(i)[:, :nthreads << 14], N_FIELDS, nthreads, ebs)
    total, nbytes, used = 0.0, 0, 1
    for i in range(args.steps):
        s = sample(i)
        _, dt, used = cpu_oracle_threads(s, N_FIELDS, nthreads, ebs)
        total += dt
        nbytes += s.nbytes
    value = nbytes / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": gpu_config(args.n, 1),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": used, "kind": "oracle",
                         "sample": "per step %d whole 1024-particle blocks (every %dth, rotating offset) x 6 "
                                   "fields; C++ oracle compress + decompress over %d host threads by block "
                                   "range; absolute bounds from the relative bound over the whole snapshot, so "
                                   "the blocks are encoded as in the GPU arm's stream" % (per_step, stride, used)},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gpu_config(n, world):
    in_bytes = 4.0 * n * N_FIELDS
    return {"workload": WORKLOAD, "n": n, "fields": N_FIELDS, "eb_mode": "rel", "eb": REL_EB,
            "seg_bits": SEG_BITS, "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs (%.2f GB) larger than L2 (129 MB); no flush" % (in_bytes / 1e9)}


# ----------------------------------------------------------------------------- GPU arm: one workload's round trip

COMPRESS_STAGES = ("range", "info", "qse", "scan", "compact")


def round_trip(gpz, x, eb, mode, steps, warmup, stream, dev, world=1, clocks_index=None):
    """Time `steps` round trips (gpz_compress, then gpz_decompress of its
    stream) of the [F, n] device array x, after `warmup`, with CUDA events on
    the launching stream; the input is resident in HBM.  Returns a dict with
    the round-trip time, the per-stage kernel times (stage events on the same
    stream), the stream size, ratio, PSNR and max |error| / eb, the decoded
    output and the compressor (for the callers that reuse them)."""
    import torch
    F, n = x.shape
    fields = [x[f] for f in range(F)]
    comp = gpz.Compressor(n, F, eb, mode, SEG_BITS, want_perm=False, device=dev)
    dec = gpz.Decompressor(n, F, device=dev)
    # one checked round trip with the permutation: ratio, PSNR, error bound
    chk = gpz.Compressor(n, F, eb, mode, SEG_BITS, want_perm=True, device=dev)
    size = chk(fields)
    out = dec(chk.out, size)
    perm = chk.perm[:n].long()
    hdr = chk.out[:4 * (16 + 2 * F)].cpu().numpy().view(np.uint32)
    ebs = [float(hdr[16 + 2 * f].view(np.float32)) for f in range(F)]
    psnr, worst = psnr_and_error(x, out, perm, ebs)
    out_host = out.cpu()
    del chk, perm, out
    torch.cuda.empty_cache()

    def step():
        comp(fields, stream, sync=False)
        dec(comp.out, size, stream, check=False)

    # the clock sampler starts before the warm-up, so that starting it does
    # not delay the first launches of the timed region; it samples until the
    # timed region ends
    clk = ClockSampler(clocks_index) if clocks_index is not None else None
    if clk:
        clk.__enter__()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    for ws in (comp.ws, dec.ws):
        st = gpz.gpz_sync_status(ws)
        if st != gpz.OK:
            raise gpz.GpzError(st, "warm-up")
    gpz.gpz_launch_count(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    import torch.distributed as dist
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    if world > 1:
        dist.barrier()
    launches = gpz.gpz_launch_count()
    for ws in (comp.ws, dec.ws):
        st = gpz.gpz_sync_status(ws)
        if st != gpz.OK:
            raise gpz.GpzError(st, "timed region")
    ms = ranks_max([ev0.elapsed_time(ev1) / steps], dev)[0]
    # per-kernel times: a separate pass with an event after every kernel (the
    # timed region above records none)
    kreps = max(1, min(steps, 50))
    gpz.gpz_set_stage_timing(True, stream)
    gpz.gpz_stage_times()  # clear
    for _ in range(kreps):
        step()
    torch.cuda.synchronize()
    stages = gpz.gpz_stage_times(16)
    gpz.gpz_set_stage_timing(False, stream)
    comp_ms = sum(stages[k][0] for k in COMPRESS_STAGES if k in stages) / kreps
    dec_ms = stages.get("decompress", (0.0, 1))[0] / kreps
    return {"ms": ms, "comp_ms": comp_ms, "dec_ms": dec_ms, "stages": stages, "steps": steps, "kreps": kreps,
            "size": size,
            "ratio": x.numel() * 4.0 / size, "psnr": psnr, "worst": worst, "launches": launches,
            "clocks": clk.summary() if clk else None, "comp": comp, "dec": dec, "out_host": out_host,
            "in_bytes": 4.0 * n * F, "rel": mode == gpz.EB_REL}


def direction_rooflines(rt, peak, peak_kind):
    """Compression and decompression each against the HBM roofline, in the
    algorithmic bytes of each direction: compression reads the input once
    per pass that needs it (the range pass with a relative bound, then the
    fused kernel) and writes the stream; decompression reads the stream and
    writes the output.  Temporary slots, offsets and tables are
    implementation bytes and are not counted."""
    inb, size = rt["in_bytes"], float(rt["size"])
    cb = (2.0 if rt["rel"] else 1.0) * inb + size
    db = size + inb
    out = []
    for b, ms in ((cb, rt["comp_ms"]), (db, rt["dec_ms"])):
        ach = b / (ms / 1e3) / 1e9 if ms else None
        out.append({"bytes": int(b), "ms": r4(ms), "achieved_gbs": r4(ach), "frac": r4(ach / peak) if ach else None,
                    "frac_of_nominal": r4(ach / NOMINAL_HBM_GBS) if ach else None,
                    "peak": peak, "peak_source": peak_kind})
    out[0]["bytes_counted"] = ("input read by the range pass and by the fused kernel, stream written" if rt["rel"]
                               else "input read by the fused kernel, stream written")
    out[1]["bytes_counted"] = "stream read, output written"
    return out


def workload_summary(rt, peak, peak_kind, name, n, F, eb, mode_name):
    """A compact sub-object for a secondary workload of the default line."""
    cr, dr = direction_rooflines(rt, peak, peak_kind)
    return {"workload": name, "n": n, "fields": F, "eb_mode": mode_name, "eb": eb,
            "value": r4(rt["in_bytes"] / (rt["ms"] / 1e3) / 1e9), "unit": "GB/s", "ms_per_step": r4(rt["ms"]),
            "compress_gbs": r4(rt["in_bytes"] / rt["comp_ms"] / 1e6) if rt["comp_ms"] else None,
            "decompress_gbs": r4(rt["in_bytes"] / rt["dec_ms"] / 1e6) if rt["dec_ms"] else None,
            "compress_frac": cr["frac"], "decompress_frac": dr["frac"],
            "ratio": r4(rt["ratio"]), "psnr_db": r4(rt["psnr"]), "max_err_over_eb": r4(rt["worst"])}


# ----------------------------------------------------------------------------- GPU arm: end to end

def e2e_measure(gpz, x, out_ref_host, steps, dev, world):
    """The round trip through the C ABI with host buffers: every step uploads
    the input from pinned host memory, compresses, moves the stream to pinned
    host memory and back (gpz_copy_stream, sized on the device), decompresses
    and downloads the output.  Three forms:
      - pipelined (the value): two buffer sets, copies and kernels on four
        streams (input uploads and output downloads on the copy engines, the
        stream's trips by SM copies, the kernels), ordered only by events, so
        that step i+1's upload overlaps step i's kernels and downloads; the
        host never waits inside the timed region;
      - sequential: the same work on one stream, one step after another;
      - with_alloc: sequential, each gpz_compress / gpz_decompress given no
        workspace, so that it allocates and frees its own (the paper's
        end-to-end accounting, Section 6)."""
    import torch
    F, n = x.shape
    in_bytes = 4.0 * n * F
    h_in = torch.empty((F, n), dtype=torch.float32, pin_memory=True)
    h_in.copy_(x)
    k = max(3, steps)
    sets = []
    for j in range(2):
        c_ = gpz.Compressor(n, F, REL_EB, gpz.EB_REL, SEG_BITS, want_perm=False, device=dev)
        sets.append({"comp": c_, "dec": gpz.Decompressor(n, F, device=dev), "d_in": torch.empty_like(x),
                     "d_stream": torch.empty_like(c_.out),
                     "h_stream": torch.empty(c_.capacity, dtype=torch.uint8, pin_memory=True),
                     "h_out": torch.empty((F, n), dtype=torch.float32, pin_memory=True),
                     "h_size": torch.zeros(1, dtype=torch.int64, pin_memory=True)})
    cap = sets[0]["comp"].capacity
    s_up, s_run, s_sm, s_down = (torch.cuda.Stream(dev) for _ in range(4))
    ev = [{name: torch.cuda.Event() for name in ("in_ready", "in_free", "compressed", "stream_up", "decoded",
                                                 "out_down")} for _ in range(2)]
    for e in ev:  # nothing to wait for at the start
        for name in ("in_free", "stream_up", "decoded", "out_down"):
            e[name].record(s_run)

    def pipelined_step(i):
        b, e = sets[i % 2], ev[i % 2]
        s_up.wait_event(e["in_free"])
        with torch.cuda.stream(s_up):
            b["d_in"].copy_(h_in, non_blocking=True)
        e["in_ready"].record(s_up)
        s_run.wait_event(e["in_ready"])
        s_run.wait_event(e["stream_up"])  # the previous use of this set's stream buffers is done
        b["comp"]([b["d_in"][f] for f in range(F)], s_run, sync=False)
        e["in_free"].record(s_run)
        e["compressed"].record(s_run)
        s_sm.wait_event(e["compressed"])
        s_sm.wait_event(e["decoded"])  # the previous decode of this set has read d_stream
        if gpz.gpz_copy_stream(b["h_stream"], b["comp"].out, b["comp"].d_size, cap, s_sm) != gpz.OK:
            raise RuntimeError("gpz_copy_stream (to host)")
        if gpz.gpz_copy_stream(b["d_stream"], b["h_stream"], b["comp"].d_size, cap, s_sm) != gpz.OK:
            raise RuntimeError("gpz_copy_stream (to device)")
        with torch.cuda.stream(s_sm):
            b["h_size"].copy_(b["comp"].d_size, non_blocking=True)
        e["stream_up"].record(s_sm)
        s_run.wait_event(e["stream_up"])
        s_run.wait_event(e["out_down"])  # the previous output of this set is on the host
        o_ = b["dec"](b["d_stream"], cap, s_run, check=False)  # the header bounds what is read
        e["decoded"].record(s_run)
        s_down.wait_event(e["decoded"])
        with torch.cuda.stream(s_down):
            b["h_out"].copy_(o_, non_blocking=True)
        e["out_down"].record(s_down)

    def run(steps_):
        for i in range(steps_):
            pipelined_step(i)

    run(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(k)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / k
    last = sets[(k - 1) % 2]
    size = int(last["h_size"].item())
    ok = bool(torch.equal(last["h_out"], out_ref_host)) if out_ref_host is not None else None
    for b in sets:
        for ws in (b["comp"].ws, b["dec"].ws):
            st = gpz.gpz_sync_status(ws)
            if st != gpz.OK:
                raise gpz.GpzError(st, "end-to-end (device)")

    # sequential: one stream, one step after another (no host wait either)
    b, s = sets[0], s_run

    def seq_step():
        with torch.cuda.stream(s):
            b["d_in"].copy_(h_in, non_blocking=True)
        b["comp"]([b["d_in"][f] for f in range(F)], s, sync=False)
        gpz.gpz_copy_stream(b["h_stream"], b["comp"].out, b["comp"].d_size, cap, s)
        gpz.gpz_copy_stream(b["d_stream"], b["h_stream"], b["comp"].d_size, cap, s)
        o_ = b["dec"](b["d_stream"], cap, s, check=False)
        with torch.cuda.stream(s):
            b["h_out"].copy_(o_, non_blocking=True)
            b["h_size"].copy_(b["comp"].d_size, non_blocking=True)

    seq_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        seq_step()
    torch.cuda.synchronize()
    dt_seq = (time.perf_counter() - t0) / k

    # with_alloc: every call allocates its own workspace (and synchronises)
    params = gpz.make_params(F, REL_EB, gpz.EB_REL, SEG_BITS)
    import ctypes as C
    hsz = C.c_uint64(0)

    def alloc_step():
        with torch.cuda.stream(s):
            b["d_in"].copy_(h_in, non_blocking=True)
        st = gpz.gpz_compress(b["d_in"], n, params, b["comp"].out, cap, b["comp"].d_size, hsz, None, None, 0, s)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_compress (own workspace)")
        with torch.cuda.stream(s):
            b["h_stream"][:hsz.value].copy_(b["comp"].out[:hsz.value], non_blocking=True)
            b["d_stream"][:hsz.value].copy_(b["h_stream"][:hsz.value], non_blocking=True)
        st = gpz.gpz_decompress(b["d_stream"], hsz.value, b["dec"].out, F, n, None, 0, s)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_decompress (own workspace)")
        with torch.cuda.stream(s):
            b["h_out"].copy_(b["dec"].out, non_blocking=True)
        s.synchronize()

    alloc_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        alloc_step()
    torch.cuda.synchronize()
    dt_alloc = (time.perf_counter() - t0) / k
    ok_alloc = bool(torch.equal(b["h_out"], out_ref_host)) if out_ref_host is not None else None

    # the paper's own end-to-end accounting (Section 6.2): the data already on
    # the device, each call allocating, synchronising and freeing its own
    # workspace, host clock around the call; compression and decompression
    # timed apart, as the paper reports them
    def dev_compress():
        st = gpz.gpz_compress(b["d_in"], n, params, b["comp"].out, cap, b["comp"].d_size, hsz, None, None, 0, s)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_compress (own workspace, device data)")

    def dev_decompress():
        st = gpz.gpz_decompress(b["comp"].out, hsz.value, b["dec"].out, F, n, None, 0, s)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_decompress (own workspace, device data)")

    def host_timed(fn):
        fn()
        torch.cuda.synchronize()
        t0_ = time.perf_counter()
        for _ in range(k):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0_) / k

    dt_dc = host_timed(dev_compress)
    dt_dd = host_timed(dev_decompress)
    dt, dt_seq, dt_alloc, dt_dc, dt_dd = ranks_max([dt, dt_seq, dt_alloc, dt_dc, dt_dd], dev)
    h2d, d2h = int(in_bytes + size), int(in_bytes + size + 8)
    del sets, h_in
    torch.cuda.empty_cache()
    return {"value": r4(job_gbs(world, in_bytes, 1, dt)), "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": r4(1e3 * dt), "steps": k, "pipelined": True,
            "host_waits_in_timed_region": 0, "output_checked": ok,
            "sequential": {"value": r4(job_gbs(world, in_bytes, 1, dt_seq)), "ms_per_step": r4(1e3 * dt_seq)},
            "with_alloc": {"value": r4(job_gbs(world, in_bytes, 1, dt_alloc)), "ms_per_step": r4(1e3 * dt_alloc),
                           "output_checked": ok_alloc,
                           "note": "sequential, gpz_compress / gpz_decompress each allocate and free their "
                                   "workspace (stream-ordered) and synchronise; stream sized on the host"},
            "device_with_alloc": {"compress_gbs": r4(job_gbs(world, in_bytes, 1, dt_dc)),
                                  "decompress_gbs": r4(job_gbs(world, in_bytes, 1, dt_dd)),
                                  "compress_ms": r4(1e3 * dt_dc), "decompress_ms": r4(1e3 * dt_dd),
                                  "note": "data resident on the device; each call allocates, synchronises and "
                                          "frees its own workspace; host clock (the paper's end-to-end "
                                          "accounting, no host link)"}}


# ----------------------------------------------------------------------------- GPU arm: variants on the snapshot

def timed_steps(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def variants_measure(gpz, args, x, rt, stream, dev, world):
    """Fused compaction, interleaved records, fp64 input and 64-bit
    intermediates on the same snapshot; each the GB/s of its own round trip
    (fp64 forms: GB/s of fp64 input) and its check."""
    import ctypes as C
    import torch
    F, n = x.shape
    in_bytes = 4.0 * n * F
    comp, dec, size = rt["comp"], rt["dec"], rt["size"]
    fields = [x[f] for f in range(F)]
    hs = gpz._stream_handle(stream)
    out = {}
    if not args.no_fused:
        # the in-kernel form of Section 4.4 (decoupled look-back over blocks);
        # the stream must be the same bytes
        cf = gpz.Compressor(n, F, REL_EB, gpz.EB_REL, SEG_BITS, device=dev, flags=gpz.FLAG_FUSED_COMPACTION)

        def fstep():
            cf(fields, stream, sync=False)
            dec(cf.out, size, stream, check=False)

        ms = timed_steps(fstep, min(args.steps, 60), args.warmup, stream)
        same = bool(torch.equal(cf.out[:size], comp.out[:size]))
        out["fused_compaction"] = {"value": r4(in_bytes / ms / 1e6), "ms_per_step": r4(ms), "same_stream": same,
                                   "blocks_via_copy_kernel": gpz.compress_deferred_blocks(cf.ws)}
        del cf
    if not args.no_aos:
        x_aos = x.t().contiguous()
        params = gpz.make_params(F, REL_EB, gpz.EB_REL, SEG_BITS)
        cap = gpz.gpz_bound_size(n, F)
        a_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        a_size = torch.zeros(1, dtype=torch.int64, device=dev)
        cws = gpz.gpz_compress_aos_workspace_size(n, F)
        dws = gpz.gpz_decompress_aos_workspace_size(n, F)
        a_cws = torch.empty(cws, dtype=torch.uint8, device=dev)
        a_dws = torch.zeros(dws, dtype=torch.uint8, device=dev)
        a_rec = torch.empty((n, F), dtype=torch.float32, device=dev)

        def astep():
            st1 = gpz.lib.gpz_compress_aos(x_aos.data_ptr(), n, C.byref(params), a_out.data_ptr(), cap,
                                           a_size.data_ptr(), None, None, a_cws.data_ptr(), cws, hs)
            st2 = gpz.lib.gpz_decompress_aos(a_out.data_ptr(), size, a_rec.data_ptr(), F, n, a_dws.data_ptr(), dws,
                                             hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "aos round trip")

        ms = timed_steps(astep, min(args.steps, 60), args.warmup, stream)
        for wsb in (a_cws, a_dws):
            stc = gpz.gpz_sync_status(wsb)
            if stc != gpz.OK:
                raise gpz.GpzError(stc, "aos round trip (device)")
        same = int(a_size.item()) == size and bool(torch.equal(a_out[:size], comp.out[:size]))
        out["aos"] = {"value": r4(in_bytes / ms / 1e6), "ms_per_step": r4(ms), "same_stream": same,
                      "records_checked": bool(torch.equal(a_rec.t(), dec(comp.out, size)))}
        del x_aos, a_out, a_cws, a_dws, a_rec
    if not args.no_f64:
        x64 = x.double()
        params = gpz.make_params(F, REL_EB, gpz.EB_REL, SEG_BITS)
        cap = gpz.gpz_bound_size(n, F)
        f_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        f_size = torch.zeros(1, dtype=torch.int64, device=dev)
        cws = int(gpz.lib.gpz_compress_f64_workspace_size(n, F))
        dws = int(gpz.lib.gpz_decompress_f64_workspace_size(n, F))
        f_cws = torch.empty(cws, dtype=torch.uint8, device=dev)
        f_dws = torch.zeros(dws, dtype=torch.uint8, device=dev)
        f_rec = torch.empty((F, n), dtype=torch.float64, device=dev)
        in_ptrs = gpz._ptr_array([x64[f] for f in range(F)])
        out_ptrs = gpz._ptr_array([f_rec[f] for f in range(F)])
        h_sz = C.c_uint64(0)

        def fstep64():
            st1 = gpz.lib.gpz_compress_f64(in_ptrs, n, C.byref(params), f_out.data_ptr(), cap, f_size.data_ptr(),
                                           C.byref(h_sz), None, f_cws.data_ptr(), cws, None, hs)
            st2 = gpz.lib.gpz_decompress_f64(f_out.data_ptr(), h_sz.value, out_ptrs, F, n, f_dws.data_ptr(), dws, hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "fp64 round trip")

        ms = timed_steps(fstep64, min(args.steps, 30), args.warmup, stream)
        stc = gpz.gpz_sync_status(f_dws)
        if stc != gpz.OK:
            raise gpz.GpzError(stc, "fp64 round trip (device)")
        out["f64"] = {"value": r4(8.0 * n * F / ms / 1e6), "unit": "GB/s of fp64 input", "ms_per_step": r4(ms),
                      "ratio_vs_fp64": r4(8.0 * n * F / h_sz.value)}
        del x64, f_out, f_cws, f_dws, f_rec
    if not args.no_wide:
        x64 = x.double()
        wide_rel = 1e-12  # a bound fp32 cannot hold
        cap = gpz.gpz_bound_size_wide(n, F)
        w_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        w_size = torch.zeros(1, dtype=torch.int64, device=dev)
        cws = int(gpz.lib.gpz_compress_wide_workspace_size(n, F))
        w_cws = torch.empty(cws, dtype=torch.uint8, device=dev)
        w_dws = torch.zeros(256, dtype=torch.uint8, device=dev)
        w_rec = torch.empty((F, n), dtype=torch.float64, device=dev)
        in_ptrs = gpz._ptr_array([x64[f] for f in range(F)])
        out_ptrs = gpz._ptr_array([w_rec[f] for f in range(F)])
        h_sz = C.c_uint64(0)
        used = (C.c_double * F)()
        rel_params = gpz.make_params(F, wide_rel, gpz.EB_REL, SEG_BITS)
        st = gpz.lib.gpz_compress_wide(in_ptrs, n, C.byref(rel_params), w_out.data_ptr(), cap, None, C.byref(h_sz),
                                       None, w_cws.data_ptr(), cws, used, hs)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_compress_wide")
        params = gpz.make_params(F, [used[f] for f in range(F)], gpz.EB_ABS, SEG_BITS)

        def wstep():
            st1 = gpz.lib.gpz_compress_wide(in_ptrs, n, C.byref(params), w_out.data_ptr(), cap, w_size.data_ptr(),
                                            None, None, w_cws.data_ptr(), cws, None, hs)
            st2 = gpz.lib.gpz_decompress_wide(w_out.data_ptr(), cap, out_ptrs, F, n, w_dws.data_ptr(), 256, hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "64-bit round trip")

        ms = timed_steps(wstep, min(args.steps, 20), args.warmup, stream)
        stc = gpz.gpz_sync_status(w_dws)
        if stc != gpz.OK:
            raise gpz.GpzError(stc, "64-bit round trip (device)")
        out["wide"] = {"value": r4(8.0 * n * F / ms / 1e6), "unit": "GB/s of fp64 input", "ms_per_step": r4(ms),
                       "rel_eb": wide_rel, "ratio_vs_fp64": r4(8.0 * n * F / int(w_size.item()))}
        del x64, w_out, w_cws, w_dws, w_rec
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- GPU arm: the default line

def run_gpz(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = load_peaks()

    n, F = args.n, N_FIELDS
    x = make_workload(n, rank, dev)
    rt = round_trip(gpz, x, REL_EB, gpz.EB_REL, args.steps, args.warmup, stream, dev, world, clocks_index=local)
    in_bytes = rt["in_bytes"]
    value = job_gbs(world, in_bytes, args.steps, rt["ms"] * args.steps / 1e3)
    size = rt["size"]
    payload_bytes = size - 4 * (16 + 2 * F + (n + 1023) // 1024 + 1)
    nb = (n + 1023) // 1024
    # each kernel's algorithmic bytes per step (read + write), for its roofline
    algo = {
        "range": in_bytes,                       # one read of every field
        "info": 8.0 * (F + 1) * nb,              # read each block's extremes, write its widths
        "qse": in_bytes + payload_bytes,         # read the input, write the encoded blocks
        "scan": 8.0 * nb,                        # read sizes, write offsets
        "compact": 2.0 * payload_bytes,          # read the temporary blocks, write the stream
        "decompress": size + in_bytes,           # read the stream, write every value
    }
    kernels = {}
    for k, (tot, cnt) in rt["stages"].items():
        if cnt == 0:
            continue
        step_s = tot / rt["kreps"] / 1e3
        ach = algo.get(k, 0.0) / step_s / 1e9
        kernels[k] = [r4(1e3 * step_s), r4(ach / peak)]
    dom = max(kernels, key=lambda k: kernels[k][0])
    kname = {"qse": "gpz_qse_tile_kernel"}.get(dom, "gpz_%s_kernel" % dom)
    dom_ms = kernels[dom][0]
    roofline = {"bound": "hbm", "kernel": kname, "achieved": r4(algo[dom] / (dom_ms / 1e3) / 1e9), "peak": peak,
                "unit": "GB/s", "frac": r4(algo[dom] / (dom_ms / 1e3) / 1e9 / peak), "traffic": recorded_traffic(dom),
                "peak_source": peak_kind, "note": "frac of %s copy bandwidth" % peak_kind,
                "frac_of_nominal": r4(algo[dom] / (dom_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS),
                "nominal_peak": NOMINAL_HBM_GBS}
    comp_roof, dec_roof = direction_rooflines(rt, peak, peak_kind)
    result = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rt["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": gpu_config(n, world),
        "roofline": roofline, "gpu_launches": rt["launches"], "clocks": rt["clocks"],
    }
    out_ref_host = rt["out_host"]
    timings = {}

    def timed_part(name, fn):
        t0 = time.perf_counter()
        v = fn()
        timings[name] = round(time.perf_counter() - t0, 1)
        return v

    variants = timed_part("variants", lambda: variants_measure(gpz, args, x, rt, stream, dev, world))
    del rt["comp"], rt["dec"]
    torch.cuda.empty_cache()
    if not args.no_e2e:
        result["e2e"] = timed_part("e2e", lambda: e2e_measure(gpz, x, out_ref_host,
                                                              max(3, min(20, args.steps // 10)), dev, world))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def cpu():
            ebs = absolute_bounds(x.cpu().numpy(), REL_EB)
            sample = host_blocks(x, np.arange(0, nb, 4))
            gbs1, tc, td = cpu_oracle_sample(sample, F, ebs)
            whole = x.cpu().numpy()
            gbs, dt, used = cpu_oracle_threads(whole, F, os.cpu_count() or 1, ebs)
            return {"value": gbs, "unit": "GB/s", "cores": used, "kind": "oracle",
                    "sample": "the whole snapshot (%d particles x 6 fields), one compress + decompress, the C++ "
                              "oracle over %d host threads by contiguous block ranges, relative eb over the "
                              "snapshot; %.1f s" % (n, used, dt),
                    "single_thread": {"value": gbs1, "cores": 1,
                                      "sample": "every 4th 1024-particle block (%d particles x 6 fields); %.1f s"
                                                % (sample.shape[1], tc + td)}}
        result["cpu_baseline"] = timed_part("cpu_baseline", cpu)
    del x
    torch.cuda.empty_cache()

    result["kernels_ms_frac"] = kernels
    result["variants"] = variants
    if not args.no_small:
        def small():
            xs = torch.from_numpy(synth.uniform_box(1_000_000, seed=0)).to(dev)
            r = round_trip(gpz, xs, 1e-2, gpz.EB_ABS, max(20, args.steps), args.warmup, stream, dev, world)
            return workload_summary(r, peak, peak_kind, "uniform [0,256)^3, seed 0", 1_000_000, 3, 1e-2, "abs")
        result["small"] = timed_part("small", small)
    if not args.no_lidar:
        def lidar():
            xl = synth.lidar(200_000_000, seed=3, device=dev)
            r = round_trip(gpz, xl, 1e-3, gpz.EB_ABS, max(5, args.steps // 10), args.warmup, stream, dev, world)
            return workload_summary(r, peak, peak_kind, "LiDAR-like scan, 10 km tile, seed 3", 200_000_000, 3,
                                    1e-3, "abs (m)")
        result["lidar"] = timed_part("lidar", lidar)
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_batched:
        result["batched"] = timed_part("batched", lambda: batched_measure(args, embedded=True))
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_served:
        result["served"] = timed_part("served", lambda: served_measure(args, embedded=True))
        torch.cuda.empty_cache()
    result["part_seconds"] = timings
    # the gate figures last, so that a record keeping the end of the line keeps them
    result["compress_roofline"] = comp_roof
    result["decompress_roofline"] = dec_roof
    result["compress_gbs"] = r4(in_bytes / rt["comp_ms"] / 1e6) if rt["comp_ms"] else None
    result["decompress_gbs"] = r4(in_bytes / rt["dec_ms"] / 1e6) if rt["dec_ms"] else None
    result["stream_bytes"] = size
    result["ratio"] = r4(rt["ratio"])
    result["psnr_db"] = r4(rt["psnr"])
    result["max_err_over_eb"] = r4(rt["worst"])
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ----------------------------------------------------------------------------- batched workload

def batched_measure(args, embedded=False):
    """Batched compress + decompress of many uneven chunks: the batched plans
    (tuned, replayed as CUDA graphs) against one call per chunk, eager and
    captured in one CUDA graph.  Returns the result dict (embedded: the
    compact form of the default line)."""
    import ctypes as C
    import torch
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    steps = args.batched_steps if embedded else args.steps
    warm = min(args.warmup, 3) if embedded else args.warmup
    t0 = time.perf_counter()
    wl = synth.batched_workload(n_chunks=args.chunks, lo=args.chunk_lo, hi=args.chunk_hi, seed=4, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    in_bytes = float(wl.input_bytes())
    params = [gpz.make_params(wl.F[c], [wl.rel[c]] * wl.F[c], gpz.EB_REL, SEG_BITS) for c in range(wl.count)]
    bc = gpz.BatchCompressor([(wl.fields(c), params[c]) for c in range(wl.count)], device=dev, use_graph=True)
    bc()
    st, per = bc.status()
    if st != gpz.OK:
        raise gpz.GpzError(st, "batched compress")
    sizes = bc.sizes.tolist()
    streams = bc.streams()
    bd = gpz.BatchDecompressor([(streams[c], sizes[c], wl.F[c], wl.n[c]) for c in range(wl.count)], device=dev,
                               use_graph=True)
    bd()
    st, _ = bd.status()
    if st != gpz.OK:
        raise gpz.GpzError(st, "batched decompress")

    def batched_step():
        bc(stream)
        bd(stream)

    def timed(fn, steps_, warm_):
        for _ in range(warm_):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps_):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps_

    if args.batched_only and not embedded:
        ms = timed(batched_step, steps, warm)
        out = {"workload": "batched (plans only, default shapes)", "chunks": wl.count,
               "input_gb": in_bytes / 1e9, "ms_per_step": ms, "gbs": in_bytes / (ms / 1e3) / 1e9}
        bc.close()
        bd.close()
        return out

    # tuned launch shapes (the outputs are rewritten with the same bytes)
    ccfg, cms = bc.tune(reps=2)
    dcfg, dms = bd.tune(reps=2)

    # parity: every chunk's stream equals its single-call stream; sampled
    # small chunks equal the CPU oracle's
    ws_max = max(gpz.gpz_compress_workspace_size(wl.n[c], wl.F[c]) for c in range(wl.count))
    ws = torch.empty(ws_max, dtype=torch.uint8, device=dev)
    cap_max = max(gpz.gpz_bound_size(wl.n[c], wl.F[c]) for c in range(wl.count))
    scratch = torch.empty(cap_max, dtype=torch.uint8, device=dev)
    hsize = C.c_uint64(0)
    equal = 0
    for c in range(wl.count):
        rc = gpz.gpz_compress(wl.fields(c), wl.n[c], params[c], scratch, cap_max, None, hsize, None, ws, ws_max)
        if rc != gpz.OK:
            raise gpz.GpzError(rc, "gpz_compress")
        equal += int(hsize.value == sizes[c] and torch.equal(scratch[:sizes[c]], streams[c]))
    from oracle import gpz_oracle
    gpz_oracle.lib()
    small = [c for c in range(wl.count) if wl.n[c] <= 40000][:8]
    oracle_equal = 0
    for c in small:
        xh = torch.stack(wl.fields(c)).cpu().numpy()
        rs, _ = gpz_oracle.compress(xh, [wl.rel[c]] * wl.F[c], 1, SEG_BITS, want_perm=False)
        oracle_equal += int(np.array_equal(streams[c].cpu().numpy(), rs))
    del scratch

    # one call per chunk through the public API (same buffers, same order of
    # work: every chunk compressed, then every chunk decompressed)
    d_size = torch.zeros(wl.count, dtype=torch.int64, device=dev)
    dec_ws = torch.zeros(max(gpz.gpz_decompress_workspace_size(), 256), dtype=torch.uint8, device=dev)
    sh = C.c_void_p(stream.cuda_stream)
    comp_args, dec_args = [], []
    for c in range(wl.count):
        comp_args.append((gpz._ptr_array(wl.fields(c)), wl.n[c], C.byref(params[c]), bc.outs[c].data_ptr(),
                          gpz.gpz_bound_size(wl.n[c], wl.F[c]), d_size[c:].data_ptr()))
        outs = bd.outs[c]
        dec_args.append((streams[c].data_ptr(), sizes[c], gpz._ptr_array([outs[f] for f in range(wl.F[c])]),
                         wl.F[c], wl.n[c]))

    def per_chunk_step(s_handle):
        for a in comp_args:
            gpz.lib.gpz_compress(a[0], a[1], a[2], a[3], a[4], a[5], None, None, ws.data_ptr(), ws_max, s_handle)
        for a in dec_args:
            gpz.lib.gpz_decompress(a[0], a[1], a[2], a[3], a[4], dec_ws.data_ptr(), dec_ws.numel(), s_handle)

    gpz.gpz_launch_count(reset=True)
    with ClockSampler(0) as clk:
        batched_ms = timed(batched_step, steps, warm)
    launches = gpz.gpz_launch_count() // max(1, steps + warm)
    pc_steps = max(1, min(3, steps))
    per_chunk_ms = timed(lambda: per_chunk_step(sh), pc_steps, 1)
    per_chunk_launches = (gpz.gpz_launch_count(reset=True) - launches * (steps + warm)) // (pc_steps + 1)
    # the same per-chunk calls captured into one CUDA graph
    per_chunk_graph_ms, graph_note = None, None
    try:
        graph = torch.cuda.CUDAGraph()
        cap_stream = torch.cuda.Stream(dev)
        cap_stream.wait_stream(stream)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="thread_local"):
            per_chunk_step(C.c_void_p(cap_stream.cuda_stream))
        torch.cuda.synchronize()
        per_chunk_graph_ms = timed(graph.replay, pc_steps, 1)
        del graph
    except Exception as exc:  # reported, not fatal: the eager comparison stands
        graph_note = "capture failed: %s" % str(exc).splitlines()[0][:200]
    for w in (bc, bd):
        st, _ = w.status()
        if st != gpz.OK:
            raise gpz.GpzError(st, "timed region")

    # per-kernel times of one eager run of each plan
    gpz.gpz_set_stage_timing(True, stream)
    gpz.gpz_stage_times()
    bc.use_graph = bd.use_graph = False
    for _ in range(2):
        batched_step()
    torch.cuda.synchronize()
    stages = gpz.gpz_stage_times(16)
    gpz.gpz_set_stage_timing(False, stream)
    total_stream = float(sum(sizes))
    nblocks = sum((n + 1023) // 1024 for n in wl.n)
    payload = total_stream - 4.0 * sum(16 + 2 * F + (n + 1023) // 1024 + 1 for n, F in zip(wl.n, wl.F))
    algo = {"batch_qse": 2 * in_bytes + payload, "batch_scan": 12.0 * nblocks, "batch_compact": 2 * payload,
            "batch_decompress": total_stream + in_bytes}
    peak, peak_kind = load_peaks()
    kernels = {}
    runs = 2
    for k, (tot, cnt) in stages.items():
        run_s = tot / runs / 1e3  # all launches of the stage in one run (one per field-count group)
        ach = algo[k] / run_s / 1e9 if k in algo else None
        kernels[k] = {"ms_per_run": 1e3 * run_s, "launches_per_run": cnt // runs, "algorithmic_bytes": algo.get(k),
                      "achieved_gbs": ach, "frac": ach / peak if ach else None}
    dom = max((k for k in kernels if k in algo), key=lambda k: kernels[k]["ms_per_run"])
    bc.close()
    bd.close()
    workload = ("batched: %d chunks, particles log-uniform in [%d, %d] (total %d), 3 fields (uniform box) or 6 "
                "(cosmology-like), relative eb 1e-3 / 1e-4, G = 3" % (wl.count, args.chunk_lo, args.chunk_hi,
                                                                       sum(wl.n)))
    value = in_bytes / (batched_ms / 1e3) / 1e9
    if embedded:
        return {"workload": workload, "value": r4(value), "unit": "GB/s", "ms_per_step": r4(batched_ms),
                "steps": steps, "input_gb": r4(in_bytes / 1e9),
                "per_chunk_eager_gbs": r4(in_bytes / (per_chunk_ms / 1e3) / 1e9),
                "per_chunk_graph_gbs": r4(in_bytes / (per_chunk_graph_ms / 1e3) / 1e9) if per_chunk_graph_ms else None,
                "speedup_vs_per_chunk_eager": r4(per_chunk_ms / batched_ms),
                "speedup_vs_per_chunk_graph": r4(per_chunk_graph_ms / batched_ms) if per_chunk_graph_ms else None,
                "launches_per_step": launches, "per_chunk_launches_per_step": per_chunk_launches,
                "ratio": r4(in_bytes / total_stream), "dominant_kernel": [dom, r4(kernels[dom]["frac"])],
                "chunks_equal_single_call": "%d/%d" % (equal, wl.count),
                "sampled_chunks_equal_oracle": "%d/%d" % (oracle_equal, len(small)),
                "tuned": {"compress": ccfg.as_dict(), "decompress": dcfg.as_dict()},
                "clocks": clk.summary(), "generate_s": r4(gen_s)}
    return {
        "metric": "batched compress+decompress GB/s (graph-replayed batched plans vs one call per chunk)",
        "value": value, "unit": "GB/s", "n_gpus": 1, "steps": steps,
        "warmup": warm, "ms_per_step": batched_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "input_gb": in_bytes / 1e9, "l2": "inputs larger than L2; no flush"},
        "per_chunk": {"eager_gbs": in_bytes / (per_chunk_ms / 1e3) / 1e9, "eager_ms": per_chunk_ms,
                      "graph_gbs": in_bytes / (per_chunk_graph_ms / 1e3) / 1e9 if per_chunk_graph_ms else None,
                      "graph_ms": per_chunk_graph_ms, "graph_note": graph_note,
                      "launches_per_step": per_chunk_launches},
        "speedup_vs_per_chunk_eager": per_chunk_ms / batched_ms,
        "speedup_vs_per_chunk_graph": per_chunk_graph_ms / batched_ms if per_chunk_graph_ms else None,
        "tuned": {"compress": ccfg.as_dict(), "compress_ms": cms, "decompress": dcfg.as_dict(), "decompress_ms": dms},
        "ratio": in_bytes / total_stream,
        "parity": {"chunks_equal_single_call": equal, "chunks": wl.count,
                   "sampled_chunks_equal_oracle": oracle_equal, "sampled": len(small)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["achieved_gbs"], "peak": peak,
                     "unit": "GB/s", "frac": kernels[dom]["frac"], "traffic": None, "peak_source": peak_kind},
        "kernels": kernels, "gpu_launches": launches, "clocks": clk.summary(), "generate_s": gen_s,
    }


# ----------------------------------------------------------------------------- served workload

SERVED_GENS = [("uniform box", 3, 1e-2, 0), ("cosmology-like", 6, 1e-4, 1), ("LiDAR-like", 3, 1e-3, 0)]


def served_measure(args, embedded=False):
    """Real-time replay of Poisson request traces against the serving engine:
    continuous batching (the first arm of --serve-arms: two lanes, up to 64
    requests per batch, an express lane for small requests) against the plain
    path (one lane, one request per launch sequence), at --rate requests/s
    and at --sat-rate, a rate above either arm's capacity, where the arms
    differ in the throughput they sustain.  Returns the result dict."""
    import torch
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pool_n = 64_000_000
    t0 = time.perf_counter()
    pools = [synth.uniform_box_torch(pool_n, seed=0, device=dev),
             synth.cosmology(pool_n, seed=2, device=dev),
             synth.lidar(pool_n, seed=3, device=dev)]
    params = [gpz.make_params(F, eb, mode, SEG_BITS) for (_, F, eb, mode) in SERVED_GENS]
    # decompression requests read resident streams: 16 sizes per generator, log-spaced in [1e5, 6.4e7]
    classes = np.unique(np.round(np.exp(np.linspace(np.log(1e5), np.log(6.4e7), 16))).astype(np.int64))
    streams = {}
    for g, (_, F, _, _) in enumerate(SERVED_GENS):
        for n in classes:
            comp = gpz.Compressor(int(n), F, params[g].eb[:F], params[g].mode, SEG_BITS, device=dev)
            size = comp([pools[g][f, :n] for f in range(F)])
            streams[(g, int(n))] = comp.out[:size].clone()
            del comp
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0

    def make_trace(requests, rate, seed):
        t_arr, size, gen, op = synth.request_trace(requests, rate=rate, lo=100_000, hi=64_000_000, seed=seed)
        rng = np.random.default_rng(seed + 1)
        reqs = []
        for i in range(requests):
            g, F = int(gen[i]), SERVED_GENS[int(gen[i])][1]
            if op[i] == 0:
                n = int(size[i])
                off = int(rng.integers(0, (pool_n - n) // 32 + 1)) * 32
                reqs.append((0, g, F, n, off))
            else:
                n = int(classes[np.argmin(np.abs(np.log(classes) - np.log(size[i])))])
                reqs.append((1, g, F, n, 0))
        return t_arr, reqs, sum(4 * r[3] * r[2] for r in reqs)

    def arm(trace, lanes, max_batch, batch_mb, lane_mb):
        t_arr, reqs, raw_bytes = trace
        srv = gpz.Server(int(args.budget_gb * (1 << 30)), lanes=lanes, max_batch=max_batch,
                         max_batch_bytes=int(batch_mb * (1 << 20)), lane_bytes=int(lane_mb * (1 << 20)))
        # warm-up: one request of each kind and generator
        warm = []
        for g, (_, F, _, _) in enumerate(SERVED_GENS):
            warm.append(srv.submit_compress([pools[g][f, :200_000] for f in range(F)], params[g]))
            s_ = streams[(g, int(classes[0]))]
            warm.append(srv.submit_decompress(s_, s_.numel(), F, int(classes[0])))
        left = len(warm)
        while left:
            for res in srv.poll(timeout_ms=5000):
                srv.release(res["id"])
                left -= 1
        results, checks = [], {}
        sample = set(range(0, len(reqs), 97))
        id_to_req = {}
        done = threading.Event()

        def poller():
            got = 0
            while got < len(reqs):
                for res in srv.poll(timeout_ms=200):
                    k = id_to_req.get(res["id"])
                    while k is None:  # the submitting thread has not recorded the id yet
                        time.sleep(0.0001)
                        k = id_to_req.get(res["id"])
                    if k in sample and res["status"] == gpz.OK:
                        r = reqs[k]
                        checks[k] = (srv.stream_of(res).clone() if r[0] == 0 else
                                     srv.fields_of(res, r[2], r[3]))
                        # the copy runs on this thread's stream, which does not wait for
                        # the engine's lanes: finish it before the result's arena memory
                        # is released and reused by a later request
                        torch.cuda.current_stream().synchronize()
                    results.append((k, res))
                    srv.release(res["id"])
                    got += 1
            done.set()

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        lag = []
        start = time.perf_counter() + 0.05
        for k, r in enumerate(reqs):
            target = start + float(t_arr[k])
            while True:
                dt = target - time.perf_counter()
                if dt <= 0:
                    break
                if dt > 0.0006:
                    time.sleep(dt - 0.0004)
            kind, g, F, n, off = r
            if kind == 0:
                rid = srv.submit_compress([pools[g][f, off:off + n] for f in range(F)], params[g])
            else:
                s_ = streams[(g, n)]
                rid = srv.submit_decompress(s_, s_.numel(), F, n)
            id_to_req[rid] = k
            lag.append(time.perf_counter() - target)
        done.wait()
        th.join()
        stats = srv.stats()
        srv.close()
        # parity of the sampled results against one call per request
        equal = 0
        for k, out in checks.items():
            kind, g, F, n, off = reqs[k]
            if kind == 0:
                comp = gpz.Compressor(n, F, params[g].eb[:F], params[g].mode, SEG_BITS, device=dev)
                sz = comp([pools[g][f, off:off + n] for f in range(F)])
                equal += int(torch.equal(comp.out[:sz], out))
            else:
                s_ = streams[(g, n)]
                ref = gpz.Decompressor(n, F, device=dev)(s_, s_.numel())
                equal += int(torch.equal(ref[:, :n].view(torch.int32), out.view(torch.int32)))
        lat = np.array([(res["t_done_ns"] - res["t_submit_ns"]) / 1e6 for _, res in results])
        kinds = np.array([reqs[k][0] for k, _ in results])
        ok = all(res["status"] == gpz.OK for _, res in results)
        span = (max(res["t_done_ns"] for _, res in results) - min(res["t_submit_ns"] for _, res in results)) / 1e9
        bsz = np.array([res["batch_size"] for _, res in results])

        def pct(a, q):
            return r4(float(np.percentile(a, q))) if a.size else None
        return {
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": r4(float(lat.mean())),
            "compress_p50_ms": pct(lat[kinds == 0], 50), "compress_p99_ms": pct(lat[kinds == 0], 99),
            "decompress_p50_ms": pct(lat[kinds == 1], 50), "decompress_p99_ms": pct(lat[kinds == 1], 99),
            "aggregate_gbs": r4(raw_bytes / span / 1e9), "span_s": r4(span), "all_ok": ok,
            "batches": stats["batches"], "mean_batch": r4(float(bsz.mean())), "max_batch": int(bsz.max()),
            "arena_peak_gb": r4(stats["arena_peak"] / 1e9), "submit_lag_p99_ms": r4(1e3 * float(np.percentile(lag, 99))),
            "sampled_equal_single_call": "%d/%d" % (equal, len(checks)), "lanes": lanes, "max_batch_cfg": max_batch,
            "max_batch_mb": batch_mb, "express_lane_mb": lane_mb,
        }

    specs = [spec.split(":") for spec in args.serve_arms.split(",")]
    names = [s[0] for s in specs]
    loads = [("rate_%d" % int(args.rate), make_trace(args.requests, args.rate, 5)),
             ("saturated_%d" % int(args.sat_rate), make_trace(args.sat_requests, args.sat_rate, 7))]
    runs = {}
    with ClockSampler(0) as clk:
        for label, trace in loads:
            runs[label] = {"offered_gbs": r4(trace[2] / float(trace[0][-1]) / 1e9), "requests": len(trace[1]),
                           "raw_gb": r4(trace[2] / 1e9)}
            for (name, lanes, mb, bmb, lmb) in specs:
                runs[label][name] = arm(trace, int(lanes), int(mb), float(bmb), float(lmb))
    served, plain = names[0], ("plain" if "plain" in names else names[-1])
    sat = runs[loads[1][0]]
    summary = {
        "workload": "served: Poisson traces, 100K-64M particles log-uniform, generators uniform box (3 fields, abs "
                    "1e-2) / cosmology-like (6, rel 1e-4) / LiDAR-like (3, abs 1e-3), half compress, half "
                    "decompress (resident streams of 16 size classes), %.0f GB admission budget" % args.budget_gb,
        "served_arm": served, "plain_arm": plain,
        "p99_ms": runs[loads[0][0]][served]["p99_ms"], "plain_p99_ms": runs[loads[0][0]][plain]["p99_ms"],
        "saturated_gbs": sat[served]["aggregate_gbs"], "plain_saturated_gbs": sat[plain]["aggregate_gbs"],
        "saturated_p99_ms": sat[served]["p99_ms"], "plain_saturated_p99_ms": sat[plain]["p99_ms"],
        "loads": runs, "clocks": clk.summary(), "prepare_s": r4(prep_s),
    }
    if embedded:
        return summary
    return {
        "metric": "served p50/p99 latency (ms) and aggregate GB/s: continuous batching vs plain path",
        "value": summary["p99_ms"], "unit": "ms (p99 latency)", "n_gpus": 1, "steps": args.requests, "warmup": 6,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": summary["workload"], "rate": args.rate, "sat_rate": args.sat_rate},
        "served": summary,
    }


def run_sweep(args):
    """Ratio, quality and throughput over error bounds and segment bits G on
    the three single-array workloads (the paper's rate-distortion view,
    Fig. 7, on synthetic stand-ins): per point the compression ratio, bits
    per value, PSNR, max |error| / eb and compress / decompress GB/s (CUDA
    events, stage timing).  One JSON line."""
    import torch
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz, synth

    dev = torch.device("cuda", 0)
    workloads = [
        ("uniform 1e6 x 3, absolute eb", lambda: synth.uniform_box_torch(1_000_000, seed=0, device=dev),
         gpz.EB_ABS, [1e-1, 1e-2, 1e-3, 1e-4]),
        ("cosmology 2^26 x 6, relative eb", lambda: synth.cosmology(1 << 26, seed=2, device=dev),
         gpz.EB_REL, [1e-2, 1e-3, 1e-4, 1e-5]),
        ("LiDAR 2e8 x 3, absolute eb (m)", lambda: synth.lidar(200_000_000, seed=3, device=dev),
         gpz.EB_ABS, [1e-1, 1e-2, 1e-3]),
    ]
    points = []
    for name, make, mode, ebs in workloads:
        x = make()
        F, n = x.shape
        fields = [x[f] for f in range(F)]
        in_bytes = 4.0 * n * F
        dec = gpz.Decompressor(n, F, device=dev)
        for eb in ebs:
            for G in (0, 1, 2, 3):
                comp = gpz.Compressor(n, F, eb, mode, G, want_perm=True, device=dev)
                size = comp(fields)
                out = dec(comp.out, size)
                hdr = comp.out[:4 * (16 + 2 * F)].cpu().numpy().view(np.uint32)
                ebf = [float(hdr[16 + 2 * f].view(np.float32)) for f in range(F)]
                psnr, worst = psnr_and_error(x, out, comp.perm[:n].long(), ebf)
                reps = 5
                gpz.gpz_set_stage_timing(True)
                gpz.gpz_stage_times()
                for _ in range(reps):
                    comp(fields, sync=False)
                    dec(comp.out, size, check=False)
                torch.cuda.synchronize()
                st = gpz.gpz_stage_times()
                gpz.gpz_set_stage_timing(False)
                c_ms = sum(st[k][0] for k in ("range", "info", "qse", "scan", "compact") if k in st) / reps
                d_ms = st.get("decompress", (0.0, 1))[0] / reps
                points.append({"workload": name, "eb": eb, "G": G, "ratio": in_bytes / size,
                               "bits_per_value": 8.0 * size / (n * F), "psnr_db": psnr, "max_err_over_eb": worst,
                               "compress_gbs": in_bytes / c_ms / 1e6, "decompress_gbs": in_bytes / d_ms / 1e6})
                del comp, out
                torch.cuda.empty_cache()
        del x, fields, dec
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "sweep", "unit": "GB/s of input; ratio = input / stream bytes",
                      "data": "synthetic", "points": points}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        if rank == 0:
            print(json.dumps(batched_measure(args)), flush=True)
    elif args.workload == "served":
        if rank == 0:
            print(json.dumps(served_measure(args)), flush=True)
    elif args.workload == "sweep":
        if rank == 0:
            run_sweep(args)
    else:
        run_gpz(args, rank, world, local)


if __name__ == "__main__":
    main()
