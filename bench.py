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

One JSON line on rank 0.  The reference arm (--impl reference) times the
plain single-threaded CPU oracle on a bounded sample of the same workload.

    python bench.py --workload served [--requests 4000]

replays a Poisson trace (2,000 requests/s, 100K-64M particles log-uniform,
the uniform-box, cosmology-like and LiDAR-like generators, half compress and
half decompress) in real time against the serving engine with a 40 GB
admission budget: continuous batching over two lanes against the plain path
(one request per launch sequence, one lane); p50 / p99 latency and aggregate
GB/s of each.

    python bench.py --workload batched [--chunks 4096] [--steps K] [--warmup W]

measures the batched form instead (one line, not the headline): 4,096 chunks
with log-uniform particle counts in 10K-4M, 3 or 6 fields, relative bounds
1e-3 / 1e-4, compressed and decompressed by the batched launches
replayed as CUDA graphs with a tuned launch shape, against the same chunks
through one gpz_compress / gpz_decompress call each (eager, and captured in
one CUDA graph).
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
    ap.add_argument("--workload", default="cosmology", choices=["cosmology", "batched", "served", "sweep"])
    ap.add_argument("--requests", type=int, default=4000, help="served workload: requests per arm")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="served workload: admission budget")
    ap.add_argument("--rate", type=float, default=2000.0, help="served workload: requests per second")
    ap.add_argument("--serve-arms", default="batched:2:64:256:64,plain:1:1:0:0",
                    help="served workload: name:lanes:max_batch:max_batch_MB:express_lane_MB, comma separated; "
                         "the first is reported as the served value, the one named plain as the comparison")
    ap.add_argument("--chunks", type=int, default=4096, help="batched workload: number of chunks")
    ap.add_argument("--chunk-lo", type=int, default=10_000)
    ap.add_argument("--chunk-hi", type=int, default=4_000_000)
    ap.add_argument("--batched-only", action="store_true",
                    help="batched workload: time the batched plans only (default shapes; no tuning, no per-chunk "
                         "arm, no parity pass): for profiling")
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


def cpu_oracle_sample(x_host_blocks, n_fields):
    """Time the CPU oracle (single thread) on a host sample; returns GB/s of input per round trip."""
    from oracle import gpz_oracle
    gpz_oracle.lib()
    t0 = time.perf_counter()
    stream, _ = gpz_oracle.compress(x_host_blocks, REL_EB, 1, SEG_BITS, want_perm=False)
    t1 = time.perf_counter()
    gpz_oracle.decompress(stream, n_fields, x_host_blocks.shape[1])
    t2 = time.perf_counter()
    return x_host_blocks.nbytes / (t2 - t0) / 1e9, t1 - t0, t2 - t1


def cpu_oracle_threads(x_host, n_fields, threads):
    """The oracle, unchanged, over `threads` host threads: each compresses and
    then decompresses a contiguous range of whole blocks (blocks are
    independent).  The relative bound is first turned into each field's
    absolute bound over the whole array, as the oracle itself computes it, so
    every block is encoded as in one call on the whole array.  ctypes releases
    the interpreter lock during the C calls.  Returns (GB/s of input per round
    trip, wall seconds, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import gpz_oracle
    gpz_oracle.lib()
    F, n = x_host.shape
    ebs = []
    for f in range(F):
        v = x_host[f][~np.isnan(x_host[f])]
        rng = float(v.max()) - float(v.min()) if v.size else 0.0
        e = REL_EB * rng
        ebs.append(e if (0.0 < rng < float("inf") and 0.0 < e < float("inf")) else REL_EB)
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


def host_sample(x_dev, every=4):
    """Every `every`-th 1024-particle block of the device workload, on the host."""
    import torch
    n = x_dev.shape[1]
    nb = n // 1024
    idx = torch.arange(0, nb, every, device=x_dev.device)
    sel = (idx[:, None] * 1024 + torch.arange(1024, device=x_dev.device)[None, :]).reshape(-1)
    return x_dev[:, sel].cpu().numpy(), sel.numel()


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host's cores (one thread per core,
    each on a contiguous range of whole blocks), on the same workload, metric
    and unit.  Each step is a bounded sample of whole 1024-particle blocks
    spread over the snapshot (rotating offset), sized so that all steps
    together take about 90 s of single-core work per core."""
    if rank != 0:
        return
    import torch
    from paper_2508_10305_gb300 import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    x = synth.cosmology(args.n, seed=SEED, device=dev)
    nb = args.n // 1024
    nthreads = os.cpu_count() or 1
    per_step = int(max(8 * nthreads, min(nb, nthreads * 90.0 * 1.4e6 / max(1, args.steps) / 1024)))
    stride = max(1, nb // per_step)

    def sample(i):
        blocks = torch.arange(i % stride, nb, stride, device=x.device)[:per_step]
        sel = (blocks[:, None] * 1024 + torch.arange(1024, device=x.device)[None, :]).reshape(-1)
        return x[:, sel].cpu().numpy()

    for i in range(args.warmup):
        cpu_oracle_threads(sample(i)[:, :nthreads << 14], N_FIELDS, nthreads)
    total, nbytes, used = 0.0, 0, 1
    for i in range(args.steps):
        s = sample(i)
        _, dt, used = cpu_oracle_threads(s, N_FIELDS, nthreads)
        total += dt
        nbytes += s.nbytes
    value = nbytes / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "fields": N_FIELDS, "eb_mode": "rel", "eb": REL_EB,
                   "seg_bits": SEG_BITS},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": used, "kind": "oracle",
                         "sample": "per step %d whole 1024-particle blocks (every %dth, rotating offset) x 6 "
                                   "fields; C++ oracle compress + decompress over %d host threads by block "
                                   "range; relative eb over the sample" % (per_step, stride, used)},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def run_gpz(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    n, F = args.n, N_FIELDS
    x = make_workload(n, rank, dev)
    fields = [x[f] for f in range(F)]
    comp = gpz.Compressor(n, F, REL_EB, gpz.EB_REL, SEG_BITS, want_perm=False, device=dev)
    dec = gpz.Decompressor(n, F, device=dev)
    stream = torch.cuda.current_stream(dev)

    # one checked round trip with the permutation: ratio, PSNR, error bound
    chk = gpz.Compressor(n, F, REL_EB, gpz.EB_REL, SEG_BITS, want_perm=True, device=dev)
    size = chk(fields)
    out = dec(chk.out, size)
    perm = chk.perm[:n].long()
    hdr = chk.out[:4 * (16 + 2 * F)].cpu().numpy().view(np.uint32)
    ebs = [float(hdr[16 + 2 * f].view(np.float32)) for f in range(F)]
    psnr, worst = psnr_and_error(x, out, perm, ebs)
    ratio = x.numel() * 4 / size
    out_ref_host = out.cpu() if not args.no_e2e else None
    del chk, perm, out
    torch.cuda.empty_cache()

    def step():
        comp(fields, stream, sync=False)
        dec(comp.out, size, stream, check=False)

    # the stream size is data-dependent but fixed for this input: decompress
    # reads exactly `size` bytes of the compressor's output buffer
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for ws in (comp.ws, dec.ws):
        st = gpz.gpz_sync_status(ws)
        if st != gpz.OK:
            raise gpz.GpzError(st, "warm-up")

    gpz.gpz_set_stage_timing(True)
    gpz.gpz_stage_times()  # clear
    gpz.gpz_launch_count(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = gpz.gpz_launch_count()
    stages = gpz.gpz_stage_times()
    gpz.gpz_set_stage_timing(False)
    elapsed_ms = ev0.elapsed_time(ev1)
    for ws in (comp.ws, dec.ws):
        st = gpz.gpz_sync_status(ws)
        if st != gpz.OK:
            raise gpz.GpzError(st, "timed region")

    elapsed_ms = ranks_max([elapsed_ms], dev)[0]
    in_bytes = 4.0 * n * F
    value = job_gbs(world, in_bytes, args.steps, elapsed_ms / 1e3)

    comp_ms = sum(stages[k][0] for k in ("range", "info", "qse", "scan", "compact") if k in stages) / args.steps
    dec_ms = stages.get("decompress", (0.0, 1))[0] / args.steps

    # roofline of each kernel: algorithmic bytes per launch / mean launch time
    peak, peak_kind = load_peaks()
    payload_bytes = size - 4 * (16 + 2 * F + (n + 1023) // 1024 + 1)
    algo = {
        "range": in_bytes,                       # one read of every field
        "info": 8.0 * (F + 1) * ((n + 1023) // 1024),  # read each block's extremes, write its widths
        "qse": in_bytes + payload_bytes,         # read the input, write the encoded blocks
        "scan": 8.0 * ((n + 1023) // 1024),      # read sizes, write offsets
        "compact": 2.0 * payload_bytes,          # read temporary blocks, write the stream
        "decompress": size + in_bytes,           # read the stream, write every value
    }
    kernels = {}
    for k, (tot, cnt) in stages.items():
        if cnt == 0:
            continue
        mean_s = tot / cnt / 1e3
        ach = algo.get(k, 0.0) / mean_s / 1e9
        kernels[k] = {"mean_ms": 1e3 * mean_s, "launches": cnt, "algorithmic_bytes": algo.get(k),
                      "achieved_gbs": ach, "frac": ach / peak}
    dom = max(kernels, key=lambda k: kernels[k]["mean_ms"])
    step_bytes = sum(algo[k] for k in ("range", "qse", "decompress")) + size  # stream written once by compaction
    # with a relative bound the fused kernel is the variant that reads the range pass's block extremes
    kname = "gpz_qse_pre_kernel" if dom == "qse" else "gpz_%s_kernel" % dom
    roofline = {"bound": "hbm", "kernel": kname, "achieved": kernels[dom]["achieved_gbs"],
                "peak": peak, "unit": "GB/s", "frac": kernels[dom]["frac"],
                "traffic": recorded_traffic(dom), "peak_source": peak_kind,
                "note": "frac of %s copy bandwidth" % peak_kind,
                "frac_of_nominal": kernels[dom]["achieved_gbs"] / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS}

    result = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "fields": F, "eb_mode": "rel", "eb": REL_EB,
                   "seg_bits": SEG_BITS, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs (%.2f GB) larger than L2 (129 MB); no flush" % (in_bytes / 1e9)},
        "compress_gbs": in_bytes / (comp_ms / 1e3) / 1e9 if comp_ms else None,
        "decompress_gbs": in_bytes / (dec_ms / 1e3) / 1e9 if dec_ms else None,
        "ratio": ratio, "psnr_db": psnr, "max_err_over_eb": worst, "stream_bytes": size,
        "step_roofline_frac": (step_bytes / (elapsed_ms / args.steps / 1e3) / 1e9) / peak,
        "roofline": roofline, "kernels": kernels, "gpu_launches": launches,
        "clocks": clk.summary(),
    }

    # the fused compaction (blocks placed from the fused kernel by a
    # decoupled look-back over blocks) on the same workload, against the
    # three-step form timed above; the stream must be the same bytes
    if not args.no_fused:
        ref_stream = comp.out[:size].clone()
        comp.params.flags = gpz.FLAG_FUSED_COMPACTION  # this compressor's later calls only
        try:
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            kf = min(args.steps, 60)
            gpz.gpz_set_stage_timing(True)
            gpz.gpz_stage_times()
            ev0.record(stream)
            for _ in range(kf):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
            st_f = gpz.gpz_stage_times()
            gpz.gpz_set_stage_timing(False)
            deferred = gpz.compress_deferred_blocks(comp.ws)
            same = bool(torch.equal(comp.out[:size], ref_stream))
        finally:
            comp.params.flags = 0
        ms_f = ranks_max([ev0.elapsed_time(ev1) / kf], dev)[0]
        result["fused_compaction"] = {
            "value": job_gbs(world, in_bytes, 1, ms_f / 1e3), "unit": "GB/s", "ms_per_step": ms_f, "steps": kf,
            "stage_ms": {k: v[0] / max(v[1], 1) for k, v in st_f.items()},
            "blocks_not_placed": deferred, "blocks": (n + 1023) // 1024, "same_stream": same}
        del ref_stream

    # interleaved records (gpz_compress_aos / gpz_decompress_aos: a transpose
    # around the same kernels) on the same snapshot, particle-major
    if not args.no_aos:
        import ctypes as C
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
        hs = gpz._stream_handle(stream)

        def aos_step():
            st1 = gpz.lib.gpz_compress_aos(x_aos.data_ptr(), n, C.byref(params), a_out.data_ptr(), cap,
                                           a_size.data_ptr(), None, None, a_cws.data_ptr(), cws, hs)
            st2 = gpz.lib.gpz_decompress_aos(a_out.data_ptr(), size, a_rec.data_ptr(), F, n, a_dws.data_ptr(), dws,
                                             hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "aos round trip")

        for _ in range(args.warmup):
            aos_step()
        torch.cuda.synchronize()
        same_aos = int(a_size.item()) == size and bool(torch.equal(a_out[:size], comp.out[:size]))
        ka = min(args.steps, 60)
        gpz.gpz_set_stage_timing(True)
        gpz.gpz_stage_times()
        ev0.record(stream)
        for _ in range(ka):
            aos_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        st_a = gpz.gpz_stage_times()
        gpz.gpz_set_stage_timing(False)
        for wsb in (a_cws, a_dws):
            stc = gpz.gpz_sync_status(wsb)
            if stc != gpz.OK:
                raise gpz.GpzError(stc, "aos round trip (device)")
        ms_a = ranks_max([ev0.elapsed_time(ev1) / ka], dev)[0]
        tr = st_a.get("aos", (0.0, 1))
        result["aos"] = {"value": job_gbs(world, in_bytes, 1, ms_a / 1e3), "unit": "GB/s", "ms_per_step": ms_a,
                         "steps": ka, "transpose_ms": tr[0] / max(tr[1], 1),
                         "transpose_gbs": 2 * in_bytes / (tr[0] / max(tr[1], 1)) / 1e6 if tr[0] else None,
                         "same_stream": same_aos,
                         "records_checked": bool(torch.equal(a_rec.t(), dec(comp.out, size)))}
        del x_aos, a_out, a_cws, a_dws, a_rec

    # fp64 input and output (gpz_compress_f64 / gpz_decompress_f64: a rounding
    # pass and a widening pass around the same kernels) on the snapshot
    # widened to fp64; GB/s of fp64 input
    if not args.no_f64:
        import ctypes as C
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
        hs = gpz._stream_handle(stream)
        h_sz = C.c_uint64(0)

        def f64_step():
            st1 = gpz.lib.gpz_compress_f64(in_ptrs, n, C.byref(params), f_out.data_ptr(), cap, f_size.data_ptr(),
                                           C.byref(h_sz), None, f_cws.data_ptr(), cws, None, hs)
            st2 = gpz.lib.gpz_decompress_f64(f_out.data_ptr(), h_sz.value, out_ptrs, F, n, f_dws.data_ptr(), dws, hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "fp64 round trip")

        for _ in range(args.warmup):
            f64_step()
        torch.cuda.synchronize()
        kf = min(args.steps, 30)
        gpz.gpz_set_stage_timing(True)
        gpz.gpz_stage_times()
        ev0.record(stream)
        for _ in range(kf):
            f64_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        st_f = gpz.gpz_stage_times()
        gpz.gpz_set_stage_timing(False)
        stc = gpz.gpz_sync_status(f_dws)
        if stc != gpz.OK:
            raise gpz.GpzError(stc, "fp64 round trip (device)")
        ms_f = ranks_max([ev0.elapsed_time(ev1) / kf], dev)[0]
        # every sampled value within the bound of its fp64 input: |x - x^| <= eb' + max rounding error
        used = (C.c_double * F)()
        gpz.lib.gpz_compress_f64(in_ptrs, n, C.byref(params), f_out.data_ptr(), cap, None, C.byref(h_sz), None,
                                 f_cws.data_ptr(), cws, used, hs)
        result["f64"] = {"value": job_gbs(world, 8.0 * n * F, 1, ms_f / 1e3), "unit": "GB/s of fp64 input",
                         "ms_per_step": ms_f, "steps": kf, "ratio_vs_fp64": 8.0 * n * F / h_sz.value,
                         "stage_ms": {k: v[0] / max(v[1], 1) for k, v in st_f.items()},
                         "eb_reduced": [used[f] for f in range(F)]}
        del x64, f_out, f_cws, f_dws, f_rec

    # 64-bit intermediates (gpz_compress_wide / gpz_decompress_wide) on the
    # snapshot widened to fp64 with a relative bound of 1e-12, which fp32
    # cannot hold; the absolute bounds come from one relative call, then every
    # timed step runs without a host synchronisation; GB/s of fp64 input
    if not args.no_wide:
        import ctypes as C
        x64 = x.double()
        wide_rel = 1e-12
        cap = gpz.gpz_bound_size_wide(n, F)
        w_out = torch.empty(cap, dtype=torch.uint8, device=dev)
        w_size = torch.zeros(1, dtype=torch.int64, device=dev)
        cws = int(gpz.lib.gpz_compress_wide_workspace_size(n, F))
        w_cws = torch.empty(cws, dtype=torch.uint8, device=dev)
        w_dws = torch.zeros(256, dtype=torch.uint8, device=dev)
        w_rec = torch.empty((F, n), dtype=torch.float64, device=dev)
        in_ptrs = gpz._ptr_array([x64[f] for f in range(F)])
        out_ptrs = gpz._ptr_array([w_rec[f] for f in range(F)])
        hs = gpz._stream_handle(stream)
        h_sz = C.c_uint64(0)
        used = (C.c_double * F)()
        rel_params = gpz.make_params(F, wide_rel, gpz.EB_REL, SEG_BITS)
        st = gpz.lib.gpz_compress_wide(in_ptrs, n, C.byref(rel_params), w_out.data_ptr(), cap, None, C.byref(h_sz),
                                       None, w_cws.data_ptr(), cws, used, hs)
        if st != gpz.OK:
            raise gpz.GpzError(st, "gpz_compress_wide")
        params = gpz.make_params(F, [used[f] for f in range(F)], gpz.EB_ABS, SEG_BITS)

        def wide_step():
            st1 = gpz.lib.gpz_compress_wide(in_ptrs, n, C.byref(params), w_out.data_ptr(), cap, w_size.data_ptr(),
                                            None, None, w_cws.data_ptr(), cws, None, hs)
            st2 = gpz.lib.gpz_decompress_wide(w_out.data_ptr(), cap, out_ptrs, F, n, w_dws.data_ptr(), 256, hs)
            if st1 != gpz.OK or st2 != gpz.OK:
                raise gpz.GpzError(st1 or st2, "64-bit round trip")

        for _ in range(args.warmup):
            wide_step()
        torch.cuda.synchronize()
        kw = min(args.steps, 20)
        gpz.gpz_set_stage_timing(True)
        gpz.gpz_stage_times()
        ev0.record(stream)
        for _ in range(kw):
            wide_step()
        ev1.record(stream)
        torch.cuda.synchronize()
        st_w = gpz.gpz_stage_times()
        gpz.gpz_set_stage_timing(False)
        stc = gpz.gpz_sync_status(w_dws)
        if stc != gpz.OK:
            raise gpz.GpzError(stc, "64-bit round trip (device)")
        ms_w = ranks_max([ev0.elapsed_time(ev1) / kw], dev)[0]
        wsize = int(w_size.item())
        # the bound on every value, in fp64 (x reordered by a permutation from one more call)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        gpz.lib.gpz_compress_wide(in_ptrs, n, C.byref(params), w_out.data_ptr(), cap, None, C.byref(h_sz),
                                  perm.data_ptr(), w_cws.data_ptr(), cws, None, hs)
        gpz.lib.gpz_decompress_wide(w_out.data_ptr(), cap, out_ptrs, F, n, w_dws.data_ptr(), 256, hs)
        torch.cuda.synchronize()
        pl = perm.long()
        worst = max(float(((x64[f][pl] - w_rec[f]).abs().max() / used[f]).item()) for f in range(F))
        result["wide"] = {"value": job_gbs(world, 8.0 * n * F, 1, ms_w / 1e3), "unit": "GB/s of fp64 input",
                          "ms_per_step": ms_w, "steps": kw, "rel_eb": wide_rel,
                          "ratio_vs_fp64": 8.0 * n * F / wsize, "max_err_over_eb": worst,
                          "stage_ms": {k: v[0] / max(v[1], 1) for k, v in st_w.items()}}
        del x64, w_out, w_cws, w_dws, w_rec, perm

    # end to end through the public API with host buffers: H2D input ->
    # compress -> D2H stream -> H2D stream -> decompress -> D2H output, every
    # step.  Timed twice: one step after another on one stream, and pipelined
    # (two buffer sets; the next step's uploads overlap this step's downloads
    # and kernels on separate copy and compute streams), the form a user
    # streaming snapshots through the library would run.
    if not args.no_e2e:
        h_in = torch.empty((F, n), dtype=torch.float32, pin_memory=True)
        h_in.copy_(x)
        k = max(3, min(20, args.steps // 10))

        # (a) one step after another
        h_stream = torch.empty(comp.capacity, dtype=torch.uint8, pin_memory=True)
        h_out = torch.empty((F, n), dtype=torch.float32, pin_memory=True)
        d_in = torch.empty_like(x)
        d_stream = torch.empty_like(comp.out)

        def e2e_step():
            d_in.copy_(h_in, non_blocking=True)
            sz = comp([d_in[f] for f in range(F)], stream, sync=True)
            h_stream[:sz].copy_(comp.out[:sz], non_blocking=True)
            d_stream[:sz].copy_(h_stream[:sz], non_blocking=True)
            o = dec(d_stream, sz, stream, check=False)
            h_out.copy_(o, non_blocking=True)
            return sz

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            sz = e2e_step()
        torch.cuda.synchronize()
        dt_seq = (time.perf_counter() - t0) / k
        del h_stream, h_out, d_in, d_stream
        del comp, dec
        torch.cuda.empty_cache()

        # (b) pipelined: buffer set j = i % 2 per step i
        # uploads, kernels, downloads
        s_up, s_run, s_down = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        sets = []
        for j in range(2):
            c_ = gpz.Compressor(n, F, REL_EB, gpz.EB_REL, SEG_BITS, want_perm=False, device=dev)
            sets.append({"comp": c_, "dec": gpz.Decompressor(n, F, device=dev), "d_in": torch.empty_like(x),
                         "d_stream": torch.empty_like(c_.out),
                         "h_stream": torch.empty(c_.capacity, dtype=torch.uint8, pin_memory=True),
                         "h_out": torch.empty((F, n), dtype=torch.float32, pin_memory=True),
                         "h_size": torch.zeros(1, dtype=torch.int64, pin_memory=True),
                         "in_ready": torch.cuda.Event(), "in_free": torch.cuda.Event(),
                         "size_ready": torch.cuda.Event(), "stream_down": torch.cuda.Event(),
                         "stream_up": torch.cuda.Event(), "decoded": torch.cuda.Event(), "out_down": torch.cuda.Event()})
        for b in sets:  # nothing to wait for at the start
            for name in ("in_free", "stream_down", "decoded", "out_down"):
                b[name].record(s_run)

        def upload_input(i):
            b = sets[i % 2]
            s_up.wait_event(b["in_free"])
            with torch.cuda.stream(s_up):
                b["d_in"].copy_(h_in, non_blocking=True)
            b["in_ready"].record(s_up)

        def run_pipelined(steps):
            upload_input(0)
            for i in range(steps):
                b = sets[i % 2]
                s_run.wait_event(b["in_ready"])
                s_run.wait_event(b["stream_down"])  # the previous use of this set's output buffer is on the host
                b["comp"]([b["d_in"][f] for f in range(F)], s_run, sync=False)
                b["in_free"].record(s_run)
                with torch.cuda.stream(s_run):
                    b["h_size"].copy_(b["comp"].d_size, non_blocking=True)
                b["size_ready"].record(s_run)
                if i + 1 < steps:
                    upload_input(i + 1)  # overlaps this step's downloads and kernels
                b["size_ready"].synchronize()
                sz_ = int(b["h_size"].item())
                s_down.wait_event(b["size_ready"])
                with torch.cuda.stream(s_down):
                    b["h_stream"][:sz_].copy_(b["comp"].out[:sz_], non_blocking=True)
                b["stream_down"].record(s_down)
                s_up.wait_event(b["stream_down"])
                s_up.wait_event(b["decoded"])  # the previous decode of this set has read d_stream
                with torch.cuda.stream(s_up):
                    b["d_stream"][:sz_].copy_(b["h_stream"][:sz_], non_blocking=True)
                b["stream_up"].record(s_up)
                s_run.wait_event(b["stream_up"])
                s_run.wait_event(b["out_down"])  # the previous output of this set is on the host
                o_ = b["dec"](b["d_stream"], sz_, s_run, check=False)
                b["decoded"].record(s_run)
                s_down.wait_event(b["decoded"])
                with torch.cuda.stream(s_down):
                    b["h_out"].copy_(o_, non_blocking=True)
                b["out_down"].record(s_down)
            return sz_

        run_pipelined(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sz = run_pipelined(k)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / k
        # the pipelined steps' outputs are the same values as the device path's
        ok_e2e = bool(torch.equal(sets[(k - 1) % 2]["h_out"], out_ref_host)) if out_ref_host is not None else None
        dt, dt_seq = ranks_max([dt, dt_seq], dev)
        result["e2e"] = {"value": job_gbs(world, in_bytes, 1, dt), "unit": "GB/s",
                         "h2d_bytes_per_step": int(in_bytes + sz), "d2h_bytes_per_step": int(in_bytes + sz + 8),
                         "ms_per_step": 1e3 * dt, "pipelined": True, "output_checked": ok_e2e,
                         "sequential": {"value": job_gbs(world, in_bytes, 1, dt_seq), "ms_per_step": 1e3 * dt_seq}}
        del sets, h_in

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, npart = host_sample(x, every=4)
        gbs1, tc, td = cpu_oracle_sample(sample, F)
        nthreads = os.cpu_count() or 1
        whole, _ = host_sample(x, every=1)
        gbs, dt, used = cpu_oracle_threads(whole, F, nthreads)
        result["cpu_baseline"] = {
            "value": gbs, "unit": "GB/s", "cores": used, "kind": "oracle",
            "sample": "the whole snapshot (%d particles x 6 fields), one compress + decompress, the C++ oracle "
                      "over %d host threads by contiguous block ranges, relative eb over the snapshot; %.1f s"
                      % (whole.shape[1], used, dt),
            "single_thread": {"value": gbs1, "cores": 1,
                              "sample": "every 4th 1024-particle block (%d particles x 6 fields), relative eb "
                                        "over the sample; %.1f s" % (npart, tc + td)}}
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ----------------------------------------------------------------------------- batched workload

def run_batched(args):
    """Batched compress + decompress of many uneven chunks: the persistent
    batched plans (tuned, replayed as CUDA graphs) against one call per chunk."""
    import ctypes as C
    import torch
    from paper_2508_10305_gb300 import build
    build.build()
    from paper_2508_10305_gb300 import gpz, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
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

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    if args.batched_only:
        ms = timed(batched_step, args.steps, args.warmup)
        print(json.dumps({"workload": "batched (plans only, default shapes)", "chunks": wl.count,
                          "input_gb": in_bytes / 1e9, "ms_per_step": ms,
                          "gbs": in_bytes / (ms / 1e3) / 1e9}), flush=True)
        return

    # tuned launch shapes (the outputs are rewritten with the same bytes)
    ccfg, cms = bc.tune(reps=2)
    dcfg, dms = bd.tune(reps=2)

    # parity: every chunk's stream equals its single-call stream; sampled
    # small chunks equal the CPU oracle's; every value decodes within eb
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
        x = torch.stack(wl.fields(c)).cpu().numpy()
        rs, _ = gpz_oracle.compress(x, [wl.rel[c]] * wl.F[c], 1, SEG_BITS, want_perm=False)
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
        batched_ms = timed(batched_step, args.steps, args.warmup)
    launches = gpz.gpz_launch_count() // max(1, args.steps + args.warmup)
    pc_steps = max(1, min(3, args.steps))
    per_chunk_ms = timed(lambda: per_chunk_step(sh), pc_steps, 1)
    per_chunk_launches = (gpz.gpz_launch_count(reset=True) - launches * (args.steps + args.warmup)) // (pc_steps + 1)
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
    gpz.gpz_set_stage_timing(True)
    gpz.gpz_stage_times()
    bc.use_graph = bd.use_graph = False
    for _ in range(2):
        batched_step()
    torch.cuda.synchronize()
    stages = gpz.gpz_stage_times(16)
    gpz.gpz_set_stage_timing(False)
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
    line = {
        "metric": "batched compress+decompress GB/s (graph-replayed batched plans vs one call per chunk)",
        "value": in_bytes / (batched_ms / 1e3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": batched_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched: %d chunks, particles log-uniform in [%d, %d] (total %d), 3 fields "
                               "(uniform box) or 6 (cosmology-like), relative eb 1e-3 / 1e-4, G = 3"
                               % (wl.count, args.chunk_lo, args.chunk_hi, sum(wl.n)),
                   "input_gb": in_bytes / 1e9, "l2": "inputs larger than L2; no flush"},
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
    bc.close()
    bd.close()
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- served workload

SERVED_GENS = [("uniform box", 3, 1e-2, 0), ("cosmology-like", 6, 1e-4, 1), ("LiDAR-like", 3, 1e-3, 0)]


def run_served(args):
    """Real-time replay of a Poisson request trace against the serving engine:
    continuous batching (two lanes, up to 64 requests per batch) against the
    plain path (one lane, one request per launch sequence)."""
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
    t_arr, size, gen, op = synth.request_trace(args.requests, rate=args.rate, lo=100_000, hi=64_000_000, seed=5)
    rng = np.random.default_rng(6)
    reqs = []
    for i in range(args.requests):
        g, F = int(gen[i]), SERVED_GENS[int(gen[i])][1]
        if op[i] == 0:
            n = int(size[i])
            off = int(rng.integers(0, (pool_n - n) // 32 + 1)) * 32
            reqs.append((0, g, F, n, off))
        else:
            n = int(classes[np.argmin(np.abs(np.log(classes) - np.log(size[i])))])
            reqs.append((1, g, F, n, 0))
    raw_bytes = sum(4 * r[3] * r[2] for r in reqs)

    def arm(lanes, max_batch, batch_mb, lane_mb):
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
            return float(np.percentile(a, q)) if a.size else None
        return {
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(lat.mean()),
            "compress_p50_ms": pct(lat[kinds == 0], 50), "compress_p99_ms": pct(lat[kinds == 0], 99),
            "decompress_p50_ms": pct(lat[kinds == 1], 50), "decompress_p99_ms": pct(lat[kinds == 1], 99),
            "aggregate_gbs": raw_bytes / span / 1e9, "span_s": span, "all_ok": ok,
            "batches": stats["batches"], "mean_batch": float(bsz.mean()), "max_batch": int(bsz.max()),
            "arena_peak_gb": stats["arena_peak"] / 1e9, "submit_lag_p99_ms": 1e3 * float(np.percentile(lag, 99)),
            "sampled_equal_single_call": equal, "sampled": len(checks), "lanes": lanes, "max_batch_cfg": max_batch,
            "max_batch_mb": batch_mb, "express_lane_mb": lane_mb,
        }

    arms = {}
    with ClockSampler(0) as clk:
        for spec in args.serve_arms.split(","):
            name, lanes, mb, bmb, lmb = spec.split(":")
            arms[name] = arm(int(lanes), int(mb), float(bmb), float(lmb))
    names = list(arms)
    batched, plain = arms[names[0]], arms.get("plain", arms[names[-1]])
    offered = raw_bytes / float(t_arr[-1]) / 1e9
    line = {
        "metric": "served p50/p99 latency (ms) and aggregate GB/s: continuous batching vs plain path",
        "value": batched["p99_ms"], "unit": "ms (p99 latency)", "n_gpus": 1, "steps": args.requests, "warmup": 6,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "served: Poisson %d requests/s, %d requests, 100K-64M particles log-uniform, "
                               "generators uniform box (3 fields, abs 1e-2) / cosmology-like (6, rel 1e-4) / "
                               "LiDAR-like (3, abs 1e-3), half compress, half decompress (resident streams of 16 "
                               "size classes)" % (args.rate, args.requests),
                   "budget_gb": args.budget_gb, "offered_gbs": offered, "raw_gb": raw_bytes / 1e9},
        "served_arm": names[0], "arms": arms,
        "p99_speedup_vs_plain": plain["p99_ms"] / batched["p99_ms"],
        "p50_speedup_vs_plain": plain["p50_ms"] / batched["p50_ms"],
        "clocks": clk.summary(), "prepare_s": prep_s,
    }
    print(json.dumps(line), flush=True)


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
            run_batched(args)
    elif args.workload == "served":
        if rank == 0:
            run_served(args)
    elif args.workload == "sweep":
        if rank == 0:
            run_sweep(args)
    else:
        run_gpz(args, rank, world, local)


if __name__ == "__main__":
    main()
