"""The benchmark's multi-rank path on CPU: two processes over the gloo
backend (the GPU run uses one process per GPU over NCCL; the host logic is
the same).  Ranks are replicas: each draws its own snapshot, no collective
touches the data, and the job's time is the slowest rank's."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = {"env": list(bench.dist_env())}
    # the slowest rank's time, element by element
    r["max"] = bench.ranks_max([1.0 + rank, 10.0 - rank, 0.5], "cpu")
    # each rank's own snapshot: identical shape, different values
    x = bench.make_workload(4096, rank, "cpu")
    sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(sums, x.double().sum().reshape(1))
    r["sums"] = [float(s.item()) for s in sums]
    r["shape"] = list(x.shape)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, "rank%d.json" % rank), "w") as fh:
        json.dump(r, fh)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in range(world):
        assert res[r]["env"] == [r, world, 0]
        assert res[r]["max"] == [2.0, 10.0, 0.5]
        assert res[r]["shape"] == [6, 4096]
        assert res[r]["sums"] == res[0]["sums"]
    assert res[0]["sums"][0] != res[0]["sums"][1]


def test_job_throughput_is_weak_scaling():
    import bench
    one = bench.job_gbs(1, 1.6e9, 10, 0.02)
    assert one == pytest.approx(800.0)
    # two ranks, same per-rank work, slowest rank 10% slower: 2 x 1.6 GB x 10 / 0.022 s
    assert bench.job_gbs(2, 1.6e9, 10, 0.022) == pytest.approx(2 * 800.0 / 1.1)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class A:
        n, steps, warmup, gpus = 4096, 1, 0, 2
    bench.run_reference(A, 1, 2)  # rank 1: no work, no output
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    """Rank 0 of the reference arm times the oracle on a sample of the
    snapshot and prints one JSON line with the same metric, unit and config
    as the GPU arm, marked as the reference, with its CPU baseline and an
    e2e object of zero transfer bytes."""
    import json
    import bench
    from oracle import build as oracle_build
    oracle_build.build()

    class A:
        n, steps, warmup, gpus = 1 << 16, 1, 0, 1
    bench.run_reference(A, 0, 1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GB/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["config"]["workload"] == bench.WORKLOAD and line["config"]["n"] == 1 << 16
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_encodes_the_gpu_arms_blocks():
    """The reference arm turns the relative bound into absolute bounds over
    the whole snapshot (bench.absolute_bounds) before compressing its block
    samples, so every sampled block is encoded word for word as in the
    stream of the whole snapshot with the relative bound -- the stream the
    GPU arm writes.  Checked with the oracle on a small snapshot, and the
    reference line's config is the GPU arm's."""
    import numpy as np
    import bench
    from oracle import gpz_oracle as o
    from paper_2508_10305_gb300 import synth
    x = synth.cosmology(1 << 15, seed=2).numpy()
    F, n = x.shape
    whole, _ = o.compress(x, bench.REL_EB, 1, bench.SEG_BITS)
    ebs = bench.absolute_bounds(x, bench.REL_EB)
    blocks = np.arange(1, n // 1024, 5)
    sel = (blocks[:, None] * 1024 + np.arange(1024)[None, :]).reshape(-1)
    part, _ = o.compress(np.ascontiguousarray(x[:, sel]), ebs, 0, bench.SEG_BITS)
    w, p = whole.view(np.uint32), part.view(np.uint32)
    nb, nbp = n // 1024, blocks.size
    tw, tp = w[16 + 2 * F:16 + 2 * F + nb + 1], p[16 + 2 * F:16 + 2 * F + nbp + 1]
    pw, pp = w[16 + 2 * F + nb + 1:], p[16 + 2 * F + nbp + 1:]
    for k, b in enumerate(blocks):
        assert np.array_equal(pw[tw[b]:tw[b + 1]], pp[tp[k]:tp[k + 1]]), b
    assert w[16:16 + 2 * F].tolist() == p[16:16 + 2 * F].tolist()  # eb and step of every field
    assert bench.gpu_config(1 << 26, 1)["workload"] == bench.WORKLOAD
