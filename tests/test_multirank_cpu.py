"""The N>1 path of the benchmark on CPU ranks (gloo, world size 2).

Several GPUs run independent replicas: each rank reconstructs its own specimen,
the only exchange is the timing reduction (maximum over ranks) and the barrier
around the timed region. These tests run that host logic on two CPU processes,
and run the benchmark's reference arm under torch.distributed.run with two
ranks (rank 0 alone measures and prints, the other exits 0 without work).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2401_11101_gb300 import inputs as I
    # rank r measured (r + 1) ms for one form and (10 - r) ms for the other
    t = bench.max_over_ranks([rank + 1.0, 10.0 - rank], "cpu")
    dist.barrier()
    geom, _, d = I.make_projections("c1", slab=rank)
    res = {"t": t, "value": bench.job_gvox_s(geom.nvox, world, t[0]),
           "d_sum": float(d.double().sum()), "d_first": d.flatten()[:8].tolist()}
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_timing_reduction_and_replica_inputs_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # both ranks hold the element-wise maximum: the slowest rank sets the time
    for r in res:
        assert r["t"] == [2.0, 10.0]
    # whole-job throughput counts the voxels of every rank over that time
    nvox = 64 * 64 * 64
    assert abs(res[0]["value"] - world * nvox / 2e-3 / 1e9) < 1e-12
    assert res[0]["value"] == res[1]["value"]
    # each replica reconstructs its own specimen
    assert res[0]["d_first"] != res[1]["d_first"]
    # rank 0's specimen is the single-GPU workload itself
    from paper_2401_11101_gb300 import inputs as I
    _, _, d0 = I.make_projections("c1")
    assert np.isclose(float(d0.double().sum()), res[0]["d_sum"], rtol=0, atol=0)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
           "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "GVox/s"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
