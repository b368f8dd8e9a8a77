"""The multi-GPU (N > 1) host path of bench.py, run as world-size-2 gloo
ranks on the CPU: every rank merges its own replica (weak scaling, no
data-path collective), the step time is the max over ranks, and the
whole-job rate counts every rank's units; the reference arm runs on rank 0
only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [3.0, 5.0][rank]
    worst = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.weak_scaling_value(1000, worst, world)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"worst": worst, "value": value}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value(tmp_path):
    port = _free_port()
    ctx = tmp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert res[0] == res[1]
    assert res[0]["worst"] == 5.0
    # 2 ranks x 1000 units in 5 ms = 4e5 units/s = 4e-4 G units/s.
    assert abs(res[0]["value"] - 2 * 1000 / 5e-3 / 1e9) < 1e-12


def test_reference_arm_only_rank0_prints():
    """Under torchrun the reference arm runs on rank 0; other ranks exit 0
    without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--log2-a", "12", "--log2-b", "10"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--log2-a", "12", "--log2-b", "10"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
