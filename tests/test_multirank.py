"""The multi-GPU host logic of bench.py on CPU ranks (gloo, world size 2).

The path shards by replicas only (every rank renders its own frame, no data
exchange), so what runs across ranks is the host side: the maximum of the
per-rank step times (a step lasts as long as the slowest rank), the job
throughput that counts every rank's samples, and the reference arm, which
only rank 0 runs and prints.  Ranks are separate processes rendezvousing on
127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = dist.get_rank()
t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
v = bench.job_msamples_per_s(dist.get_world_size(), 2_000_000, 10, t)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "max": t, "value": v}}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    e = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
             MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    e.pop("CUDA_VISIBLE_DEVICES", None)
    return e


def test_max_over_ranks_and_job_throughput_on_two_gloo_ranks():
    port = _free_port()
    code = WORKER.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 2.5  # the slower rank's time, on every rank
        assert abs(o["value"] - 2 * 2_000_000 * 10 / 2.5 / 1e6) < 1e-9


def test_reference_arm_prints_on_rank_zero_only():
    args = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
            "--steps", "1", "--warmup", "3", "--ref-samples", "4", "--workload", "small"]
    port = _free_port()
    res = [subprocess.run(args, env=_env(r, 2, port), capture_output=True, text=True, timeout=600,
                          cwd=ROOT) for r in range(2)]
    assert res[0].returncode == 0, res[0].stderr
    assert res[1].returncode == 0, res[1].stderr
    assert res[1].stdout.strip() == ""
    line = json.loads(res[0].stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
