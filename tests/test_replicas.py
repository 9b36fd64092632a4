"""The multi-process parts of bench.py on the CPU: the max-over-ranks timing and
whole-job rate of the replica runs (two gloo ranks), and the reference arm, which
only rank 0 runs."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_rate(10.0 * (rank + 1), 1000, world, device="cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in res:
        assert ms == 20.0                       # the slower rank's time on both
        assert value == pytest.approx(2 * 1000 / 0.020)  # both ranks' units


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(4.0, 100, 1) == (4.0, 100 / 0.004)


def _reference(env_rank):
    env = dict(os.environ, RANK=str(env_rank), WORLD_SIZE="2", LOCAL_RANK=str(env_rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0", "--ref-n", "8", "--workload", "wave"],
                          capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_rank0_prints_one_line_other_ranks_exit():
    r0, r1 = _reference(0), _reference(1)
    assert r0.returncode == 0 and r1.returncode == 0, r0.stderr + r1.stderr
    assert r1.stdout.strip() == ""
    lines = [ln for ln in r0.stdout.strip().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "cell-updates/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
