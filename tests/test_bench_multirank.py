"""The multi-rank path of bench.py on CPU: two gloo ranks.

bench.py --gpus N runs one replica of the workload per rank (the primaries of different
ranks are independent, no data-path collective); the only collective is the maximum of the
per-rank timings, and rank 0 reports primaries of all ranks over that maximum.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, timings, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, e2e = bench.max_over_ranks(timings[rank], world)
    out.put((rank, ms, e2e, bench.aggregate_rate(200_000, world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_replicas():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    timings = [[18.0, 19.5], [21.0, 19.0]]   # (device ms, end-to-end ms) of each rank
    procs = [mp.Process(target=_rank, args=(r, 2, port, timings, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, rate in got:
        assert ms == 21.0 and e2e == 19.5
        assert rate == pytest.approx(2 * 200_000 / 21e-3)


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun every rank starts bench.py; the oracle (reference arm) runs on rank 0
    # alone and the other ranks exit 0 without output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
