"""The N > 1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1 (one process per
GPU on a GPU node; here the ranks have no GPU).  Checks that the slowest rank's time is
what every rank reports, that the whole-job rate counts every rank's units over that
time, that each rank draws its own seeded right-hand side, and that the reference arm
runs on rank 0 only (the other ranks exit without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    import tg_inputs as gi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    bench.rank_barrier(world, dev)
    local_ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    ms = bench.max_over_ranks_of(local_ms, world, dev)
    rate = bench.weak_scaling_rate(1, ms, world)
    b = gi.rhs(1000, seed=rank)
    out[rank] = (ms, rate, float(b[:8].sum()))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_max_time_and_rate():
    port = _free_port()
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    assert res[0][0] == res[1][0] == 150.0                      # every rank sees the slowest time
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1000.0 / 150.0)
    assert res[0][2] != res[1][2]                               # per-rank seeded inputs


def test_reference_arm_runs_on_rank_zero_only():
    """A non-zero rank of the reference arm exits 0 without output or work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
