"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the
whole-job rate uses the slowest rank's time and every rank's particles, and
under a multi-rank launch only rank 0 of the reference arm does any work."""
import os
import socket
import subprocess
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=2)
    try:
        ms = (10.0, 20.0)[rank]
        particles = (100.0, 300.0)[rank]
        out[rank] = bench.aggregate_ranks(ms, particles, 5, 2, "cpu")
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms_max, p_all, value = res[r]
        assert ms_max == 20.0 and p_all == 400.0
        assert abs(value - 400.0 * 5 / 0.020) < 1e-6 * value


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
