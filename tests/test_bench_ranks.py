"""Host-side logic of bench.py's N-GPU form, on CPU (gloo, world size 2, 127.0.0.1).

The N-rank bench runs independent replicas (the path does not shard): every rank times its own steps
between barriers, the job's time per step is the maximum over ranks, rank 0 alone prints, and the
reference arm does its work on rank 0 only while the other ranks exit without work.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r's step times: r + 1 and 5 - r seconds
        t = bench.max_over_ranks([rank + 1.0, 5.0 - rank], world, "cpu")
        dist.barrier()
        out[rank] = t.tolist()
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_maximum_over_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        got = dict(out)
    assert got[0] == got[1] == [2.0, 5.0]


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert np.array_equal(bench.max_over_ranks([0.5, 0.25], 1, "cpu"), [0.5, 0.25])


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_roofline_arithmetic():
    """achieved = algorithmic bytes per launch / mean launch time; frac = achieved / measured peak; the
    dominant class is the one with the most device time; traffic comes from the capture table."""
    sys.path.insert(0, ROOT)
    import bench
    tot = {("dslash", 2): [1000, 20.0, 1000 * 2.0e6],   # 20 us per launch, 2 MB each -> 100 GB/s
           ("vector", 1): [500, 5.0, 500 * 1.0e6]}
    roof, shares = bench.shares_and_roofline(tot, {"hbm_gbs": 5000.0}, traffic={("dslash", 2): 1.5e6})
    assert roof["kernel"] == "dslash/f16" and roof["launches"] == 1000
    assert abs(roof["avg_us"] - 20.0) < 1e-9 and abs(roof["achieved"] - 100.0) < 1e-6
    assert abs(roof["frac"] - 0.02) < 1e-9 and roof["peak"] == 5000.0 and roof["traffic"] == 1.5e6
    assert abs(shares["dslash/f16"]["share"] - 0.8) < 1e-9 and abs(shares["vector/f32"]["share"] - 0.2) < 1e-9
    roof, _ = bench.shares_and_roofline({("vector", 1): [10, 1.0, 1e7]}, {"hbm_gbs": 5000.0})
    assert roof["traffic"] is None
