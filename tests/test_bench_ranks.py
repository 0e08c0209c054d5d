"""Host logic of bench.py's replica runs (one process per GPU under torchrun): the timed region's
length is the slowest rank's (all-reduce MAX), and the whole-job time per source divides it by the
sources all ranks solved.  Two gloo ranks on the CPU stand in for two GPUs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        t = bench.max_over_ranks(1.0 + 2.5 * rank, w, "cpu")  # the ranks' step times differ
        v = bench.job_seconds_per_source(t, 4, w)
        with open(os.path.join(out, "rank%d.txt" % rank), "w") as f:
            f.write("%d %d %d %r %r\n" % (r, w, local, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for rank in range(2):
        r, w, local, t, v = open(tmp_path / ("rank%d.txt" % rank)).read().split()
        assert (int(r), int(w), int(local)) == (rank, 2, rank)
        assert float(t) == 3.5                 # max over ranks, seen by both
        assert float(v) == 3.5 / (4 * 2)       # 4 sources on each of 2 ranks


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.0, 1) == 2.0
    assert bench.job_seconds_per_source(2.0, 4, 1) == 0.5


def test_cpu_baseline_host_facts_and_all_cores_leg():
    sys.path.insert(0, ROOT)
    import bench
    info = bench.host_info()
    assert info["nproc"] >= 1 and info["cpu_model"]
    r = bench.oracle_all_cores(4, 100)  # a 4^3 sample in every process
    assert 1 <= r["processes"] <= info["nproc"]
    assert r["value"] == pytest.approx(r["per_process_s"] / r["processes"])
