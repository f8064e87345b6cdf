"""The N > 1 bookkeeping of bench.py on CPU ranks (gloo, world size 2): every rank filters the
same per-rank work (weak scaling, no data-path collective), the job time is the slowest
rank's (one MAX all-reduce), and the whole-job value counts the pixels of all ranks."""
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


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [0.010, 0.025][rank]          # rank 1 is the slow one
    value, job_s = bench._job_rate(3.0e6, 4, local, world, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(f"{value!r} {job_s!r}")
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [tuple(float(v) for v in open(tmp_path / f"r{r}.txt").read().split()) for r in range(2)]
    assert vals[0] == vals[1]                       # every rank reports the same job figures
    value, job_s = vals[0]
    assert job_s == pytest.approx(0.025)           # the slowest rank
    assert value == pytest.approx(2 * 3.0e6 * 4 / 0.025 / 1e6)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, job_s = bench._job_rate(1.0e6, 10, 0.5, 1)
    assert (value, job_s) == (pytest.approx(20.0), 0.5)
