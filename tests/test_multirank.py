"""The replicas-only multi-GPU path of bench.py, on the CPU: two gloo ranks on
127.0.0.1 each time their own replica (one image each, no collective on the
data path); every rank ends with the slowest rank's time and the whole-job
throughput ranks x megapixels / slowest time (weak scaling), and each replica
draws its own landmarks."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [4.0, 6.5][rank]
    ms_max, value = bench.weak_scaling_value(ms, 2.0736, world, "cpu", dist)
    dist.barrier()
    q.put((rank, ms_max, value, bench.replica_seed(100, rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, ms_max, value, seed in res:
        assert ms_max == 6.5
        assert abs(value - 2 * 2.0736 / 6.5e-3) < 1e-9
    assert [r[3] for r in res] == [100, 101]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.weak_scaling_value(5.0, 2.0736, 1, "cpu")
    assert ms_max == 5.0 and abs(value - 2.0736 / 5e-3) < 1e-9
