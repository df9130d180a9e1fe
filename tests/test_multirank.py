"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica closing its own work, and
the whole-job aggregation (max time over ranks, summed work) that bench.py reports."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank          # rank 1 is slower
    work_local = 1000.0 * (rank + 1)
    ms, work = bench.aggregate(ms_local, work_local)
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (150.0, 3000.0)


def test_single_process_aggregation_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(12.5, 7.0) == (12.5, 7.0)
