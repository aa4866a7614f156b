"""The multi-GPU form is replicas only (every rank advances its own domain, no data-path
collective): the bench's cross-rank timing (barrier + max of the ranks' times) and its
whole-job rate, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = max_t = bench.max_over_ranks(torch, dist, 1.5 + rank, device="cpu")
    out[rank] = (t, bench.job_rate(1000, 10, ws, max_t))
    dist.destroy_process_group()


def test_two_replicas_time_is_the_slowest_rank_and_rate_counts_both():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5          # both ranks see the slower rank's time
    assert res[0][1] == res[1][1] == 1000 * 10 * 2 / 2.5 / 1e6
