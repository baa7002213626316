"""The N>1 benchmark path is replicas only (one independent problem per GPU,
no data-path collective).  Its only cross-rank step, the max over ranks of the
timed region and the whole-job value, runs here as two gloo ranks on CPU."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, e2e = bench.job_times(100.0 + 50.0 * rank, 7.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, e2e, bench.job_value(world, 1.0e12, ms)))
    dist.destroy_process_group()


def test_two_replicas_take_the_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == 150.0 and r[2] == 14.0 for r in res)
    assert abs(res[0][3] - 2.0 / 0.150) < 1e-12
