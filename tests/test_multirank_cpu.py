"""Host logic of the multi-replica benchmark on 2 gloo ranks (CPU only): the job time is the
maximum over ranks and the whole-job throughput sums the replicas' work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.dist_env()
    ms = bench.reduce_max(1.0 + rank * 2.5, w, device="cpu")
    q.put((r, w, lr, ms))
    dist.destroy_process_group()


def test_reduce_max_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert all(o[3] == 3.5 for o in out)


def test_step_bytes_formula():
    import bench
    sp, pk = bench.step_bytes(M=10, nnz=20, R=5, N=4, sz=4)
    assert sp == 11 * 8 + 20 * 8 + 5 * 4 * 4 + 10 * 4 * 4
    assert pk == 2 * 5 * 4 * 4 + 5 * 4
