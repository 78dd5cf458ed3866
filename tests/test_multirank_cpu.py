"""Two-rank host logic of bench.py on CPU (gloo): the ranks take disjoint
wave-vector batches that tile the path, and the step time is the maximum over
ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    nk, kps = 64, 2
    mine = [bench.k_indices(s, rank, ws, kps, nk) for s in range(16)]
    gathered = [None] * ws
    dist.all_gather_object(gathered, mine)
    t = bench.max_over_ranks(ws, 1.0 + rank)
    dist.barrier()
    if rank == 0:
        q.put((gathered, t))
    dist.destroy_process_group()


def test_two_ranks_disjoint_batches_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 2.0
    for s in range(16):
        a, b = set(gathered[0][s]), set(gathered[1][s])
        assert not (a & b)
    # 16 steps x 2 ranks x 2 k = 64 distinct indices: the whole path once
    allk = [k for r in range(2) for s in range(16) for k in gathered[r][s]]
    assert sorted(allk) == list(range(64))
