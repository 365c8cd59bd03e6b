"""Host logic of the multi-GPU benchmark path, on CPU with the gloo backend
(two ranks): every rank runs its own replica, the job time is the slowest
rank's, and the whole-job rate counts the units of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.ranks()
        local_seconds = 1.5 + rank            # rank 1 is the slowest
        t = bench.max_over_ranks(local_seconds, "cpu")
        out.put((r, w, lr, t, bench.job_rate(1000, 10, w, t)))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_reduce_to_the_slowest_and_count_every_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == 2.5                       # max over ranks, seen by every rank
        assert r[4] == pytest.approx(1e-6 * 1000 * 10 * 2 / 2.5)


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not tdist.is_initialized()
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(2e6, 5, 1, 2.0) == pytest.approx(5.0)
