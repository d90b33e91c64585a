"""The benchmark's multi-rank path on CPU: two gloo ranks through the same
set-up, barrier, max-over-ranks and replica aggregation that bench.py runs
under torchrun (no GPU involved)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_setup(world)
    seconds = 1.0 + 0.5 * r                     # ranks finish at different times
    bench.barrier_sync(w)
    t_max = bench.max_over_ranks(seconds, w)
    q.put((r, w, local, t_max, bench.replica_value(100.0, t_max, w)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_and_replica_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[3] == pytest.approx(1.5) for g in got)          # the slowest rank's time
    assert all(g[4] == pytest.approx(100.0 * 2 / 1.5) for g in got)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_value(10.0, 2.0, 1) == 5.0


def test_solve_launch_count():
    """gpu_launches: per solve the init kernel, the sweeps as launched (four per graph
    pass, four per host-loop batch, capped at max_iters by the host loop only), with
    their pre-kernels, and the extraction sweep."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.solve_launches([22] * 10, False, 5000, 1) == 10 * (1 + 24 + 1)   # sweeps 23, 24 empty
    assert bench.solve_launches([19], False, 5000, 1) == 1 + 20 + 1
    assert bench.solve_launches([19], True, 5000, 1) == 1 + 20 + 1
    assert bench.solve_launches([22], True, 5000, 1) == 1 + 24 + 1
    assert bench.solve_launches([5], True, 5, 1) == 1 + 5 + 1                 # capped at max_iters
    assert bench.solve_launches([5], False, 5, 1) == 1 + 8 + 1                # the graph body runs whole
    assert bench.solve_launches([15], False, 5000, 3) == 1 + (16 + 1) * 3     # two pre-kernels per sweep
    assert bench.solve_launches([0], False, 0, 1) == 1 + 0 + 1               # extraction only
