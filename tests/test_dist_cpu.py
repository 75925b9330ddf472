"""bench.py's multi-rank host logic on CPU: two gloo ranks, no GPU.

Under torchrun each rank processes its own window (weak scaling, no
collective on the data path); the step time is the maximum over ranks and
the packet count the sum.  These are the only collectives, checked here.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    t = bench.reduce_over_ranks(10.0 + 5.0 * r, w, "max")        # step times of the ranks
    n = bench.reduce_over_ranks(1000.0 * (r + 1), w, "sum")      # packets of the ranks
    spec0 = bench.T.spec_window_64m(scale_shift=10)
    spec = spec0 if r == 0 else bench.T.TrafficSpec(**{**spec0.__dict__, "seed": spec0.seed + 0x100 * r})
    out[r] = (r, w, local, t, n, spec.seed)
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(120) if hasattr(pytest.mark, "timeout") else (lambda f: f)
def test_two_gloo_ranks_max_and_sum():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert set(out.keys()) == {0, 1}
    for r in (0, 1):
        rank, world, local, t, n, seed = out[r]
        assert (rank, world, local) == (r, 2, r)
        assert t == 15.0          # max over ranks
        assert n == 3000.0        # sum over ranks
    assert out[0][5] != out[1][5]  # each rank its own window


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_over_ranks(3.5, 1, "max") == 3.5
    assert bench.reduce_over_ranks(3.5, 1, "sum") == 3.5
    bench.barrier(1)
