"""shard.py's collective steps on CPU with two and four gloo ranks, no GPU.

The sketch exchange must leave in each rank's own slice the OR of every
rank's copy of that slice, and the host-list gather must return every
rank's hosts merged by ip.  The OR is injected here as a plain torch
bitwise OR on CPU tensors (on a GPU it is cbaa_or_words).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _words(rank, n):
    rng = np.random.default_rng(100 + rank)
    return (rng.integers(0, 1 << 32, n, dtype=np.uint64) & rng.integers(0, 1 << 32, n, dtype=np.uint64)) \
        .astype(np.uint32)


def _hosts(rank, k):
    from paper_1901_06207_b300 import cbaa as C
    h = np.zeros(k, dtype=C.HOST_DTYPE)
    h["ip"] = (np.arange(k, dtype=np.uint32) * 7919 + rank) * 4 + rank     # disjoint across ranks
    h["z"] = rank
    h["est"] = 1000.0 + rank
    return h


def _rank_main(rank, world, port, words, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_1901_06207_b300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mem = torch.from_numpy(_words(rank, words).view(np.int32).copy())
    recv = torch.empty_like(mem)

    def or_fn(dst, srcs):
        for s in srcs:
            dst.bitwise_or_(s)

    own = shard.exchange_slices(mem, rank, world, recv, or_fn)
    got = shard.gather_hosts(_hosts(rank, 3 + 5 * rank), rank, world, "cpu")
    # the asynchronous path's gather: fixed-capacity blocks and info words, tensor to tensor
    cap = 16
    block = torch.zeros(4 * cap, dtype=torch.int32)
    h = _hosts(rank, 3 + 5 * rank)[:cap]
    block[:4 * h.size] = torch.from_numpy(h.view(np.int32).copy())
    info = torch.tensor([0, h.size, rank, 0, 0, 0, 0, 0], dtype=torch.int32)
    blocks = torch.zeros((world, 4 * cap), dtype=torch.int32)
    infos = torch.zeros((world, 8), dtype=torch.int32)
    shard.gather_blocks(block, info, blocks, infos, world)
    out[rank] = (own.numpy().view(np.uint32).copy(), got, blocks.numpy().copy(), infos.numpy().copy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_exchange_and_gather(world):
    words = 4096
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, words, out), nprocs=world, join=True)
    per = words // world
    full = np.zeros(words, dtype=np.uint32)
    for r in range(world):
        full |= _words(r, words)
    want_hosts = np.sort(np.concatenate([_hosts(r, 3 + 5 * r) for r in range(world)]), order="ip")
    for r in range(world):
        own, got, blocks, infos = out[r]
        assert np.array_equal(own, full[r * per:(r + 1) * per]), r
        assert np.array_equal(got, want_hosts), r
        for j in range(world):                    # every rank holds every rank's block and count
            hj = _hosts(j, 3 + 5 * j)[:16]
            assert infos[j, 1] == hj.size and infos[j, 2] == j
            assert np.array_equal(blocks[j].view(np.uint8).view(want_hosts.dtype)[:hj.size], hj)


def test_owned_ranges_partition_the_sketches():
    from paper_1901_06207_b300 import shard
    geo = {"r": 5}
    for world in (1, 2, 4, 8, 16, 32):
        spans = [shard.owned_range(geo, k, world) for k in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == 32
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    with pytest.raises(ValueError):
        shard.owned_range(geo, 0, 3)


def _fail_main(rank, world, port, mode, out):
    """Rank 1 fails before the sketch exchange (exits, or stalls past the group's timeout); rank 0
    must come back from the exchange with an error instead of waiting forever."""
    import datetime
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_1901_06207_b300 import shard
    def group():
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=3))

    if rank == 1:
        try:
            group()
        except Exception:  # noqa: BLE001 -- the failing rank's own errors do not matter
            pass
        if mode == "stall":
            time.sleep(8)                                  # alive, but never joins the exchange
        os._exit(0)                                        # gone mid-window, no goodbye
    t0 = time.perf_counter()
    try:                                                   # rank 1 may already be gone during the setup
        group()
        mem = torch.from_numpy(_words(rank, 1024).view(np.int32).copy())
        recv = torch.empty_like(mem)
        shard.exchange_slices(mem, rank, world, recv, lambda d, srcs: None)
        out[0] = ("no error", time.perf_counter() - t0)
    except Exception as e:  # noqa: BLE001 -- any collective error is the detection
        out[0] = (type(e).__name__, time.perf_counter() - t0)
    os._exit(0)


@pytest.mark.parametrize("mode", ["exit", "stall"])
def test_failed_rank_is_detected_on_the_host(mode):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_fail_main, args=(2, port, mode, out), nprocs=2, join=True)
    what, waited = out[0]
    assert what != "no error", what
    assert waited < 10.0, waited
