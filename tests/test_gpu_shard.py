"""Sketch-sharded merge and restoration on one GPU, with the ranks emulated in one process.

Each emulated rank holds the router cube of its share of the packets.  The
owner of sketches [lo, hi) ORs the other ranks' copies of that slice into
its own (cbaa_or_words, what the all-to-all delivers) and restores only its
sketches (cbaa_detect_range_async).  The owners' host lists together must
equal the detect of one cube holding every packet, and the oracle's.  No
collective runs here: the exchange is plain slicing of device tensors.
"""
import numpy as np
import pytest

import geometries as GEO
from paper_1901_06207_b300 import traffic as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_06207_b300 import build
    build.build()
    from paper_1901_06207_b300 import cbaa
    return cbaa


def _dev(pairs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).cuda()


def _range_hosts(C, cube, lo, hi, theta, ws):
    import torch
    out = torch.zeros(4 * (1 << 16), dtype=torch.int32, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    cube.detect_range_async(lo, hi, theta, ws, out, info)
    hosts, inf = C.hosts_from_device(out, info)
    assert inf["status"] == C.OK
    return hosts


@pytest.mark.parametrize("geo,theta", [("L2", 1024), ("TINY2", 128)])
def test_ranges_cover_the_full_detect(C, geo, theta):
    d = GEO.ALL[geo]
    w = T.make_window(T.spec_window_64m(scale_shift=4)) if geo == "L2" else \
        T.make_window(T.TrafficSpec(n_packets=1 << 18, n_hosts=3000, n_planted=200, planted_lo=150,
                                    planted_hi=700, planted_dist="uniform", bg_mode="per_host", zipf_a=1.2,
                                    bg_max=64, seed=0x5A1D))
    cube = C.Cube(d)
    cube.update(_dev(w.pairs))
    ws = C.Workspace(d)
    full = cube.detect(theta, ws=ws)
    S = 1 << d["r"]
    for parts in (1, 2, 4, 8):
        per = S // parts
        got = np.concatenate([_range_hosts(C, cube, k * per, (k + 1) * per, theta, ws) for k in range(parts)])
        assert np.array_equal(np.sort(got, order="ip"), full), parts
    with pytest.raises(C.CbaaError):
        _range_hosts(C, cube, 3, 3, theta, ws)
    with pytest.raises(C.CbaaError):
        _range_hosts(C, cube, 0, S + 1, theta, ws)


@pytest.mark.parametrize("world", [2, 4])
def test_emulated_ranks_equal_one_cube_and_oracle(C, oracle, world):
    from paper_1901_06207_b300 import shard
    d, theta = GEO.L2, 1024
    w = T.make_window(T.spec_window_64m(scale_shift=4))
    rid, _ = T.split_by_router(w.pairs, 77, world)
    cubes = [C.Cube(d) for _ in range(world)]
    for k in range(world):
        cubes[k].update(_dev(w.pairs[rid == k]))
    words = cubes[0].memory.numel()
    per = words // world
    ws = C.Workspace(d)
    lists = []
    for k in range(world):                     # owner k: OR the others' copies of its slice, restore it
        own = cubes[k].memory[k * per:(k + 1) * per]
        C.or_words(own, [cubes[j].memory[k * per:(k + 1) * per] for j in range(world) if j != k])
        lo, hi = shard.owned_range(d, k, world)
        lists.append(_range_hosts(C, cubes[k], lo, hi, theta, ws))
    got = np.sort(np.concatenate(lists), order="ip")
    one = C.Cube(d)
    one.update(_dev(w.pairs))
    assert np.array_equal(got, one.detect(theta, ws=ws))
    want = oracle.detect(d, oracle.build_cube(d, w.pairs), theta)["hosts"]
    assert np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z"], want["z"])


def test_or_words_arguments(C):
    import torch
    a = torch.zeros(64, dtype=torch.int32, device="cuda")
    b = torch.full((64,), 5, dtype=torch.int32, device="cuda")
    C.or_words(a, [b, b])
    assert int(a.sum().item()) == 5 * 64
    C.or_words(a, [])
    with pytest.raises(C.CbaaError):
        C.or_words(a, [a])                     # dst among srcs
    with pytest.raises(C.CbaaError):
        C.or_words(a[1:], [b[1:]])             # 63 words: not a multiple of 4, not 16-byte aligned
