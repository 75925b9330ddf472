"""The asynchronous global-server step: device merge of owners' host lists, and the whole step on one
GPU against the plain detect and the oracle."""
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


@pytest.mark.parametrize("k,cap,out_cap", [(1, 64, 64), (3, 500, 2000), (8, 1024, 10000), (4, 300, 700)])
def test_merge_hosts_sorted_union(C, k, cap, out_cap):
    """k sorted lists of disjoint addresses (some empty, some longer than their block holds) merge into
    the sorted union; counts add up; a merged list longer than the output reports CAPACITY."""
    import torch
    rng = np.random.default_rng(5 + k)
    allips = rng.choice(1 << 32, size=k * cap, replace=False).astype(np.uint32)
    parts = np.array_split(allips, k)
    blocks = np.zeros((k, cap), dtype=C.HOST_DTYPE)
    infos = np.zeros((k, 8), dtype=np.int32)
    kept = []
    for j, p in enumerate(parts):
        n = [0, len(p), len(p) // 2, len(p) + 5][j % 4]          # empty, full, half, more than the block
        h = np.sort(p[:min(n, cap)])
        blocks[j]["ip"][:h.size] = h
        blocks[j]["z"][:h.size] = j
        blocks[j]["est"][:h.size] = np.arange(h.size, dtype=np.float32)
        infos[j, 1] = n                                         # n_hosts (may exceed the block)
        infos[j, 0] = C.ERR_CAPACITY if n > cap else C.OK       # as the range detect reports it
        infos[j, 2], infos[j, 3] = j + 1, 10 * j
        kept.append(blocks[j][:h.size])
    want = np.sort(np.concatenate(kept), order="ip")
    dev_blocks = torch.from_numpy(blocks.view(np.int32).reshape(k, 4 * cap).copy()).cuda()
    dev_infos = torch.from_numpy(infos).cuda()
    out = torch.zeros(4 * out_cap, dtype=torch.int32, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    C.merge_hosts(dev_blocks, dev_infos, out, info)
    hosts, inf = C.hosts_from_device(out, info)
    placed = min(want.size, out_cap)                            # records a block overflow left out are not there
    assert np.array_equal(hosts[:placed], want[:placed])
    assert inf["n_hosts"] == int(infos[:, 1].sum()) and inf["n_hot"] == int(infos[:, 2].sum())
    overflow = bool((infos[:, 1] > cap).any()) or int(infos[:, 1].sum()) > out_cap
    assert inf["status"] == (C.ERR_CAPACITY if overflow else C.OK)


def test_async_step_on_one_rank_matches_plain_and_oracle(C, oracle):
    """World of one: enqueue() on a side stream, two windows double-buffered, no host wait until the end;
    each slot's host list equals the plain detect's and the oracle's."""
    import torch
    from paper_1901_06207_b300.shard import ShardedDetector
    d, theta = GEO.TINY2, 128
    wins = []
    for seed in (0xA5, 0xA6):
        spec = T.TrafficSpec(n_packets=1 << 17, n_hosts=3000, n_planted=150, planted_lo=160, planted_hi=900,
                             planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=64, seed=seed)
        wins.append(T.make_window(spec).pairs)
    det = ShardedDetector(d, theta, 0, 1, cap=1 << 12)
    cubes = [C.Cube(d) for _ in range(2)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for b, pairs in enumerate(wins):
            cubes[b].update(torch.from_numpy(pairs.view(np.int32)).cuda())
            det.enqueue(cubes[b], b)
    torch.cuda.current_stream().wait_stream(side)
    for b, pairs in enumerate(wins):
        hosts, info = det.result(b)
        assert info["status"] == C.OK
        want = oracle.detect(d, oracle.build_cube(d, pairs), theta)["hosts"]
        assert hosts.size == want.size > 0
        assert np.array_equal(hosts["ip"], want["ip"]) and np.array_equal(hosts["z"], want["z"])
        assert np.array_equal(hosts, cubes[b].detect(theta))
