"""Batched router windows replayed from one CUDA graph against the oracle and the plain path."""
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


def _windows(n_windows, n_routers, n_packets):
    out = []
    for w in range(n_windows):
        spec = T.TrafficSpec(n_packets=n_packets, n_hosts=3000, n_planted=150, planted_lo=160, planted_hi=900,
                             planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=64, seed=0xBA70 + w)
        out.append(T.router_window(spec, n_routers))
    return out


def test_graph_batched_windows_match_oracle_and_plain(C, oracle):
    import torch
    from paper_1901_06207_b300.batch import RouterWindows
    d, theta, R = GEO.TINY2, 128, 5
    wins = _windows(3, R, 1 << 17)
    dev = []
    for pairs, counts, _ in wins:
        p = torch.from_numpy(pairs.view(np.int32)).cuda()
        bounds = np.concatenate([[0], np.cumsum(counts)])
        dev.append([p[bounds[j]:bounds[j + 1]] if counts[j] else None for j in range(R)])
    rw = RouterWindows(d, R, theta, max_pairs=1 << 17, n_windows=len(wins))
    rw.capture(dev)
    for _ in range(2):                                  # replays are repeatable
        rw.replay()
        res = rw.results()
        for w, (pairs, counts, _) in enumerate(wins):
            hosts, info = res[w]
            assert info["status"] == C.OK
            want = oracle.detect(d, oracle.build_cube(d, pairs), theta)["hosts"]
            assert hosts.size == want.size and np.array_equal(hosts["ip"], want["ip"])
            assert np.array_equal(hosts["z"], want["z"]) and np.array_equal(hosts["flags"], want["flags"])
            assert np.allclose(hosts["est"], want["est"], rtol=1e-6)
            plain = C.Cube(d)                            # the plain single-cube path, no graph
            plain.update(torch.from_numpy(pairs.view(np.int32)).cuda())
            assert np.array_equal(plain.detect(theta), hosts)
    # the router cubes hold the last window's per-router traffic
    pairs, counts, _ = wins[-1]
    bounds = np.concatenate([[0], np.cumsum(counts)])
    for j in range(R):
        assert np.array_equal(rw.routers[j].to_numpy(), oracle.build_cube(d, pairs[bounds[j]:bounds[j + 1]]))


def test_full_size_router_windows(C, oracle):
    """The batched benchmark's configuration: 16M-packet windows of the 64M shape over 8 routers with
    lognormal loads, the L2 geometry, the tuned tiling, one graph; every window's host list and the
    last window's router cubes against the oracle (4 windows: both global buffers, twice)."""
    import os
    import torch
    from paper_1901_06207_b300.batch import RouterWindows
    d, theta, R = GEO.L2, 1024, 8
    wins = [T.router_window(T.spec_window_64m(seed=0xC0FFEE20 + w, scale_shift=2), R)[:2] for w in range(4)]
    dev = []
    for pairs, counts in wins:
        p = torch.from_numpy(pairs.view(np.int32)).cuda()
        b = np.concatenate([[0], np.cumsum(counts)])
        dev.append([p[b[j]:b[j + 1]] if counts[j] else None for j in range(R)])
    base = C.get_tuning()
    try:
        rw = RouterWindows(d, R, theta, max_pairs=max(int(c.sum()) for _, c in wins), n_windows=len(wins))
        rw.tune(dev)
        rw.capture(dev)
        rw.replay()
        res = rw.results()
    finally:
        C.set_tuning(**base)
    threads = max(1, min(os.cpu_count() or 1, 16))
    for w, (pairs, counts) in enumerate(wins):
        hosts, info = res[w]
        assert info["status"] == C.OK
        want = oracle.detect(d, oracle.update_threads(d, oracle.new_cube(d), pairs, threads), theta)["hosts"]
        assert hosts.size == want.size and np.array_equal(hosts["ip"], want["ip"])
        assert np.array_equal(hosts["z"], want["z"]) and np.array_equal(hosts["flags"], want["flags"])
        assert np.allclose(hosts["est"], want["est"], rtol=1e-6)
    pairs, counts = wins[-1]
    b = np.concatenate([[0], np.cumsum(counts)])
    for j in range(R):
        assert np.array_equal(rw.routers[j].to_numpy(), oracle.build_cube(d, pairs[b[j]:b[j + 1]]))
