"""Continuous-batching serving: every (tenant, window) result is the same alone and in the mix."""
import numpy as np
import pytest

import geometries as GEO
from paper_1901_06207_b300 import traffic as T

pytestmark = pytest.mark.gpu
THETA = 128


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_06207_b300 import build
    build.build()
    from paper_1901_06207_b300 import cbaa
    return cbaa


def _traffic(tenant, window):
    spec = T.TrafficSpec(n_packets=(1 << 17) + 4099 * tenant, n_hosts=3000, n_planted=120, planted_lo=160,
                         planted_hi=900, planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=64,
                         seed=0x5E00 + 16 * tenant + window)
    return T.make_window(spec).pairs


def _batches(pairs, seed):
    """Uneven batch sizes, log-uniform in [2^10, 2^15]."""
    rng = np.random.default_rng(seed)
    out, i = [], 0
    while i < pairs.shape[0]:
        n = int(np.exp(rng.uniform(np.log(1 << 10), np.log(1 << 15))))
        out.append(pairs[i:i + n])
        i += n
    return out


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).pin_memory()


def _run(C, tenants, windows, n_slots, n_cubes, interleave_seed=None):
    from paper_1901_06207_b300.serve import Server
    srv = Server(GEO.TINY2, THETA, n_slots=n_slots, slot_pairs=1 << 15, n_cubes=n_cubes, cap=1 << 12)
    streams = {t: [(w, b) for w in range(windows) for b in _batches(_traffic(t, w), 100 * t + w)] for t in tenants}
    order = [t for t in tenants for _ in streams[t]]
    if interleave_seed is not None:
        np.random.default_rng(interleave_seed).shuffle(order)
    pos = {t: 0 for t in tenants}
    for t in order:                       # each tenant's batches stay in order; tenants interleave
        w, b = streams[t][pos[t]]
        pos[t] += 1
        srv.submit(t, w, _pinned(b))
        if pos[t] == len(streams[t]) or streams[t][pos[t]][0] != w:
            srv.close(t, w)
    res = srv.drain(timeout_s=120)
    return {(r.tenant, r.window): r for r in res}, srv


def test_serving_results_same_alone_and_mixed(C, oracle):
    tenants, windows = [0, 1, 2], 2
    alone = {}
    for t in tenants:
        r, _ = _run(C, [t], windows, n_slots=2, n_cubes=2)
        alone.update(r)
    mixed, srv = _run(C, tenants, windows, n_slots=3, n_cubes=2, interleave_seed=7)
    assert set(mixed) == set(alone) == {(t, w) for t in tenants for w in range(windows)}
    for key, r in mixed.items():
        a = alone[key]
        assert r.info["status"] == C.OK and a.info["status"] == C.OK
        assert r.packets == a.packets
        assert np.array_equal(r.hosts, a.hosts), key            # bit-exact, estimates included
        t, w = key
        want = oracle.detect(GEO.TINY2, oracle.build_cube(GEO.TINY2, _traffic(t, w)), THETA)["hosts"]
        assert np.array_equal(r.hosts["ip"], want["ip"]) and np.array_equal(r.hosts["z"], want["z"])
        assert r.latency_s >= 0
    # memory-based admission: two cubes for three tenants -- never more in use, and windows had to wait
    assert srv.stats["max_cubes_in_use"] <= 2
    assert srv.stats["queued_for_cube"] > 0


def test_queued_batches_share_a_slot_update(C, oracle):
    """A burst queued at once: batches of one window join the admitted one in its slot while they fit
    (one update for several batches), never across a window's close; results equal the oracle's."""
    from paper_1901_06207_b300.serve import Server
    srv = Server(GEO.TINY2, THETA, n_slots=2, slot_pairs=1 << 16, n_cubes=2, cap=1 << 12)
    for w in range(2):
        for b in _batches(_traffic(0, w), 900 + w):
            srv.submit(0, w, _pinned(b), poll=False)
        srv.close(0, w, poll=False)
    res = {r.window: r for r in srv.drain(timeout_s=120)}
    assert set(res) == {0, 1}
    assert srv.stats["updates"] < srv.stats["batches"]
    for w in range(2):
        pairs = _traffic(0, w)
        assert res[w].packets == pairs.shape[0] and res[w].info["status"] == C.OK
        want = oracle.detect(GEO.TINY2, oracle.build_cube(GEO.TINY2, pairs), THETA)["hosts"]
        assert np.array_equal(res[w].hosts["ip"], want["ip"]) and np.array_equal(res[w].hosts["z"], want["z"])


def test_close_without_batches_yields_an_empty_result(C, oracle):
    """A window closed without any batch still yields a result: the detect of an empty cube (no
    packets, no hosts, status OK), even while another window of the tenant is open; a close for a window
    that a newer window's batch already closed adds nothing."""
    from paper_1901_06207_b300.serve import Server
    srv = Server(GEO.TINY2, THETA, n_slots=2, slot_pairs=1 << 16, n_cubes=2, cap=1 << 12)
    pairs0, pairs2 = _traffic(0, 0), _traffic(0, 2)
    srv.close(0, 5)                                   # nothing open, never seen: empty result
    for b in _batches(pairs0, 700):
        srv.submit(0, 0, _pinned(b))
    srv.close(0, 1)                                   # window 0 stays open; window 1 got nothing
    for b in _batches(pairs2, 702):                   # window 2's first batch closes window 0
        srv.submit(0, 2, _pinned(b))
    srv.close(0, 0)                                   # already closed by window 2: no second result
    srv.close(0, 2)
    res = srv.drain(timeout_s=120)
    got = sorted((r.window, r.packets, r.hosts.size) for r in res)
    want0 = oracle.detect(GEO.TINY2, oracle.build_cube(GEO.TINY2, pairs0), THETA)["hosts"]
    want2 = oracle.detect(GEO.TINY2, oracle.build_cube(GEO.TINY2, pairs2), THETA)["hosts"]
    assert [w for w, _, _ in got] == [0, 1, 2, 5]
    by = {r.window: r for r in res}
    for w in (1, 5):
        assert by[w].packets == 0 and by[w].hosts.size == 0 and by[w].info["status"] == C.OK
    assert want0.size > 0 and np.array_equal(by[0].hosts["ip"], want0["ip"])
    assert np.array_equal(by[2].hosts["ip"], want2["ip"]) and by[2].packets == pairs2.shape[0]


def test_serving_budget_and_batch_limits(C):
    from paper_1901_06207_b300.serve import Server
    with pytest.raises(C.CbaaError):
        Server(GEO.TINY2, THETA, n_slots=2, slot_pairs=1 << 15, mem_budget=1 << 20)    # no room for a cube
    srv = Server(GEO.TINY2, THETA, n_slots=1, slot_pairs=1 << 10, n_cubes=1)
    with pytest.raises(C.CbaaError):
        srv.submit(0, 0, _pinned(np.zeros((2048, 2), np.uint32)))                     # larger than a slot


def test_full_size_serving_window(C, oracle):
    """The serving benchmark's configuration: the 64M-packet window of the core-network shape cut into
    batches log-uniform in [64Ki, 4Mi] pairs, served into the 256 MiB geometry (r=6, c=2^13) by 4 staging
    slots of 4Mi pairs and 4 cubes as one window; host list against the oracle's."""
    import os
    import torch
    from paper_1901_06207_b300.serve import Server
    d, theta = GEO.SERVE, 1024
    pairs = T.make_window(T.spec_window_64m(seed=0xC0FFEE30)).pairs
    pool = torch.from_numpy(pairs.view(np.int32)).pin_memory()
    rng = np.random.default_rng(0x5E7E)
    srv = Server(d, theta, n_slots=4, slot_pairs=4 << 20, n_cubes=4)
    off = 0
    while off < pairs.shape[0]:
        n = int(np.exp(rng.uniform(np.log(1 << 16), np.log(4 << 20))))
        srv.submit(0, 0, pool[off:off + n])
        off += n
    srv.close(0, 0)
    res = srv.drain(timeout_s=300)
    assert len(res) == 1 and res[0].packets == pairs.shape[0] and res[0].info["status"] == C.OK
    threads = max(1, min(os.cpu_count() or 1, 8))                # 8 private 256 MiB cubes on the host
    want = oracle.detect(d, oracle.update_threads(d, oracle.new_cube(d), pairs, threads), theta)["hosts"]
    got = res[0].hosts
    assert got.size == want.size and got.size > 0
    assert np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z"], want["z"])
    assert np.array_equal(got["flags"], want["flags"]) and np.allclose(got["est"], want["est"], rtol=1e-6)
