"""GPU parity: the CUDA path against the CPU oracle on the same seeded inputs.

Bar: cubes, per-column zero counts, Zmax and host lists (ip, Z, flags) are
bit-exact; eps is the same IEEE double; FP32 estimates agree to a relative
1e-6 (both sides evaluate Thm. 2 in double and round once to float).
"""
import ctypes

import numpy as np
import pytest

import geometries as GEO
from paper_1901_06207_b300 import traffic as T

pytestmark = pytest.mark.gpu
EST_RTOL = 1e-6


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_06207_b300 import build
    build.build()
    from paper_1901_06207_b300 import cbaa
    return cbaa


def dev_pairs(pairs: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).cuda()


def tiny_window(seed, n=1 << 16, planted=40, lo=150, hi=600, hosts=2000, bg_max=60):
    spec = T.TrafficSpec(n_packets=n, n_hosts=hosts, n_planted=planted, planted_lo=lo, planted_hi=hi,
                         planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=bg_max, seed=seed)
    return T.make_window(spec)


def assert_hosts_equal(got: np.ndarray, want: np.ndarray):
    assert got.size == want.size, (got.size, want.size)
    assert np.array_equal(got["ip"], want["ip"])
    assert np.array_equal(got["z"], want["z"])
    assert np.array_equal(got["flags"], want["flags"])
    w = want["est"].astype(np.float64)
    g = got["est"].astype(np.float64)
    assert np.all(np.abs(g - w) <= EST_RTOL * np.maximum(np.abs(w), 1.0)), np.max(np.abs(g - w))


WINDOWS = {
    "tiny": lambda: tiny_window(31, n=1 << 18, planted=300, lo=150, hi=700, hosts=3000, bg_max=64),
    "tiny_sat": lambda: tiny_window(32, n=1 << 18, planted=200, lo=600, hi=3000, hosts=3000, bg_max=64),
    "1m": lambda: T.make_window(T.spec_window_1m()),
    "4m": lambda: T.make_window(T.spec_window_64m(scale_shift=4)),
}
_cache = {}


def window(name):
    if name not in _cache:
        _cache[name] = WINDOWS[name]()
    return _cache[name]


CUBE_CASES = [("TINY", "tiny"), ("TINY2", "tiny"), ("PAPER", "1m"), ("L2", "4m"), ("SERVE", "4m"),
              ("UNDERSIZED", "4m"), ("QUAD", "tiny"), ("DUO", "tiny")]


@pytest.mark.parametrize("geo,win", CUBE_CASES)
def test_update_cube_bit_exact(C, oracle, geo, win):
    d = GEO.ALL[geo]
    w = window(win)
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    got = cube.to_numpy()
    want = oracle.build_cube(d, w.pairs)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("geo,win", CUBE_CASES)
def test_binned_update_cube_bit_exact(C, oracle, geo, win):
    """The partitioned update sets exactly the bits of Alg. 1."""
    d = GEO.ALL[geo]
    w = window(win)
    cube = C.Cube(d)
    ws = C.UpdateWorkspace(d, w.pairs.shape[0])
    cube.update_binned(dev_pairs(w.pairs), ws)
    assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, w.pairs))


def test_binned_update_passes_ragged_and_incremental(C, oracle):
    """Small workspace (many passes), odd counts, 8-byte-aligned starts, on top of earlier bits."""
    import torch
    d = GEO.L2
    w = window("4m")
    p = dev_pairs(w.pairs)
    cube = C.Cube(d)
    half = 1_000_001
    cube.update(p, n=half)                                  # earlier bits from the direct path
    ws = C.UpdateWorkspace(d, 300_007)
    bounds = [half, half + 1, half + 8191, 2_500_003, w.pairs.shape[0]]
    for a, b in zip(bounds[:-1], bounds[1:]):
        cube.update_binned_ptr(p.data_ptr() + 8 * a, b - a, ws)
    torch.cuda.synchronize()
    assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, w.pairs))


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_binned_update_every_scatter_shape(C, oracle, shape, kind):
    """Launch shapes and tilings change timing only: every one gives the oracle's cube."""
    d = GEO.L2
    w = window("4m")
    before = C.get_tuning()
    try:
        C.set_tuning(scatter_shape=shape, count_blocks_per_sm=2 + shape, apply_items_per_sm=1 + 3 * shape,
                     tile_kind=kind)
        cube = C.Cube(d)
        cube.update_binned(dev_pairs(w.pairs), C.UpdateWorkspace(d, w.pairs.shape[0]))
        assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, w.pairs))
    finally:
        C.set_tuning(**before)


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("geo,win,k", [("TINY2", "tiny", 5), ("L2", "4m", 8), ("TINY", "tiny", 16),
                                       ("PAPER", "1m", 2), ("SERVE", "4m", 1)])
def test_multi_router_update(C, oracle, geo, win, k, kind):
    """One partitioned pass over k router cubes: each equals the oracle cube of its own packets."""
    before = C.get_tuning()
    C.set_tuning(**{**before, "tile_kind": kind})
    try:
        _multi_router_case(C, oracle, geo, win, k)
    finally:
        C.set_tuning(**before)


def _multi_router_case(C, oracle, geo, win, k):
    d = GEO.ALL[geo]
    w = window(win)
    rid, _ = T.split_by_router(w.pairs, 91, k)
    parts = [w.pairs[rid == j] for j in range(k)]
    cubes = [C.Cube(d) for _ in range(k)]
    ws = C.UpdateWorkspace(d, max(1, w.pairs.shape[0] // 3), n_cubes=k)     # several passes
    C.update_multi(cubes, [dev_pairs(p) if p.size else None for p in parts], ws)
    for j in range(k):
        assert np.array_equal(cubes[j].to_numpy(), oracle.build_cube(d, parts[j])), j
    glob = C.Cube(d)
    glob.merge(cubes)
    assert np.array_equal(glob.to_numpy(), oracle.build_cube(d, w.pairs))


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("geo,win,k", [("TINY2", "tiny", 5), ("L2", "4m", 8)])
def test_multi_router_update_merges_into_global(C, oracle, geo, win, k, kind):
    """cbaa_cube_update_multi_merge: each router cube is the oracle cube of its own packets, and the
    global cube -- holding earlier bits of its own -- gains exactly the OR of all router cubes (the
    merge of Section III.C done in the update pass); a small workspace forces several passes."""
    import torch
    d = GEO.ALL[geo]
    w = window(win)
    rid, _ = T.split_by_router(w.pairs, 93, k)
    parts = [w.pairs[rid == j] for j in range(k)]
    earlier = tiny_window(77, n=1 << 14).pairs
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "tile_kind": kind})
        cubes = [C.Cube(d) for _ in range(k)]
        glob = C.Cube(d)
        glob.update(dev_pairs(earlier))
        ws = C.UpdateWorkspace(d, max(1, w.pairs.shape[0] // 3), n_cubes=k)
        C.update_multi(cubes, [dev_pairs(p) if p.size else None for p in parts], ws, merge_into=glob)
        torch.cuda.synchronize()
    finally:
        C.set_tuning(**before)
    for j in range(k):
        assert np.array_equal(cubes[j].to_numpy(), oracle.build_cube(d, parts[j])), j
    assert np.array_equal(glob.to_numpy(), oracle.build_cube(d, np.concatenate([earlier, w.pairs])))


def test_multi_merge_rejects_bad_global(C):
    d = GEO.TINY
    cubes = [C.Cube(d) for _ in range(2)]
    pairs = [dev_pairs(tiny_window(78, n=1 << 10).pairs), None]
    ws = C.UpdateWorkspace(d, 1 << 10, n_cubes=2)
    with pytest.raises(C.CbaaError) as e:
        C.update_multi(cubes, pairs, ws, merge_into=cubes[1])            # a router cube itself
    assert e.value.status == C.ERR_INVALID_ARG
    with pytest.raises(C.CbaaError) as e:
        C.update_multi(cubes, pairs, ws, merge_into=C.Cube(GEO.TINY2))   # another structure
    assert e.value.status == C.ERR_GEOMETRY


@pytest.mark.parametrize("shape", [0, 6])
@pytest.mark.parametrize("kind", [2, 3])
def test_multi_router_segment_edges(C, oracle, shape, kind):
    """Router segments of 0, 1, 2 and about one routing block of packets (4096 or 8192): some
    blocks meet many segments, so the routing tables fall back to every cube's tiles, others meet
    one or two; every cube must still be the oracle's cube of its own packets."""
    d = GEO.TINY
    rng = np.random.default_rng(41)
    P = 4096 if shape == 0 else 8192
    lens = [1, 0, 2, 3, P - 1, 1, 1, P, P + 1, 2 * P + 5, 7, 5 * P, 1, 0, 3 * P - 2, 1]
    pairs = rng.integers(0, 2**32, size=(sum(lens), 2), dtype=np.uint64).astype(np.uint32)
    cut = np.concatenate([[0], np.cumsum(lens)])
    parts = [pairs[cut[j]:cut[j + 1]] for j in range(len(lens))]
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "tile_kind": kind, "scatter_shape": shape})
        cubes = [C.Cube(d) for _ in parts]
        C.update_multi(cubes, [dev_pairs(p) if p.shape[0] else None for p in parts],
                       C.UpdateWorkspace(d, pairs.shape[0], n_cubes=len(parts)))
        for j, p in enumerate(parts):
            assert np.array_equal(cubes[j].to_numpy(), oracle.build_cube(d, p)), j
    finally:
        C.set_tuning(**before)


@pytest.mark.parametrize("kind", [1, 2, 3])
@pytest.mark.parametrize("geo", ["L2", "PAPER"])
def test_binned_update_skewed_runs(C, oracle, geo, kind):
    """Half the packets one pair, a fifth one source to many peers: a few tiles take most of
    the records (tile runs of millions next to runs of a few), against the oracle's cube."""
    d = GEO.ALL[geo]
    rng = np.random.default_rng(11)
    n = 1_500_003
    pairs = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    pairs[: n // 2] = (0x0A000001, 0x0B000002)
    fan = slice(n // 2, n // 2 + n // 5)
    pairs[fan, 0] = 0x0C000003
    pairs = pairs[rng.permutation(n)]
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "tile_kind": kind})
        cube = C.Cube(d)
        cube.update_binned(dev_pairs(pairs), C.UpdateWorkspace(d, n))
        assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, pairs))
    finally:
        C.set_tuning(**before)


@pytest.mark.parametrize("geo,routers", [("L2", 1), ("L2", 3), ("PAPER", 1)])
def test_sampled_capacities_overflow(C, oracle, geo, routers):
    """tile_kind 3 sizes each tile's run from every 16th tile of 1024 packets.  Here one source
    sends half of the packets, but only in the tiles the sample skips, so its tiles get runs sized
    for background traffic and tens of thousands of records overflow: the overflow path must
    still give the oracle's cubes."""
    d = GEO.ALL[geo]
    rng = np.random.default_rng(21)
    n = 1 << 21
    pairs = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    hot = ((np.arange(n) // 1024) % 16 != 0) & (rng.random(n) < 0.5)
    pairs[hot, 0] = 0x0D0E0A0F
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "tile_kind": 3})
        if routers == 1:
            cube = C.Cube(d)
            cube.update_binned(dev_pairs(pairs), C.UpdateWorkspace(d, n))
            assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, pairs))
        else:
            cut = np.linspace(0, n, routers + 1).astype(int)
            cubes = [C.Cube(d) for _ in range(routers)]
            C.update_multi(cubes, [dev_pairs(pairs[cut[j]:cut[j + 1]]) for j in range(routers)],
                           C.UpdateWorkspace(d, n, n_cubes=routers))
            for j in range(routers):
                assert np.array_equal(cubes[j].to_numpy(), oracle.build_cube(d, pairs[cut[j]:cut[j + 1]])), j
    finally:
        C.set_tuning(**before)


def test_update_ragged_and_unaligned(C, oracle):
    """Odd counts, a start that is only 8-byte aligned, empty and one-pair calls, uneven batches."""
    import torch
    d = GEO.TINY2
    w = window("tiny")
    p = dev_pairs(w.pairs)
    cube = C.Cube(d)
    cube.update(p, n=0)
    assert not cube.to_numpy().any()
    bounds = [0, 1, 2, 5, 1000, 1001, 4097, 70001, w.pairs.shape[0]]
    for a, b in zip(bounds[:-1], bounds[1:]):
        cube.update_ptr(p.data_ptr() + 8 * a, b - a)        # start is 8-byte aligned at odd a
    torch.cuda.synchronize()
    assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, w.pairs))


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("r,cbn", [(8, 12), (7, 13)])
def test_largest_row_tile_geometry(C, oracle, kind, r, cbn):
    """512 MiB cubes, the most the partitioned update takes: r=8, c=2^12 has the most row tiles
    (8192 of 64 KiB), r=7, c=2^13 the largest ones (4096 of 128 KiB).  Cube bit-exact and host
    list equal to the oracle's."""
    d = C.make_params(r, 3, 1, 10, [cbn])
    w = window("4m")
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "tile_kind": kind})
        cube = C.Cube(d)
        cube.update_binned(dev_pairs(w.pairs), C.UpdateWorkspace(d, w.pairs.shape[0]))
        want_cube = oracle.build_cube(d, w.pairs)
        assert np.array_equal(cube.to_numpy(), want_cube)
        assert_hosts_equal(cube.detect(1024), oracle.detect(d, want_cube, 1024)["hosts"])
    finally:
        C.set_tuning(**before)


def test_checkpoint_and_resume(C, oracle):
    """A window checkpointed mid-way (cube words to the host), restored into a fresh cube and
    finished there equals the window run without interruption, and the oracle."""
    d = GEO.L2
    w = window("4m")
    p = dev_pairs(w.pairs)
    half = 1_234_567
    ws = C.UpdateWorkspace(d, w.pairs.shape[0])
    a = C.Cube(d)
    a.update_binned(p[:half], ws)
    snap = a.to_numpy().copy()
    b = C.Cube(d)
    b.load_numpy(snap)
    b.update_binned(p[half:], ws)
    whole = C.Cube(d)
    whole.update_binned(p, ws)
    assert np.array_equal(b.to_numpy(), whole.to_numpy())
    assert np.array_equal(b.to_numpy(), oracle.build_cube(d, w.pairs))
    with pytest.raises(C.CbaaError):
        C.Cube(GEO.TINY).load_numpy(snap)


def test_update_order_and_duplicates(C):
    d = GEO.TINY
    w = window("tiny")
    c1, c2 = C.Cube(d), C.Cube(d)
    c1.update(dev_pairs(w.pairs))
    perm = np.random.default_rng(3).permutation(w.pairs.shape[0])
    c2.update(dev_pairs(np.concatenate([w.pairs[perm], w.pairs[::7]])))
    assert np.array_equal(c1.to_numpy(), c2.to_numpy())


@pytest.mark.parametrize("k", [1, 3, 20])
def test_merge_equals_union(C, oracle, k):
    """Section III.C: OR of per-router cubes equals the cube of all the traffic (k > 16 spans launches)."""
    d = GEO.TINY2
    w = window("tiny")
    rid, _ = T.split_by_router(w.pairs, 77, k)
    routers = []
    for i in range(k):
        c = C.Cube(d)
        c.update(dev_pairs(w.pairs[rid == i]))
        routers.append(c)
    dst = C.Cube(d)
    dst.merge(routers)
    assert np.array_equal(dst.to_numpy(), oracle.build_cube(d, w.pairs))


@pytest.mark.parametrize("k", [0, 1, 3, 20])
def test_merge_assign_replaces_dst(C, oracle, k):
    """cbaa_cube_merge_assign: a global cube full of an earlier window's bits becomes exactly the
    OR of the router cubes, i.e. the cube of all their traffic (k = 0: an empty cube)."""
    import torch
    d = GEO.TINY2
    w = window("tiny")
    rid, _ = T.split_by_router(w.pairs, 78, max(k, 1))
    routers = []
    for i in range(k):
        c = C.Cube(d)
        c.update(dev_pairs(w.pairs[rid == i]))
        routers.append(c)
    dst = C.Cube(d)
    dst.memory.copy_(torch.randint(-2**31, 2**31 - 1, dst.memory.shape, device="cuda", dtype=torch.int32))
    dst.merge(routers, assign=True)
    want = oracle.build_cube(d, w.pairs) if k else np.zeros_like(dst.to_numpy())
    assert np.array_equal(dst.to_numpy(), want)
    if k:
        bad = C.Cube(GEO.TINY)
        with pytest.raises(C.CbaaError):
            dst.merge(routers + [bad], assign=True)      # checked before anything is enqueued
        assert np.array_equal(dst.to_numpy(), want)


def test_merge_geometry_mismatch(C):
    a, b = C.Cube(GEO.TINY), C.Cube(GEO.with_form(GEO.TINY, 1))
    with pytest.raises(C.CbaaError) as e:
        a.merge([b])
    assert e.value.status == C.ERR_GEOMETRY
    with pytest.raises(C.CbaaError):
        a.merge([a])


@pytest.mark.parametrize("geo,win,theta,form", [("TINY", "tiny", 128, 0), ("TINY2", "tiny", 128, 1),
                                                ("PAPER", "1m", 1024, 0), ("L2", "4m", 1024, 0),
                                                ("L2", "4m", 1024, 1), ("UNDERSIZED", "4m", 1024, 0),
                                                ("QUAD", "tiny", 128, 0), ("DUO", "tiny", 128, 1)])
def test_column_stats_bit_exact(C, oracle, geo, win, theta, form):
    d = GEO.with_form(GEO.ALL[geo], form)
    w = window(win)
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    st = cube.column_stats(theta)
    host = oracle.build_cube(d, w.pairs)
    zc, za = oracle.zero_counts(d, host)
    A = d["n_ra"] + d["n_va"]
    for a in range(A):
        c = 1 << d["cbn"][a]
        assert np.array_equal(st["zc"][:, a, :c].astype(np.uint32), zc[:, a, :c])
    assert np.array_equal(st["za"], za)
    E = oracle.exp_factor(theta, d["log2_g"])
    for cs in range(1 << d["r"]):
        e = oracle.eps(d, za, cs)
        assert st["eps"][cs] == e                          # same IEEE double
        assert st["zmax"][cs] == oracle.zmax(d, e, E)


@pytest.mark.parametrize("log2_g,cbn", [(8, [9, 9, 10, 8]), (9, [10, 10, 10, 9]), (11, [9, 9, 9, 9])])
def test_column_stats_every_column_length(C, oracle, log2_g, cbn):
    """Columns of 2, 4 and 16 pieces of 16 bytes (g = 2^8, 2^9, 2^11; the 1- and 8-piece cases and the
    long columns are in the test above), with unequal array widths: zero counts, array totals, eps and
    Zmax against the oracle."""
    d = C.make_params(6, 3, 1, log2_g, cbn)
    w = window("tiny")
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    st = cube.column_stats(128)
    host = oracle.build_cube(d, w.pairs)
    zc, za = oracle.zero_counts(d, host)
    for a in range(4):
        c = 1 << d["cbn"][a]
        assert np.array_equal(st["zc"][:, a, :c].astype(np.uint32), zc[:, a, :c])
    assert np.array_equal(st["za"], za)
    E = oracle.exp_factor(128, log2_g)
    for cs in range(1 << d["r"]):
        e = oracle.eps(d, za, cs)
        assert st["eps"][cs] == e and st["zmax"][cs] == oracle.zmax(d, e, E)


DETECT_CASES = [("TINY", "tiny", 128, 0), ("TINY", "tiny", 96, 1), ("TINY", "tiny_sat", 128, 0),
                ("TINY2", "tiny", 128, 0), ("PAPER", "1m", 1024, 0), ("PAPER", "1m", 1024, 1),
                ("L2", "4m", 1024, 0), ("L2", "4m", 700, 1), ("UNDERSIZED", "4m", 1024, 0),
                ("SERVE", "4m", 1024, 0), ("QUAD", "tiny", 128, 0),
                ("DUO", "tiny", 128, 1),
                # theta beyond any estimate: form 0 keeps Zmax = 0 (only saturated columns are hot,
                # every host has Z = 0), form 1 makes it negative (no hot column, no host)
                ("TINY", "tiny_sat", 1 << 20, 0), ("TINY", "tiny_sat", 1 << 20, 1)]


@pytest.mark.parametrize("geo,win,theta,form", DETECT_CASES)
def test_detect_host_list_parity(C, oracle, geo, win, theta, form):
    d = GEO.with_form(GEO.ALL[geo], form)
    w = window(win)
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    got = cube.detect(theta)
    want = oracle.detect(d, oracle.build_cube(d, w.pairs), theta)["hosts"]
    assert_hosts_equal(got, want)
    assert np.all(np.diff(got["ip"].astype(np.int64)) > 0)       # sorted, no duplicates
    if win == "tiny_sat" and theta < (1 << 20):
        assert (got["flags"] & C.FLAG_SATURATED).any()
    if theta >= (1 << 20):
        assert np.all(got["z"] == 0) and np.all(got["flags"] & C.FLAG_SATURATED)
        assert (got.size > 0) == (form == 0), got.size


def test_detect_empty_cube_and_repeat(C):
    d = GEO.PAPER
    cube = C.Cube(d)
    assert cube.detect(1024).size == 0
    w = window("1m")
    cube.update(dev_pairs(w.pairs))
    a = cube.detect(1024)
    b = cube.detect(1024)
    assert a.size >= 20 and np.array_equal(a, b)


def test_detect_capacity_returns_smallest_ips(C):
    d = GEO.PAPER
    w = window("1m")
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    full = cube.detect(1024)
    ws = C.Workspace(d)
    out = (C.Host * 5)()
    n = ctypes.c_size_t(0)
    st = C.lib().cbaa_detect(cube.handle, 1024, ws.ptr, ws.nbytes, out, 5, ctypes.byref(n), None)
    assert st == C.ERR_CAPACITY and n.value == full.size
    got = np.frombuffer(out, dtype=C.HOST_DTYPE, count=5)
    assert np.array_equal(got, full[:5])


def test_detect_saturated_cube_reports_workspace(C):
    """Every column hot: the tuple space explodes and detect says how much it needed, without faulting."""
    import torch
    d = GEO.TINY
    cube = C.Cube(d)
    cube.memory.fill_(-1)
    ws = C.Workspace(d, max_candidates=1 << 12)
    out = (C.Host * 16)()
    n = ctypes.c_size_t(0)
    st = C.lib().cbaa_detect(cube.handle, 128, ws.ptr, ws.nbytes, out, 16, ctypes.byref(n), None)
    torch.cuda.synchronize()
    assert st == C.ERR_WORKSPACE and n.value > (1 << 12)


def test_detect_async_matches_sync(C):
    import torch
    d = GEO.L2
    w = window("4m")
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    sync = cube.detect(1024)
    ws = C.Workspace(d)
    out = torch.zeros(4 * 4096, dtype=torch.int32, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    cube.detect_async(1024, ws, out, info)
    hosts, inf = C.hosts_from_device(out, info)
    assert inf["status"] == C.OK and inf["n_hosts"] == sync.size
    assert np.array_equal(hosts, sync)


def test_full_size_64m_window(C, oracle):
    """The benchmark's workload: 64M packets into the 64 MiB L2-resident cube, launched as the bench does."""
    d = GEO.L2
    w = T.make_window(T.spec_window_64m())
    cube = C.Cube(d)
    cube.update(dev_pairs(w.pairs))
    got_cube = cube.to_numpy()
    want_cube = oracle.build_cube(d, w.pairs)
    assert np.array_equal(got_cube, want_cube)
    got = cube.detect(1024)
    want = oracle.detect(d, want_cube, 1024)["hosts"]
    assert_hosts_equal(got, want)
    assert set(w.planted_ips.tolist()) <= set(got["ip"].tolist())
    # the benchmark's own launch configuration: the autotuner's pick over every path and shape
    from paper_1901_06207_b300 import autotune
    base = C.get_tuning()
    try:
        pairs = dev_pairs(w.pairs)
        tuned = autotune.tune_update(d, pairs, use_cache=False)
        cube.reset()
        if tuned["path"] == "binned":
            cube.update_binned(pairs, C.UpdateWorkspace(d, pairs.shape[0]))
        else:
            cube.update(pairs)
        assert np.array_equal(cube.to_numpy(), want_cube), tuned["tuning"]
        assert_hosts_equal(cube.detect(1024), want)
    finally:
        C.set_tuning(**base)
