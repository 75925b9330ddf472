"""GPU parity of the heavy-source split in front of the row-tile update.

The split only decides which path sets a packet's bits -- a heavy source's
row bitmap ORed into its columns, or a routed row-tile record -- so every
setting, geometry and traffic shape must give the oracle's cube bit for bit.
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


def dev_pairs(pairs: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).cuda()


def _window(seed, n, planted, lo, hi, hosts, bg_max=64):
    spec = T.TrafficSpec(n_packets=n, n_hosts=hosts, n_planted=planted, planted_lo=lo, planted_hi=hi,
                         planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=bg_max, seed=seed)
    return T.make_window(spec).pairs


_cache = {}


def pairs_of(name):
    if name not in _cache:
        if name == "tiny":
            _cache[name] = _window(71, 1 << 18, 300, 150, 700, 3000)
        elif name == "4m":
            _cache[name] = T.make_window(T.spec_window_64m(scale_shift=4)).pairs
        elif name == "many_heavy":
            # 3000 sources of 400-900 peers each: more heavy candidates than the split holds
            _cache[name] = _window(72, 1 << 22, 3000, 400, 900, 3500, bg_max=8)
        elif name == "uniform":
            rng = np.random.default_rng(73)
            _cache[name] = rng.integers(0, 2**32, size=((1 << 20) + 333, 2), dtype=np.uint64).astype(np.uint32)
    return _cache[name]


def _run(C, d, pairs, tuning, ws_pairs=None, offset=0):
    """Update a fresh cube through cbaa_cube_update_binned with the given tuning; returns its words."""
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, **tuning})
        cube = C.Cube(d)
        p = dev_pairs(pairs)
        ws = C.UpdateWorkspace(d, ws_pairs or max(1, pairs.shape[0] - offset))
        if offset:
            cube.update_binned_ptr(p.data_ptr() + 8 * offset, pairs.shape[0] - offset, ws)
        else:
            cube.update_binned(p, ws)
        return cube.to_numpy()
    finally:
        C.set_tuning(**before)


@pytest.mark.parametrize("heavy", [1, 2, 3])
@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("geo,win", [("L2", "4m"), ("PAPER", "tiny"), ("TINY2", "tiny"), ("QUAD", "tiny"),
                                     ("DUO", "tiny"), ("SERVE", "4m"), ("UNDERSIZED", "tiny")])
def test_heavy_split_cube_bit_exact(C, oracle, geo, win, kind, heavy):
    d = GEO.ALL[geo]
    pairs = pairs_of(win)
    got = _run(C, d, pairs, dict(tile_kind=kind, heavy=heavy))
    assert np.array_equal(got, oracle.build_cube(d, pairs))


@pytest.mark.parametrize("heavy", [2, 3])
@pytest.mark.parametrize("win", ["many_heavy", "uniform"])
def test_heavy_split_more_candidates_than_room_and_none(C, oracle, win, heavy):
    """Thousands of heavy candidates (the threshold and the lower octave decide who fits), and
    uniform traffic (no slot reaches the minimum count: everything takes the row tiles)."""
    d = GEO.L2
    pairs = pairs_of(win)
    got = _run(C, d, pairs, dict(heavy=heavy, tile_kind=3))
    assert np.array_equal(got, oracle.build_cube(d, pairs))


@pytest.mark.parametrize("heavy", [2, 3])
def test_heavy_split_passes_and_unaligned_start(C, oracle, heavy):
    """A workspace for a fifth of the packets (several split passes, each with its own heavy set)
    and a start 8 bytes past a 16-byte boundary (the split's per-packet loads)."""
    d = GEO.L2
    pairs = pairs_of("4m")
    got = _run(C, d, pairs, dict(heavy=heavy, tile_kind=0), ws_pairs=pairs.shape[0] // 5, offset=1)
    assert np.array_equal(got, oracle.build_cube(d, pairs[1:]))


@pytest.mark.parametrize("split_blocks", [1, 37, 74, 4096])
@pytest.mark.parametrize("win", ["4m", "tiny"])
def test_heavy_split_fewer_blocks(C, oracle, win, split_blocks):
    """The split's grid held below one block per SM (SMs left to other streams): larger residual
    regions per block, one block for the whole window; 4096 is capped at one block per SM."""
    d = GEO.L2
    pairs = pairs_of(win)
    got = _run(C, d, pairs, dict(heavy=3, tile_kind=3, split_blocks=split_blocks))
    assert np.array_equal(got, oracle.build_cube(d, pairs))


@pytest.mark.parametrize("tuning,ws_div", [(dict(heavy=3, tile_kind=3), 1),
                                           (dict(heavy=3, tile_kind=3, split_blocks=37), 1),
                                           (dict(heavy=3, tile_kind=0), 5),
                                           (dict(heavy=1, tile_kind=2), 1),
                                           (dict(heavy=1, tile_kind=1), 1)])
@pytest.mark.parametrize("win", ["4m", "tiny"])
def test_assign_update_replaces_a_dirty_cube(C, oracle, win, tuning, ws_div):
    """cbaa_cube_update_binned_assign on a cube full of random words: the cube must become the
    oracle's cube of these packets alone -- zeroed by the split's blocks on the heavy path (one
    block per SM, 37 blocks, several passes), by a memset on the row-tile and column-tile paths."""
    d = GEO.L2
    pairs = pairs_of(win)
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, **tuning})
        cube = C.Cube(d)
        rng = np.random.default_rng(17)
        cube.load_numpy(rng.integers(0, 2**32, size=cube.nbytes // 4, dtype=np.uint64).astype(np.uint32))
        ws = C.UpdateWorkspace(d, max(1, pairs.shape[0] // ws_div))
        cube.update_binned(dev_pairs(pairs), ws, assign=True)
        got = cube.to_numpy()
    finally:
        C.set_tuning(**before)
    assert np.array_equal(got, oracle.build_cube(d, pairs))


def test_assign_update_of_no_packets_zeroes_the_cube(C):
    d = GEO.L2
    cube = C.Cube(d)
    cube.load_numpy(np.full(cube.nbytes // 4, 0xFFFFFFFF, dtype=np.uint32))
    ws = C.UpdateWorkspace(d, 1024)
    cube.update_binned(dev_pairs(np.zeros((0, 2), np.uint32)), ws, n=0, assign=True)
    assert not cube.to_numpy().any()


@pytest.mark.parametrize("heavy", [2, 3])
def test_heavy_split_skewed(C, oracle, heavy):
    """Half the packets one pair and a fifth one source to many peers (one source dominates the
    sample), the rest uniform."""
    d = GEO.L2
    rng = np.random.default_rng(11)
    n = 1_500_003
    pairs = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    pairs[: n // 2] = (0x0A000001, 0x0B000002)
    pairs[n // 2: n // 2 + n // 5, 0] = 0x0C000003
    pairs = pairs[rng.permutation(n)]
    got = _run(C, d, pairs, dict(heavy=heavy, tile_kind=2))
    assert np.array_equal(got, oracle.build_cube(d, pairs))


@pytest.mark.parametrize("heavy", [2, 3])
def test_heavy_split_with_inner_network(C, oracle, heavy):
    """Raw router traffic against an inner network: the split orients packets (and drops internal
    and transit ones) before it picks their path."""
    d = GEO.L2
    prefixes = [(0x0A000000, 8)]
    raw = T.bidirectional_pairs(pairs_of("tiny"), 0xD5, 0x0A000000, 8)
    before = C.get_tuning()
    try:
        C.set_tuning(**{**before, "heavy": heavy, "tile_kind": 3})
        cube = C.Cube(d)
        cube.set_inner_net(prefixes)
        cube.update_binned(dev_pairs(raw), C.UpdateWorkspace(d, raw.shape[0]))
        got = cube.to_numpy()
    finally:
        C.set_tuning(**before)
    assert np.array_equal(got, oracle.build_cube(d, oracle.orient(raw, prefixes)))
