"""The inner/outer model of Section III on the GPU: with NI attached to a cube, updates read raw
{src, dst} packets, keep those between NI and NO with the inner address first, and skip the rest.
Every update path must give the oracle's cube of the oriented pairs, and detect its host list."""
import numpy as np
import pytest

import geometries as GEO
from paper_1901_06207_b300 import traffic as T

pytestmark = pytest.mark.gpu

NI = [(0x0A000000, 8), (0xAC100000, 12)]          # 10.0.0.0/8, 172.16.0.0/12


@pytest.fixture(scope="module")
def C():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1901_06207_b300 import build
    build.build()
    from paper_1901_06207_b300 import cbaa
    return cbaa


@pytest.fixture(scope="module")
def raw():
    w = T.make_window(T.spec_window_64m(scale_shift=4))          # 4M packets
    return T.bidirectional_pairs(w.pairs, 0xD1, 0x0A000000, 8)


def _dev(pairs):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("geo", ["L2", "PAPER", "DUO"])
@pytest.mark.parametrize("path", ["direct", "kind1", "kind2", "kind3"])
def test_oriented_cube_equals_oracle(C, oracle, raw, geo, path):
    d = GEO.ALL[geo]
    before = C.get_tuning()
    try:
        cube = C.Cube(d)
        cube.set_inner_net(NI)
        if path == "direct":
            cube.update(_dev(raw))
        else:
            C.set_tuning(**{**before, "tile_kind": int(path[-1])})     # kind3: sampled run capacities
            cube.update_binned(_dev(raw), C.UpdateWorkspace(d, raw.shape[0]))
        assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, oracle.orient(raw, NI)))
    finally:
        C.set_tuning(**before)


def test_oriented_detect_equals_oracle(C, oracle, raw):
    d, theta = GEO.L2, 1024
    cube = C.Cube(d)
    cube.set_inner_net(NI)
    cube.update_binned(_dev(raw), C.UpdateWorkspace(d, raw.shape[0]))
    got = cube.detect(theta)
    want = oracle.detect(d, oracle.build_cube(d, oracle.orient(raw, NI)), theta)["hosts"]
    assert got.size == want.size and got.size > 0
    assert np.array_equal(got["ip"], want["ip"]) and np.array_equal(got["z"], want["z"])


def test_inner_net_reset_and_multi_cube(C, oracle, raw):
    d = GEO.L2
    oriented = oracle.orient(raw, NI)
    cube = C.Cube(d)
    cube.set_inner_net(NI)
    cube.set_inner_net(None)                                      # back to {iip, oip} input
    cube.update(_dev(oriented))
    assert np.array_equal(cube.to_numpy(), oracle.build_cube(d, oriented))
    half = raw.shape[0] // 2
    cubes = [C.Cube(d), C.Cube(d)]
    for c in cubes:
        c.set_inner_net(NI)
    ws = C.UpdateWorkspace(d, raw.shape[0], n_cubes=2)
    C.update_multi(cubes, [_dev(raw[:half]), _dev(raw[half:])], ws)
    assert np.array_equal(cubes[0].to_numpy(), oracle.build_cube(d, oracle.orient(raw[:half], NI)))
    assert np.array_equal(cubes[1].to_numpy(), oracle.build_cube(d, oracle.orient(raw[half:], NI)))
    cubes[1].set_inner_net(NI[:1])
    with pytest.raises(C.CbaaError):
        C.update_multi(cubes, [_dev(raw[:half]), _dev(raw[half:])], ws)
    with pytest.raises(C.CbaaError):
        cube.set_inner_net([(0x0A000000, 33)])
    with pytest.raises(C.CbaaError):
        cube.set_inner_net([(0x0A000000, 8)] * 17)
