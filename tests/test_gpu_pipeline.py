"""Double-buffered windows on two streams (the bench's timed loop and the serving pattern):
window k+1's reset and update overlap window k's detect.  Every window's host list must equal
the one from running the windows one at a time, and the oracle's."""
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


def _windows(k, n):
    out = []
    for w in range(k):
        spec = T.TrafficSpec(n_packets=n, n_hosts=20000, n_planted=60, planted_lo=1100, planted_hi=4000,
                             planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=200, seed=0x91E0 + w)
        out.append(T.make_window(spec).pairs)
    return out


def test_double_buffered_windows_match_serial_and_oracle(C, oracle):
    import torch
    d, theta = GEO.L2, 1024
    wins = _windows(5, 1 << 21)
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in wins]
    uws = C.UpdateWorkspace(d, max(p.shape[0] for p in wins))

    serial = []
    cube, ws = C.Cube(d), C.Workspace(d)
    for p in dev:
        cube.reset()
        cube.update_binned(p, uws)
        serial.append(cube.detect(theta, ws=ws))

    cap = 1 << 14
    cubes = [C.Cube(d), C.Cube(d)]
    wss = [C.Workspace(d), C.Workspace(d)]
    outs = torch.zeros((len(wins), 4 * cap), dtype=torch.int32, device="cuda")
    infos = torch.zeros((len(wins), 8), dtype=torch.int32, device="cuda")
    s_up, s_det = torch.cuda.Stream(), torch.cuda.Stream()
    done = [None, None]
    torch.cuda.synchronize()
    for k, p in enumerate(dev):
        b = k & 1
        with torch.cuda.stream(s_up):
            if done[b] is not None:
                s_up.wait_event(done[b])            # the cube's previous detect has finished
            cubes[b].reset()
            cubes[b].update_binned(p, uws)
            up = torch.cuda.Event()
            up.record(s_up)
        with torch.cuda.stream(s_det):
            s_det.wait_event(up)
            cubes[b].detect_async(theta, wss[b], outs[k], infos[k])
            done[b] = torch.cuda.Event()
            done[b].record(s_det)
    torch.cuda.synchronize()
    for k in range(len(wins)):
        hosts, info = C.hosts_from_device(outs[k], infos[k])
        assert info["status"] == C.OK
        assert np.array_equal(hosts, serial[k]), k
    want = oracle.detect(d, oracle.build_cube(d, wins[-1]), theta)["hosts"]
    assert np.array_equal(serial[-1]["ip"], want["ip"]) and np.array_equal(serial[-1]["z"], want["z"])
