"""Windows that overlap on the device.  Double-buffered windows on two streams (the serving
pattern): window k+1's reset and update overlap window k's detect.  Windows in flight on lanes (the
benchmark's timed loop): each lane runs its windows' update, detect and reset on its own stream with
its own cube and workspaces.  Every window's host list must equal the one from running the windows
one at a time, and the oracle's."""
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


def test_lanes_match_serial(C):
    """Windows in flight on three lanes (the bench's timed loop): lane j owns a stream, a cube, an
    update workspace and a detect workspace, and runs its windows' update, detect and reset in
    order, so one window's heavy split runs beside another's residual kernels and a third's detect.
    Every window's cube and host list must equal the serial ones."""
    import torch
    d, theta = GEO.L2, 1024
    wins = _windows(7, 1 << 22)
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in wins]
    saved = C.get_tuning()
    try:
        C.set_tuning(**{**saved, "tile_kind": 3, "heavy": 3})        # the heavy split on every pass
        n, L = max(p.shape[0] for p in wins), 3
        uws = [C.UpdateWorkspace(d, n) for _ in range(L)]
        serial_cubes, serial = [], []
        cube, ws = C.Cube(d), C.Workspace(d)
        for p in dev:
            cube.reset()
            cube.update_binned(p, uws[0])
            serial_cubes.append(cube.to_numpy())
            serial.append(cube.detect(theta, ws=ws))

        cap = 1 << 14
        cubes = [C.Cube(d) for _ in range(L)]
        wss = [C.Workspace(d) for _ in range(L)]
        streams = [torch.cuda.Stream() for _ in range(L)]
        outs = torch.zeros((len(wins), 4 * cap), dtype=torch.int32, device="cuda")
        infos = torch.zeros((len(wins), 8), dtype=torch.int32, device="cuda")
        got = []
        torch.cuda.synchronize()
        for b in range(L):
            with torch.cuda.stream(streams[b]):
                cubes[b].reset()
        for k, p in enumerate(dev):
            b = k % L
            with torch.cuda.stream(streams[b]):
                cubes[b].update_binned(p, uws[b])
                got.append(cubes[b].memory.clone())   # in the lane's order, before its reset
                cubes[b].detect_async(theta, wss[b], outs[k], infos[k])
                cubes[b].reset()
        torch.cuda.synchronize()
        for k in range(len(wins)):
            hosts, info = C.hosts_from_device(outs[k], infos[k])
            assert info["status"] == C.OK
            assert np.array_equal(hosts, serial[k]), k
            assert np.array_equal(got[k].view(torch.int32).cpu().numpy().view(np.uint32), serial_cubes[k]), k
    finally:
        C.set_tuning(**saved)
