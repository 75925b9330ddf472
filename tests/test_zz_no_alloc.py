"""The allocation-free detect entry point against the ordinary one.

cbaa_detect_static serves callers that cannot allocate device memory while
they run (a host application that owns all GPU memory through its own pool,
or an agent with a fixed memory budget): it keeps its scratch in a static
device array inside the library.  Its results must be those of
cbaa_detect_async with a caller-allocated workspace, call after call, even
though every call reuses the same array.  This file is collected last so a
stop-at-first-failure run has run everything else before it.
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


def _run_static(C, cube, theta, cap):
    import torch
    out = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
    info = torch.full((8,), -1, dtype=torch.int32, device="cuda")
    st = C.lib().cbaa_detect_static(cube.handle, theta, out.data_ptr(), cap, info.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == C.OK, C.status_str(st)
    torch.cuda.synchronize()
    return C.hosts_from_device(out, info)


def _run_async(C, cube, theta, cap):
    import torch
    ws = C.Workspace(cube.geometry)
    out = torch.zeros(4 * cap, dtype=torch.int32, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    cube.detect_async(theta, ws, out, info)
    torch.cuda.synchronize()
    return C.hosts_from_device(out, info)


def _same(a, b):
    assert a.size == b.size
    assert np.array_equal(a["ip"], b["ip"]) and np.array_equal(a["z"], b["z"])
    assert np.array_equal(a["flags"], b["flags"])
    w, g = b["est"].astype(np.float64), a["est"].astype(np.float64)
    assert np.all(np.abs(g - w) <= EST_RTOL * np.maximum(np.abs(w), 1.0))


@pytest.mark.parametrize("geo,spec", [("L2", lambda: T.spec_window_64m(scale_shift=4)),
                                      ("PAPER", T.spec_window_1m)])
def test_static_scratch_detect_matches_workspace_detect(C, geo, spec):
    import torch
    d = GEO.ALL[geo]
    w = T.make_window(spec())
    cube = C.Cube(d)
    cube.update(torch.from_numpy(w.pairs.view(np.int32)).cuda())
    cap = 1 << 14
    want, want_info = _run_async(C, cube, 1024, cap)
    assert want_info["status"] == C.OK and want.size > 0
    for _ in range(2):                      # two calls in a row share the static array
        got, got_info = _run_static(C, cube, 1024, cap)
        assert got_info["status"] == C.OK
        assert got_info["n_hosts"] == want_info["n_hosts"]
        assert got_info["n_hot"] == want_info["n_hot"]
        _same(got, want)


def test_static_scratch_rejects_oversized_geometry(C):
    """A geometry whose detect tables exceed the static array is refused before any work."""
    import torch
    d = C.make_params(8, 3, 1, 7, [14])     # 256 sketches x 2^14 columns: 32 MiB of zero counts alone
    assert C.validate(d) == C.OK
    assert C.workspace_bytes(d, 1) > C.lib().cbaa_detect_workspace_bytes(ctypes.byref(C.params(GEO.L2)), 1)
    cube = C.Cube(d)                        # 256 MiB cube
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    inf = torch.zeros(8, dtype=torch.int32, device="cuda")
    st = C.lib().cbaa_detect_static(cube.handle, 1024, out.data_ptr(), 4, inf.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == C.ERR_WORKSPACE
    assert C.workspace_bytes(d, 1) > 16 << 20
