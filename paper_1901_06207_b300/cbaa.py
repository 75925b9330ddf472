"""ctypes binding of libcbaa.so (argument marshalling only).

Every step of the detector runs in the CUDA library; this module turns
torch tensors (device memory, streams) into the pointers and sizes of the
C ABI declared in include/cbaa.h and raises on error statuses.  There is no
CPU fallback: if the library cannot be loaded, using this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcbaa.so")

MAX_ARRAYS = 8
MAX_RA = 6
FLAG_SATURATED = 1

OK, ERR_INVALID_ARG, ERR_GEOMETRY, ERR_CAPACITY, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_NO_DEVICE = \
    0, -1, -2, -3, -4, -5, -6, -7


class Params(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_uint32), ("n_ra", ctypes.c_uint32), ("n_va", ctypes.c_uint32), ("log2_g", ctypes.c_uint32),
        ("cbn", ctypes.c_uint32 * MAX_ARRAYS), ("ring_off", ctypes.c_uint32 * MAX_ARRAYS),
        ("seed_mangle", ctypes.c_uint32), ("seed_bv", ctypes.c_uint32),
        ("seed_va", ctypes.c_uint32 * MAX_ARRAYS), ("threshold_form", ctypes.c_uint32),
    ]


class Host(ctypes.Structure):
    _fields_ = [("ip", ctypes.c_uint32), ("z_union", ctypes.c_uint32), ("est", ctypes.c_float),
                ("flags", ctypes.c_uint32)]


class DetectInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_hosts", ctypes.c_uint32), ("n_hot", ctypes.c_uint32),
                ("n_tuples", ctypes.c_uint32), ("need_tuples", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 3)]


MAX_INNER = 16


class InnerNet(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("addr", ctypes.c_uint32 * MAX_INNER), ("len", ctypes.c_uint32 * MAX_INNER)]


class Tuning(ctypes.Structure):
    _fields_ = [("scatter_shape", ctypes.c_uint32), ("count_blocks_per_sm", ctypes.c_uint32),
                ("apply_items_per_sm", ctypes.c_uint32), ("direct_blocks_per_sm", ctypes.c_uint32),
                ("tile_kind", ctypes.c_uint32), ("heavy", ctypes.c_uint32), ("split_blocks", ctypes.c_uint32)]


HOST_DTYPE = np.dtype([("ip", "<u4"), ("z", "<u4"), ("est", "<f4"), ("flags", "<u4")])
assert HOST_DTYPE.itemsize == ctypes.sizeof(Host) == 16
INFO_BYTES = ctypes.sizeof(DetectInfo)


class CbaaError(RuntimeError):
    def __init__(self, status: int, what: str):
        extra = f" [{lib().cbaa_last_cuda_error().decode()}]" if status == ERR_CUDA else ""
        super().__init__(f"{what}: {status_str(status)} ({status}){extra}")
        self.status = status


_lib = None


def _signatures():
    P, vp, sz = ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_size_t
    return {
        "cbaa_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "cbaa_last_cuda_error": (ctypes.c_char_p, []),
        "cbaa_params_validate": (ctypes.c_int, [P]),
        "cbaa_cube_bytes": (sz, [P]),
        "cbaa_detect_workspace_bytes": (sz, [P, sz]),
        "cbaa_cube_init": (ctypes.c_int, [P, vp, sz, ctypes.POINTER(vp), vp]),
        "cbaa_cube_destroy": (ctypes.c_int, [vp]),
        "cbaa_cube_data": (vp, [vp]),
        "cbaa_cube_params": (ctypes.c_int, [vp, P]),
        "cbaa_cube_reset": (ctypes.c_int, [vp, vp]),
        "cbaa_cube_set_inner_net": (ctypes.c_int, [vp, ctypes.POINTER(InnerNet)]),
        "cbaa_cube_update": (ctypes.c_int, [vp, vp, sz, vp]),
        "cbaa_cube_merge": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.c_int, vp]),
        "cbaa_cube_merge_assign": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.c_int, vp]),
        "cbaa_column_stats": (ctypes.c_int, [vp, ctypes.c_uint32, vp, vp, vp, vp, vp]),
        "cbaa_detect_async": (ctypes.c_int, [vp, ctypes.c_uint32, vp, sz, vp, sz, vp, vp]),
        "cbaa_detect_range_async": (ctypes.c_int, [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, vp, sz,
                                                   vp, sz, vp, vp]),
        "cbaa_or_words": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.c_int, sz, vp]),
        "cbaa_detect": (ctypes.c_int, [vp, ctypes.c_uint32, vp, sz, vp, sz, ctypes.POINTER(sz), vp]),
        "cbaa_bench_red_or": (ctypes.c_int, [vp, sz, sz, ctypes.c_uint32, vp]),
        "cbaa_detect_static": (ctypes.c_int, [vp, ctypes.c_uint32, vp, sz, vp, vp]),
        "cbaa_update_workspace_bytes": (sz, [P, sz]),
        "cbaa_cube_update_binned": (ctypes.c_int, [vp, vp, sz, vp, sz, vp]),
        "cbaa_cube_update_binned_assign": (ctypes.c_int, [vp, vp, sz, vp, sz, vp]),
        "cbaa_update_multi_workspace_bytes": (sz, [P, ctypes.c_int, sz]),
        "cbaa_cube_update_multi": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                                  ctypes.POINTER(sz), vp, sz, vp]),
        "cbaa_cube_update_multi_merge": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                                        ctypes.POINTER(sz), vp, vp, sz, vp]),
        "cbaa_set_tuning": (ctypes.c_int, [ctypes.POINTER(Tuning)]),
        "cbaa_host_features": (ctypes.c_int, [vp, vp, vp, vp, sz, vp, vp]),
        "cbaa_mlp_forward": (ctypes.c_int, [vp, vp, sz, vp, vp]),
        "cbaa_mlp_grad": (ctypes.c_int, [vp, vp, vp, sz, ctypes.c_float, vp, vp, vp]),
        "cbaa_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_uint32, vp]),
        "cbaa_mlp_to_bf16": (ctypes.c_int, [vp, vp, vp]),
        "cbaa_learned_decide": (ctypes.c_int, [vp, vp, sz, ctypes.c_uint32, ctypes.c_float, vp, vp, vp]),
        "cbaa_learned_target": (ctypes.c_int, [vp, vp, sz, vp, vp]),
        "cbaa_merge_hosts": (ctypes.c_int, [vp, sz, ctypes.c_int, vp, vp, sz, vp, vp]),
        "cbaa_get_tuning": (ctypes.c_int, [ctypes.POINTER(Tuning)]),
    }


def lib() -> ctypes.CDLL:
    """The loaded library with every entry point's argument types declared."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcbaa.so not built at {LIB_PATH}; run python -m paper_1901_06207_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _signatures().items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def status_str(status: int) -> str:
    return lib().cbaa_status_str(status).decode()


def _check(status: int, what: str) -> int:
    if status != OK:
        raise CbaaError(status, what)
    return status


# --------------------------------------------------------------------------- geometry

def make_params(r: int, n_ra: int, n_va: int, log2_g: int, cbn, *, seed_mangle=0x3C6EF372,
                seed_bv=0xA54FF53A, seed_va=(0x510E527F, 0x9B05688C, 0x1F83D9AB, 0x5BE0CD19),
                threshold_form: int = 0) -> dict:
    """Geometry dict with CL_bs offsets splitting LP as evenly as possible, larger EPs first."""
    L = 32 - r
    base, rem = divmod(L, n_ra)
    ep = [base + 1] * rem + [base] * (n_ra - rem)
    off = [0]
    for e in ep[:-1]:
        off.append(off[-1] + e)
    cbn = list(cbn)
    if len(cbn) == 1:
        cbn = cbn * (n_ra + n_va)
    sv = list(seed_va) + [0] * (MAX_ARRAYS - len(seed_va))
    return dict(r=r, n_ra=n_ra, n_va=n_va, log2_g=log2_g, cbn=cbn + [0] * (MAX_ARRAYS - len(cbn)),
                ring_off=off + [0] * (MAX_ARRAYS - len(off)), seed_mangle=seed_mangle, seed_bv=seed_bv,
                seed_va=sv[:MAX_ARRAYS], threshold_form=threshold_form)


def params(d: dict) -> Params:
    p = Params()
    p.r, p.n_ra, p.n_va, p.log2_g = d["r"], d["n_ra"], d["n_va"], d["log2_g"]
    for k, v in enumerate(d["cbn"][:MAX_ARRAYS]):
        p.cbn[k] = v
    for k, v in enumerate(d["ring_off"][:MAX_ARRAYS]):
        p.ring_off[k] = v
    p.seed_mangle, p.seed_bv = d["seed_mangle"], d["seed_bv"]
    for k, v in enumerate(d["seed_va"][:MAX_ARRAYS]):
        p.seed_va[k] = v
    p.threshold_form = d.get("threshold_form", 0)
    return p


def validate(d: dict) -> int:
    return lib().cbaa_params_validate(ctypes.byref(params(d)))


def cube_bytes(d: dict) -> int:
    return int(lib().cbaa_cube_bytes(ctypes.byref(params(d))))


def workspace_bytes(d: dict, max_candidates: int) -> int:
    return int(lib().cbaa_detect_workspace_bytes(ctypes.byref(params(d)), max_candidates))


# --------------------------------------------------------------------------- device objects

def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Workspace:
    """Detect workspace: device bytes sized for ``max_candidates`` tuples/hosts per stage."""

    def __init__(self, d: dict, max_candidates: int = 1 << 18, device="cuda"):
        torch = _torch()
        self.nbytes = workspace_bytes(d, max_candidates)
        if self.nbytes == 0:
            raise CbaaError(ERR_INVALID_ARG, "workspace size")
        self.max_candidates = max_candidates
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()


def update_workspace_bytes(d: dict, max_pairs: int) -> int:
    return int(lib().cbaa_update_workspace_bytes(ctypes.byref(params(d)), max_pairs))


def update_multi_workspace_bytes(d: dict, n_cubes: int, max_pairs: int) -> int:
    return int(lib().cbaa_update_multi_workspace_bytes(ctypes.byref(params(d)), n_cubes, max_pairs))


def set_tuning(scatter_shape=0, count_blocks_per_sm=0, apply_items_per_sm=0, direct_blocks_per_sm=0, tile_kind=0,
               heavy=0, split_blocks=0):
    t = Tuning(scatter_shape, count_blocks_per_sm, apply_items_per_sm, direct_blocks_per_sm, tile_kind, heavy,
               split_blocks)
    _check(lib().cbaa_set_tuning(ctypes.byref(t)), "set_tuning")


def get_tuning() -> dict:
    t = Tuning()
    _check(lib().cbaa_get_tuning(ctypes.byref(t)), "get_tuning")
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def update_multi(cubes, pairs_list, ws: "UpdateWorkspace", counts=None, stream=None, merge_into=None):
    """Alg. 1 for several router cubes in one partitioned pass: pairs_list[j] feeds cubes[j].  With
    ``merge_into`` (a Cube), every bit the pass sets is ORed into it as well (the global merge)."""
    k = len(cubes)
    hs = (ctypes.c_void_p * k)(*[c.handle.value for c in cubes])
    ps = (ctypes.c_void_p * k)(*[p.data_ptr() if p is not None and p.numel() else None for p in pairs_list])
    if counts is None:
        counts = [0 if p is None else (p.shape[0] if p.dim() == 2 else p.numel() // 2) for p in pairs_list]
    ns = (ctypes.c_size_t * k)(*counts)
    if merge_into is not None:
        _check(lib().cbaa_cube_update_multi_merge(hs, k, ps, ns, merge_into.handle, ws.ptr, ws.nbytes,
                                                  _stream_ptr(stream)), "cube_update_multi_merge")
        return
    _check(lib().cbaa_cube_update_multi(hs, k, ps, ns, ws.ptr, ws.nbytes, _stream_ptr(stream)), "cube_update_multi")


class UpdateWorkspace:
    """Workspace of the partitioned update, sized for ``max_pairs`` packets per pass over ``n_cubes`` cubes."""

    def __init__(self, d: dict, max_pairs: int, device="cuda", n_cubes: int = 1):
        torch = _torch()
        self.nbytes = update_multi_workspace_bytes(d, n_cubes, max_pairs)
        if self.nbytes == 0:
            raise CbaaError(ERR_INVALID_ARG, "update workspace size")
        self.max_pairs = max_pairs
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()


class Cube:
    """A cube of bit arrays in caller (torch) device memory."""

    def __init__(self, d: dict, device="cuda", memory=None, stream=None):
        torch = _torch()
        self.geometry = dict(d)
        self._p = params(d)
        _check(lib().cbaa_params_validate(ctypes.byref(self._p)), "params")
        self.nbytes = cube_bytes(d)
        if memory is None:
            memory = torch.empty(self.nbytes // 4, dtype=torch.int32, device=device)
        self.memory = memory
        h = ctypes.c_void_p()
        _check(lib().cbaa_cube_init(ctypes.byref(self._p), memory.data_ptr(), memory.numel() * memory.element_size(),
                                    ctypes.byref(h), _stream_ptr(stream)), "cube_init")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.cbaa_cube_destroy(h)
            self.handle = None

    def to_numpy(self) -> np.ndarray:
        """The cube words as a uint32 numpy array (synchronises, copies to host)."""
        torch = _torch()
        torch.cuda.synchronize()
        return self.memory.view(torch.int32).cpu().numpy().view(np.uint32)

    def load_numpy(self, words: np.ndarray):
        """Restore cube words taken by to_numpy() (a checkpoint of a window in progress) into this
        cube, which must have the snapshot's geometry; later updates OR into the restored bits."""
        torch = _torch()
        w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1)
        if w.size * 4 != self.nbytes:
            raise CbaaError(ERR_INVALID_ARG, f"snapshot of {w.size * 4} bytes for a {self.nbytes}-byte cube")
        self.memory.view(torch.int32)[: w.size].copy_(torch.from_numpy(w.view(np.int32)))

    def reset(self, stream=None):
        _check(lib().cbaa_cube_reset(self.handle, _stream_ptr(stream)), "cube_reset")

    def set_inner_net(self, prefixes=None):
        """The monitored network NI as [(address, prefix length)] (addresses as ints, host order).
        Afterwards updates read raw {src, dst} pairs and orient them; None or [] restores {iip, oip}."""
        net = InnerNet()
        prefixes = list(prefixes or [])
        net.n = len(prefixes)
        for k, (a, ln) in enumerate(prefixes[:MAX_INNER]):
            net.addr[k], net.len[k] = int(a) & 0xFFFFFFFF, int(ln)
        _check(lib().cbaa_cube_set_inner_net(self.handle, ctypes.byref(net)), "cube_set_inner_net")

    def update(self, pairs, n: int | None = None, stream=None):
        """pairs: device uint32/int32 tensor of shape [n, 2] (iip, oip), contiguous."""
        if n is None:
            n = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
        _check(lib().cbaa_cube_update(self.handle, pairs.data_ptr(), n, _stream_ptr(stream)), "cube_update")

    def update_ptr(self, ptr: int, n: int, stream=None):
        _check(lib().cbaa_cube_update(self.handle, ptr, n, _stream_ptr(stream)), "cube_update")

    def update_binned(self, pairs, ws: "UpdateWorkspace", n: int | None = None, stream=None, assign: bool = False):
        """Partitioned Alg. 1 (same bits as update) using an UpdateWorkspace; assign=True: the cube
        becomes these packets' bits alone (no reset needed first)."""
        if n is None:
            n = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
        self.update_binned_ptr(pairs.data_ptr(), n, ws, stream, assign)

    def update_binned_ptr(self, ptr: int, n: int, ws: "UpdateWorkspace", stream=None, assign: bool = False):
        fn = lib().cbaa_cube_update_binned_assign if assign else lib().cbaa_cube_update_binned
        _check(fn(self.handle, ptr, n, ws.ptr, ws.nbytes, _stream_ptr(stream)),
               "cube_update_binned_assign" if assign else "cube_update_binned")

    def merge(self, others, stream=None, assign: bool = False):
        """self |= OR(others); assign=True: self = OR(others) without reading self (no reset needed)."""
        arr = (ctypes.c_void_p * max(1, len(others)))(*[o.handle.value for o in others])
        fn = lib().cbaa_cube_merge_assign if assign else lib().cbaa_cube_merge
        _check(fn(self.handle, arr, len(others), _stream_ptr(stream)), "cube_merge_assign" if assign else "cube_merge")

    def column_stats(self, theta: int, stream=None) -> dict:
        torch = _torch()
        g = self.geometry
        S, A = 1 << g["r"], g["n_ra"] + g["n_va"]
        cmax = max(1 << c for c in g["cbn"][:A])
        dev = self.memory.device
        zc = torch.zeros(S * A * cmax, dtype=torch.int16, device=dev)
        za = torch.zeros(S * A, dtype=torch.int64, device=dev)
        eps = torch.zeros(S, dtype=torch.float64, device=dev)
        zmax = torch.zeros(S, dtype=torch.int64, device=dev)
        _check(lib().cbaa_column_stats(self.handle, theta, zc.data_ptr(), za.data_ptr(), eps.data_ptr(),
                                       zmax.data_ptr(), _stream_ptr(stream)), "column_stats")
        torch.cuda.synchronize()
        return {"zc": zc.cpu().numpy().view(np.uint16).reshape(S, A, cmax),
                "za": za.cpu().numpy().view(np.uint64).reshape(S, A),
                "eps": eps.cpu().numpy(), "zmax": zmax.cpu().numpy()}

    def detect(self, theta: int, ws: Workspace | None = None, cap: int = 1 << 16, stream=None,
               max_retries: int = 6) -> np.ndarray:
        """Sync detect; grows the workspace and the output on WORKSPACE / CAPACITY."""
        for _ in range(max_retries):
            if ws is None:
                ws = Workspace(self.geometry, device=self.memory.device)
            out = (Host * max(1, cap))()
            n = ctypes.c_size_t(0)
            st = lib().cbaa_detect(self.handle, theta, ws.ptr, ws.nbytes, out, cap, ctypes.byref(n),
                                   _stream_ptr(stream))
            if st == ERR_WORKSPACE:
                ws = Workspace(self.geometry, max_candidates=max(2 * ws.max_candidates, 2 * int(n.value)),
                               device=self.memory.device)
                continue
            if st == ERR_CAPACITY:
                cap = int(n.value)
                continue
            _check(st, "detect")
            self.last_workspace = ws
            return np.frombuffer(out, dtype=HOST_DTYPE, count=int(n.value)).copy()
        raise CbaaError(ERR_WORKSPACE, "detect retries exhausted")

    def detect_async(self, theta: int, ws: Workspace, out, info, stream=None):
        """Enqueue a detect writing sorted hosts to device tensor ``out`` (int32 [cap*4]) and ``info``."""
        cap = out.numel() * out.element_size() // 16
        _check(lib().cbaa_detect_async(self.handle, theta, ws.ptr, ws.nbytes, out.data_ptr(), cap,
                                       info.data_ptr(), _stream_ptr(stream)), "detect_async")


    def detect_range_async(self, cs_lo: int, cs_hi: int, theta: int, ws: Workspace, out, info, stream=None):
        """detect_async restricted to the sketches cs_lo <= cs < cs_hi."""
        cap = out.numel() * out.element_size() // 16
        _check(lib().cbaa_detect_range_async(self.handle, cs_lo, cs_hi, theta, ws.ptr, ws.nbytes, out.data_ptr(), cap,
                                             info.data_ptr(), _stream_ptr(stream)), "detect_range_async")


def or_words(dst, srcs, stream=None):
    """dst |= OR of srcs, word by word (device int32/uint32 tensors of equal length, 16-byte aligned)."""
    words = dst.numel() * dst.element_size() // 4
    for t in srcs:
        if t.numel() * t.element_size() // 4 != words:
            raise ValueError("or_words: every source must have dst's length")
    arr = (ctypes.c_void_p * max(1, len(srcs)))(*[t.data_ptr() for t in srcs])
    _check(lib().cbaa_or_words(dst.data_ptr(), arr, len(srcs), words, _stream_ptr(stream)), "or_words")


def merge_hosts(blocks, infos, out, info_out, stream=None):
    """Merge k owners' sorted host lists: ``blocks`` int32 [k, 4 * cap] (cbaa_host records), ``infos``
    int32 [k, 8] (cbaa_detect_info), into ``out`` int32 [4 * out_cap] and ``info_out`` int32 [8]."""
    k = int(blocks.shape[0])
    cap = blocks.shape[1] * blocks.element_size() // 16
    out_cap = out.numel() * out.element_size() // 16
    _check(lib().cbaa_merge_hosts(blocks.data_ptr(), cap, k, infos.data_ptr(), out.data_ptr(), out_cap,
                                  info_out.data_ptr(), _stream_ptr(stream)), "merge_hosts")


def hosts_from_device(out, info) -> tuple[np.ndarray, dict]:
    """Decode a detect_async result (device tensors) into a host array and the info dict."""
    raw = info.cpu().numpy().view(np.uint8).tobytes()[:INFO_BYTES]
    inf = DetectInfo.from_buffer_copy(raw)
    d = {"status": inf.status, "n_hosts": inf.n_hosts, "n_hot": inf.n_hot, "n_tuples": inf.n_tuples,
         "need_tuples": inf.need_tuples}
    cap = out.numel() * out.element_size() // 16
    n = min(inf.n_hosts, cap)
    hosts = out.cpu().numpy().view(np.uint8).view(HOST_DTYPE)[:n].copy()
    return hosts, d
