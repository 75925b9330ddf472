"""Python face of the CBAA CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loads ``liboracle.so`` (built from ``cbaa_oracle.c`` with gcc) through
ctypes.  Only the test suite, the smoke check and the benchmark's CPU
baseline may import this module; the product package never does, and this
module imports nothing from the product package.

Every function states the passage of Xu, Ding and Hu (arXiv 1901.06207) it
follows; the arithmetic itself lives in the C file.  The FNR/FPR measures of
Section V.B (Eq. 2, Eq. 3) are plain set arithmetic and are written here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbaa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_ARRAYS = 8
SATURATED = 1


class OracleGeometry(ctypes.Structure):
    _fields_ = [
        ("r", ctypes.c_uint32), ("n_ra", ctypes.c_uint32), ("n_va", ctypes.c_uint32),
        ("log2_g", ctypes.c_uint32),
        ("cbn", ctypes.c_uint32 * MAX_ARRAYS), ("ring_off", ctypes.c_uint32 * MAX_ARRAYS),
        ("seed_mangle", ctypes.c_uint32), ("seed_bv", ctypes.c_uint32),
        ("seed_va", ctypes.c_uint32 * MAX_ARRAYS), ("threshold_form", ctypes.c_uint32),
    ]


class OracleHost(ctypes.Structure):
    _fields_ = [("ip", ctypes.c_uint32), ("z", ctypes.c_uint32), ("est_bits", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


HOST_DTYPE = np.dtype([("ip", "<u4"), ("z", "<u4"), ("est", "<f4"), ("flags", "<u4")])


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of multiply-adds)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                   "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        G = ctypes.POINTER(OracleGeometry)
        u32p, u64p = ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)
        i64p, f64p = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
        sig = {
            "oracle_mix32": (ctypes.c_uint32, [ctypes.c_uint32]),
            "oracle_unmix32": (ctypes.c_uint32, [ctypes.c_uint32]),
            "oracle_mangle": (ctypes.c_uint32, [G, ctypes.c_uint32]),
            "oracle_unmangle": (ctypes.c_uint32, [G, ctypes.c_uint32]),
            "oracle_row": (ctypes.c_uint32, [G, ctypes.c_uint32]),
            "oracle_va_col": (ctypes.c_uint32, [G, ctypes.c_uint32, ctypes.c_uint32]),
            "oracle_ra_col": (ctypes.c_uint32, [G, ctypes.c_uint32, ctypes.c_uint32]),
            "oracle_ep_len": (ctypes.c_uint32, [G, ctypes.c_uint32]),
            "oracle_cp_len": (ctypes.c_uint32, [G, ctypes.c_uint32]),
            "oracle_cube_words": (ctypes.c_uint64, [G]),
            "oracle_update": (None, [G, u32p, u32p, ctypes.c_uint64]),
            "oracle_merge": (None, [u32p, u32p, ctypes.c_uint64]),
            "oracle_update_threads": (ctypes.c_int, [G, u32p, u32p, ctypes.c_uint64, ctypes.c_int]),
            "oracle_zero_counts": (None, [G, u32p, u32p, u64p]),
            "oracle_eps": (ctypes.c_double, [G, u64p, ctypes.c_uint32]),
            "oracle_exp_factor": (ctypes.c_double, [ctypes.c_uint32, ctypes.c_uint32]),
            "oracle_zmax": (ctypes.c_int64, [G, ctypes.c_double, ctypes.c_double]),
            "oracle_estimate": (ctypes.c_float, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, u32p]),
            "oracle_detect": (ctypes.c_uint64, [G, u32p, ctypes.c_uint32, ctypes.POINTER(OracleHost),
                                                ctypes.c_uint64, f64p, i64p, u64p]),
            "oracle_bruteforce": (ctypes.c_uint64, [G, u32p, i64p, u32p, ctypes.c_uint64, ctypes.c_int]),
            "oracle_exact_counts": (ctypes.c_uint64, [u32p, ctypes.c_uint64, u64p, u32p, u32p]),
            "oracle_union_zeros": (ctypes.c_uint32, [G, u32p, ctypes.c_uint32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    assert a.flags["C_CONTIGUOUS"], "oracle buffers must be contiguous"
    return a.ctypes.data_as(ctypes.POINTER(ct))


def geometry(d: dict) -> OracleGeometry:
    """Oracle geometry from a plain dict of the geometry fields."""
    g = OracleGeometry()
    g.r, g.n_ra, g.n_va, g.log2_g = d["r"], d["n_ra"], d["n_va"], d["log2_g"]
    for k, v in enumerate(d["cbn"]):
        g.cbn[k] = v
    for k, v in enumerate(d["ring_off"]):
        g.ring_off[k] = v
    g.seed_mangle, g.seed_bv = d["seed_mangle"], d["seed_bv"]
    for k, v in enumerate(d["seed_va"]):
        g.seed_va[k] = v
    g.threshold_form = d.get("threshold_form", 0)
    return g


def _G(d):
    return ctypes.byref(geometry(d))


# --- hashing (Section III.A, Alg. 1) -------------------------------------------------------

def mix32(x: int) -> int: return lib().oracle_mix32(x)
def unmix32(y: int) -> int: return lib().oracle_unmix32(y)
def mangle(d, ip: int) -> int: return lib().oracle_mangle(_G(d), ip)
def unmangle(d, m: int) -> int: return lib().oracle_unmangle(_G(d), m)
def row(d, oip: int) -> int: return lib().oracle_row(_G(d), oip)
def va_col(d, j: int, lp: int) -> int: return lib().oracle_va_col(_G(d), j, lp)
def ra_col(d, i: int, lp: int) -> int: return lib().oracle_ra_col(_G(d), i, lp)
def ep_len(d, i: int) -> int: return lib().oracle_ep_len(_G(d), i)
def cp_len(d, i: int) -> int: return lib().oracle_cp_len(_G(d), i)


def cube_words(d) -> int:
    return int(lib().oracle_cube_words(_G(d)))


def new_cube(d) -> np.ndarray:
    return np.zeros(cube_words(d), dtype=np.uint32)


# --- Alg. 1 and the merge of Section III.C --------------------------------------------------

def update(d, cube: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32)
    assert cube.dtype == np.uint32 and cube.size == cube_words(d)
    lib().oracle_update(_G(d), _p(cube, ctypes.c_uint32), _p(pairs, ctypes.c_uint32), pairs.shape[0])
    return cube


def build_cube(d, pairs: np.ndarray) -> np.ndarray:
    return update(d, new_cube(d), pairs)


def update_threads(d, cube: np.ndarray, pairs: np.ndarray, nthreads: int) -> np.ndarray:
    """Alg. 1 on `nthreads` private cubes (one contiguous share of the pairs each), OR-ed into `cube`
    as the global cube of Section III.C is formed from same-structure router cubes."""
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32)
    assert cube.dtype == np.uint32 and cube.size == cube_words(d)
    rc = lib().oracle_update_threads(_G(d), _p(cube, ctypes.c_uint32), _p(pairs, ctypes.c_uint32),
                                     pairs.shape[0], int(nthreads))
    if rc != 0:
        raise MemoryError(f"oracle_update_threads: {nthreads} private cubes did not fit in host memory")
    return cube


def merge(dst: np.ndarray, src: np.ndarray) -> np.ndarray:
    assert dst.shape == src.shape and dst.dtype == src.dtype == np.uint32
    lib().oracle_merge(_p(dst, ctypes.c_uint32), _p(np.ascontiguousarray(src), ctypes.c_uint32), dst.size)
    return dst


# --- zero counts, Thm. 1, theta_bn, Thm. 2 --------------------------------------------------

def zero_counts(d, cube: np.ndarray):
    """(zc [S, A, c_max] uint32, za [S, A] uint64) by bit loops."""
    S, A = 1 << d["r"], d["n_ra"] + d["n_va"]
    cmax = max(1 << c for c in d["cbn"][:A])
    zc = np.zeros((S, A, cmax), dtype=np.uint32)
    za = np.zeros((S, A), dtype=np.uint64)
    lib().oracle_zero_counts(_G(d), _p(cube, ctypes.c_uint32), _p(zc, ctypes.c_uint32), _p(za, ctypes.c_uint64))
    return zc, za


def eps(d, za: np.ndarray, cs: int) -> float:
    za = np.ascontiguousarray(za, dtype=np.uint64)
    return lib().oracle_eps(_G(d), _p(za, ctypes.c_uint64), cs)


def exp_factor(theta: int, log2_g: int) -> float:
    return lib().oracle_exp_factor(theta, log2_g)


def zmax(d, eps_v: float, E: float) -> int:
    return int(lib().oracle_zmax(_G(d), eps_v, E))


def estimate(log2_g: int, z: int, eps_v: float):
    fl = ctypes.c_uint32(0)
    est = lib().oracle_estimate(log2_g, z, eps_v, ctypes.byref(fl))
    return float(np.float32(est)), int(fl.value)


# --- Alg. 2 + Alg. 3 ------------------------------------------------------------------------

def detect(d, cube: np.ndarray, theta: int, cap: int = 1 << 20) -> dict:
    """Hosts restored by Alg. 2 + Alg. 3 on every CS, sorted by ip."""
    S, nra = 1 << d["r"], d["n_ra"]
    out = (OracleHost * cap)()
    eps_o = np.zeros(S, dtype=np.float64)
    zmax_o = np.zeros(S, dtype=np.int64)
    nhot = np.zeros((S, nra), dtype=np.uint64)
    n = lib().oracle_detect(_G(d), _p(cube, ctypes.c_uint32), theta, out, cap,
                            _p(eps_o, ctypes.c_double), _p(zmax_o, ctypes.c_int64), _p(nhot, ctypes.c_uint64))
    if n > cap:
        return detect(d, cube, theta, cap=int(n))
    hosts = np.frombuffer(out, dtype=HOST_DTYPE, count=int(n)).copy()
    hosts.sort(order="ip")
    return {"hosts": hosts, "eps": eps_o, "zmax": zmax_o, "n_hot": nhot}


def bruteforce(d, cube: np.ndarray, zmax_cs: np.ndarray, nthreads: int | None = None,
               cap: int = 1 << 20) -> np.ndarray:
    """Every ip with Z_U(ip) <= Zmax(cs(ip)), by scanning all 2^32 addresses; sorted."""
    zmax_cs = np.ascontiguousarray(zmax_cs, dtype=np.int64)
    out = np.zeros(cap, dtype=np.uint32)
    n = lib().oracle_bruteforce(_G(d), _p(cube, ctypes.c_uint32), _p(zmax_cs, ctypes.c_int64),
                                _p(out, ctypes.c_uint32), cap, nthreads or os.cpu_count() or 1)
    if n > cap:
        raise RuntimeError(f"brute force found {n} > cap {cap}")
    return np.sort(out[:n])


def union_zeros(d, cube: np.ndarray, ip: int) -> int:
    return int(lib().oracle_union_zeros(_G(d), _p(cube, ctypes.c_uint32), ip))


# --- the inner/outer model of Section III ----------------------------------------------------

def in_prefixes(x: np.ndarray, prefixes) -> np.ndarray:
    """True where address x lies in one of the CIDR prefixes [(address, length)] of NI."""
    x = np.asarray(x, dtype=np.uint64)
    hit = np.zeros(x.shape, dtype=bool)
    for addr, length in prefixes:
        mask = ((0xFFFFFFFF << (32 - length)) & 0xFFFFFFFF) if length else 0
        hit |= (x & np.uint64(mask)) == np.uint64(int(addr) & mask)
    return hit


def orient(pairs: np.ndarray, prefixes) -> np.ndarray:
    """Section III: an edge router relays packets between the inner network NI and the outer
    network NO, and a host's peers are the outer addresses it sends to or receives from (Def. 1).
    Each raw {src, dst} pair with exactly one address in NI becomes {inner, outer}; pairs with both
    or neither address in NI are not traffic between NI and NO and are dropped.  Order is kept."""
    pairs = np.asarray(pairs, dtype=np.uint32)
    a_in = in_prefixes(pairs[:, 0], prefixes)
    b_in = in_prefixes(pairs[:, 1], prefixes)
    keep = a_in != b_in
    out = pairs[keep].copy()
    flip = b_in[keep]
    out[flip] = out[flip][:, ::-1]
    return out


# --- exact baseline (Section V.A) and Eq. 2 / Eq. 3 -----------------------------------------

def exact_counts(pairs: np.ndarray):
    """(ips ascending, distinct peer counts) of every source in ``pairs``."""
    pairs = np.ascontiguousarray(pairs, dtype=np.uint32)
    n = pairs.shape[0]
    keys = np.empty(n, dtype=np.uint64)
    ips = np.empty(n, dtype=np.uint32)
    cnt = np.empty(n, dtype=np.uint32)
    h = lib().oracle_exact_counts(_p(pairs, ctypes.c_uint32), n, _p(keys, ctypes.c_uint64),
                                  _p(ips, ctypes.c_uint32), _p(cnt, ctypes.c_uint32))
    return ips[:h].copy(), cnt[:h].copy()


def fnr_fpr(detected_ips: np.ndarray, exact_ips: np.ndarray, exact_cnt: np.ndarray, theta: int):
    """Eq. 2 and Eq. 3 of Section V.B.

    H = hosts with cardinality >= theta (Def. 1).  FNR = |H \\ detected| / |H|.
    FP set: detected hosts whose cardinality is below theta (the printed
    "<= theta" is read as "< theta" so that H and the FP set are disjoint);
    detected addresses that never appeared have cardinality 0 and count as
    false positives.  FPR = |FP| / |H|, with |H| in the denominator as printed.
    """
    card = dict(zip(exact_ips.tolist(), exact_cnt.tolist()))
    H = {ip for ip, c in card.items() if c >= theta}
    D = set(np.asarray(detected_ips).tolist())
    fn = len(H - D)
    fp = sum(1 for ip in D if card.get(ip, 0) < theta)
    denom = max(1, len(H))
    return fn / denom, fp / denom, len(H)
