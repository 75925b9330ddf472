"""Seeded synthetic edge-router traffic: (inner ip, outer ip) uint32 pairs.

This module is the one input generator shared by the CPU oracle's tests and
the CUDA path.  It holds none of the detector's arithmetic (no mangling, no
column or row hashing, no estimator): it only produces packets and the
nominal per-host peer counts it planted.

Traffic model (Section III, Def. 1): each packet carries an <iip, oip> pair;
a window is a multiset of such pairs.  The paper measures on a CERNET
backbone trace (Section V.A) that is not available here; these synthetic
windows stand in for it, shaped as follows.

* ``per_host`` background: every background source host gets a peer count
  drawn from a Zipf law truncated to [1, bg_max]; its peers are uniform over
  2^32.
* ``per_pair`` background: every background distinct pair draws its source
  from a Zipf(a) law over a pool of ``n_hosts`` random addresses and its
  destination uniformly over 2^32 (heavy sources then follow Zipf).
* ``n_planted`` planted super hosts get peer counts uniform or log-uniform in
  [planted_lo, planted_hi].
* distinct pairs are then repeated (uniformly chosen) until ``n_packets``
  packets exist, and the packets are shuffled.

All randomness is counter based: value ``i`` of stream ``s`` under seed
``seed`` is SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) applied to a key
derived from (seed, s) plus i, so any slice can be regenerated anywhere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)

# stream tags (any distinct constants)
S_HOSTS, S_PLANT_N, S_BG_N, S_PEERS, S_BG_SRC, S_DUP, S_SHUF, S_PORTS, S_ROUTER_W = range(1, 10)
S_DIR, S_NOISE = 10, 11


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 ``x`` (wrapping)."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    k = splitmix64(np.array([(seed & 0xFFFFFFFFFFFFFFFF) ^ (stream * 0xD1B54A32D192ED03 & 0xFFFFFFFFFFFFFFFF)],
                            dtype=np.uint64))
    return k[0]


def rand_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Values offset..offset+n-1 of counter stream (seed, stream)."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(offset, offset + n, dtype=np.uint64) * _GOLDEN + key
    return splitmix64(ctr)


def rand_unit(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (rand_u64(seed, stream, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def rand_u32(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    return (rand_u64(seed, stream, n, offset) >> np.uint64(32)).astype(np.uint32)


def distinct_u32(seed: int, stream: int, n: int) -> np.ndarray:
    """n distinct uint32 values in random order (counter based)."""
    m = n + n // 8 + 64
    while True:
        v = rand_u32(seed, stream, m)
        _, first = np.unique(v, return_index=True)
        if first.size >= n:
            first.sort()
            return v[first[:n]]
        m *= 2


def zipf_ranks(u: np.ndarray, a: float, kmax: int) -> np.ndarray:
    """Inverse-CDF draw of ranks in [1, kmax] with P(k) proportional to k^-a."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-a))
    idx = np.searchsorted(cdf, u * cdf[-1], side="right")
    return np.minimum(idx, kmax - 1).astype(np.int64) + 1


def index_bijection(i: np.ndarray, bits: int, key: int) -> np.ndarray:
    """A keyed bijection of [0, 2^bits): odd multiplies and in-range xorshifts."""
    mask = np.uint64((1 << bits) - 1)
    k = np.uint64(key & 0xFFFFFFFFFFFFFFFF)
    sh = np.uint64(max(1, (bits + 1) // 2))
    x = i.astype(np.uint64)
    with np.errstate(over="ignore"):
        for mult in (0x9E3779B97F4A7C15, 0xC2B2AE3D27D4EB4F, 0x165667B19E3779F9):
            x = (x + k) & mask
            x = (x * np.uint64(mult | 1)) & mask
            x = x ^ (x >> sh)
    return x


def shuffle_rows(a: np.ndarray, seed: int) -> np.ndarray:
    """Counter-based shuffle of the rows of ``a``."""
    n = a.shape[0]
    if n <= 1:
        return a.copy()
    key = int(stream_key(seed, S_SHUF))
    if n & (n - 1) == 0:
        perm = index_bijection(np.arange(n, dtype=np.uint64), n.bit_length() - 1, key)
        return a[perm.astype(np.int64)]
    order = np.argsort(rand_u64(seed, S_SHUF, n), kind="stable")
    return a[order]


@dataclasses.dataclass(frozen=True)
class TrafficSpec:
    """Shape of one synthetic window (see module docstring)."""
    n_packets: int
    n_hosts: int                 # background source hosts (per_host) or pool size (per_pair)
    n_planted: int
    planted_lo: int
    planted_hi: int
    planted_dist: str = "uniform"      # "uniform" | "loguniform"
    bg_mode: str = "per_host"          # "per_host" | "per_pair"
    zipf_a: float = 1.2
    bg_max: int = 200                  # per_host truncation of the background peer count
    dup_fraction: float | None = None  # per_pair: share of packets that repeat a distinct pair
    seed: int = 0


@dataclasses.dataclass
class Window:
    pairs: np.ndarray            # uint32 [n_packets, 2]: column 0 = iip (src), column 1 = oip (dst)
    planted_ips: np.ndarray      # uint32 [n_planted]
    planted_counts: np.ndarray   # int64 [n_planted], nominal distinct peers
    n_distinct_nominal: int


# Workloads named by what they are.
def spec_window_1m(seed: int = 0xC0FFEE00) -> TrafficSpec:
    """1M packets, 10^4 sources, 20 planted hosts with 1500-5000 peers, Zipf(1.2) background in [1, 200]."""
    return TrafficSpec(n_packets=1 << 20, n_hosts=10_000 - 20, n_planted=20, planted_lo=1500,
                       planted_hi=5000, planted_dist="uniform", bg_mode="per_host", zipf_a=1.2,
                       bg_max=200, dup_fraction=None, seed=seed)


def spec_window_64m(seed: int = 0xC0FFEE01, scale_shift: int = 0) -> TrafficSpec:
    """64M packets, 2^22-host Zipf(1.1) pool, 500 planted hosts log-uniform in [1024, 200k], 30% duplicates.

    ``scale_shift`` k divides packets, pool and planted count by 2^k (same shape, smaller window).
    """
    return TrafficSpec(n_packets=(1 << 26) >> scale_shift, n_hosts=(1 << 22) >> scale_shift,
                       n_planted=max(1, 500 >> scale_shift), planted_lo=1024, planted_hi=200_000,
                       planted_dist="loguniform", bg_mode="per_pair", zipf_a=1.1,
                       dup_fraction=0.30, seed=seed)


def spec_window_256m(seed: int = 0xC0FFEE40) -> TrafficSpec:
    """The 64M window's shape at four times its size: 256M packets, a 2^24-host Zipf(1.1) pool, 2000
    planted hosts log-uniform in [1024, 200k], 30% duplicates (the learned estimator's workload)."""
    return TrafficSpec(n_packets=1 << 28, n_hosts=1 << 24, n_planted=2000, planted_lo=1024, planted_hi=200_000,
                       planted_dist="loguniform", bg_mode="per_pair", zipf_a=1.1, dup_fraction=0.30, seed=seed)


def _planted_counts(spec: TrafficSpec) -> np.ndarray:
    u = rand_unit(spec.seed, S_PLANT_N, spec.n_planted)
    if spec.planted_dist == "uniform":
        c = spec.planted_lo + np.floor(u * (spec.planted_hi - spec.planted_lo + 1))
    else:
        lo, hi = math.log(spec.planted_lo), math.log(spec.planted_hi)
        c = np.floor(np.exp(lo + u * (hi - lo)))
    return np.clip(c, spec.planted_lo, spec.planted_hi).astype(np.int64)


def make_window(spec: TrafficSpec) -> Window:
    seed = spec.seed
    hosts = distinct_u32(seed, S_HOSTS, spec.n_hosts + spec.n_planted)
    planted = hosts[:spec.n_planted]
    pool = hosts[spec.n_planted:]
    pc = _planted_counts(spec)

    if spec.bg_mode == "per_host":
        bg_n = zipf_ranks(rand_unit(seed, S_BG_N, spec.n_hosts), spec.zipf_a, spec.bg_max)
        src = np.concatenate([np.repeat(planted, pc), np.repeat(pool, bg_n)])
    elif spec.bg_mode == "per_pair":
        n_distinct = int(round((1.0 - (spec.dup_fraction or 0.0)) * spec.n_packets))
        n_bg = max(0, n_distinct - int(pc.sum()))
        ranks = zipf_ranks(rand_unit(seed, S_BG_SRC, n_bg), spec.zipf_a, spec.n_hosts)
        src = np.concatenate([np.repeat(planted, pc), pool[ranks - 1]])
    else:
        raise ValueError(spec.bg_mode)

    n_d = int(src.shape[0])
    if n_d > spec.n_packets:           # keep the window size exact
        src = src[:spec.n_packets]
        n_d = spec.n_packets
    dst = rand_u32(seed, S_PEERS, n_d)
    distinct = np.stack([src.astype(np.uint32), dst], axis=1)
    n_rep = spec.n_packets - n_d
    if n_rep > 0:
        pick = (rand_u64(seed, S_DUP, n_rep) % np.uint64(n_d)).astype(np.int64)
        pairs = np.concatenate([distinct, distinct[pick]], axis=0)
    else:
        pairs = distinct
    pairs = shuffle_rows(pairs, seed)
    return Window(pairs=np.ascontiguousarray(pairs, dtype=np.uint32), planted_ips=planted,
                  planted_counts=pc, n_distinct_nominal=n_d)


# ---------------------------------------------------------------------------
# Multi-router split: each packet carries a synthetic 5-tuple (src, dst,
# sport, dport, proto); a router is chosen by hashing it against per-window
# lognormal(sigma) router weights.

def router_weights(seed: int, n_routers: int, sigma: float = 0.8) -> np.ndarray:
    u = rand_unit(seed, S_ROUTER_W, 2 * n_routers)
    u1 = np.maximum(u[:n_routers], 1e-300)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[n_routers:])   # Box-Muller
    w = np.exp(sigma * z)
    return w / w.sum()


def split_by_router(pairs: np.ndarray, seed: int, n_routers: int, sigma: float = 0.8):
    """Return (router id per packet uint8, weights).  Ports and protocol are synthesised per packet."""
    n = pairs.shape[0]
    w = router_weights(seed, n_routers, sigma)
    ports = rand_u64(seed, S_PORTS, n)                 # sport | dport << 16 | proto << 32
    with np.errstate(over="ignore"):
        key = (pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)
        h = splitmix64(key ^ splitmix64(ports & np.uint64(0xFFFFFFFFFF)))
    u = (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    rid = np.searchsorted(np.cumsum(w), u, side="right")
    return np.minimum(rid, n_routers - 1).astype(np.uint8), w


def router_window(spec: TrafficSpec, n_routers: int, sigma: float = 0.8):
    """A window split over n_routers edge routers: (packets grouped by router, packets per router, weights)."""
    w = make_window(spec)
    rid, weights = split_by_router(w.pairs, spec.seed, n_routers, sigma)
    order = np.argsort(rid, kind="stable")
    counts = np.bincount(rid, minlength=n_routers).astype(np.int64)
    return np.ascontiguousarray(w.pairs[order]), counts, weights


def bidirectional_pairs(pairs: np.ndarray, seed: int, prefix: int, length: int, flip: float = 0.5,
                        internal: float = 0.02, transit: float = 0.02) -> np.ndarray:
    """Raw {src, dst} packets of an edge router between an inner network NI = prefix/length and
    the outer network (Section III), made from a window of <inner, outer> pairs: the inner
    address is moved into NI (its low 32 - length bits kept), an outer address that falls in NI
    is moved out of it, a fraction ``flip`` of the packets travel inward (the pair reversed), and
    fractions ``internal`` / ``transit`` of the packets are replaced by NI-to-NI and
    outside-to-outside packets, which are not traffic between NI and NO."""
    pairs = np.asarray(pairs, dtype=np.uint32)
    n = pairs.shape[0]
    mask = ((0xFFFFFFFF << (32 - length)) & 0xFFFFFFFF) if length else 0
    net = np.uint32(prefix & mask)
    inner = (pairs[:, 0] & np.uint32(~mask & 0xFFFFFFFF)) | net
    outer = pairs[:, 1].copy()
    hit = (outer & np.uint32(mask)) == net
    outer[hit] ^= np.uint32(0x80000000 if length else 0)       # out of NI (length >= 1)
    out = np.stack([inner, outer], axis=1)
    v = rand_unit(seed, S_NOISE, n)
    k_int = v < internal
    k_tr = (v >= internal) & (v < internal + transit)
    out[k_int, 1] = out[k_int, 0] ^ np.uint32(1)               # the inner neighbour (length <= 31)
    out[k_tr, 0] = out[k_tr, 1] ^ np.uint32(1)                 # the outer neighbour of the peer
    u = rand_unit(seed, S_DIR, n)
    out[u < flip] = out[u < flip][:, ::-1]
    return out

