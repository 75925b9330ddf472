"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed
form, an invariant, a brute-force search over all 2^32 addresses, or a
library routine that computes the same quantity another way.  A plausible
mistake anywhere in the oracle (a dropped array, a wrong sign, a transposed
index, a wrong ring offset) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import geometries as GEO
from paper_1901_06207_b300 import traffic as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _popcount_words(words: np.ndarray) -> np.ndarray:
    return np.bitwise_count(words.astype(np.uint32)).astype(np.int64)


# ------------------------------------------------------------------ hashing (Section III.A)

def test_mix32_is_a_bijection(oracle):
    rng = np.random.default_rng(1)
    xs = [0, 1, 2, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF] + rng.integers(0, 1 << 32, 2000).tolist()
    for x in xs:
        assert oracle.unmix32(oracle.mix32(x)) == x
        assert oracle.mix32(oracle.unmix32(x)) == x
    # a bijection on 2^16 consecutive inputs has 2^16 distinct outputs
    outs = {oracle.mix32(x) for x in range(1 << 16)}
    assert len(outs) == 1 << 16


# Known answers of the published "lowbias32" finaliser (C. Wellons,
# hash-prospector), the project's definition of the paper's unspecified
# mangle and hash functions: x ^= x>>16; x *= 0x7feb352d; x ^= x>>15;
# x *= 0x846ca68b; x ^= x>>16 (mod 2^32).  The outputs were worked out once
# step by step from that definition and are stored as literals, so a
# mistyped multiplier or shift in the oracle fails here.
MIX32_KAT = [
    (0x00000000, 0x00000000),
    (0x00000001, 0x688990C0),
    (0x00000002, 0xD1132181),
    (0x00BC614E, 0x4870A1BA),
    (0x80000000, 0xCC4B4124),
    (0xC0FFEE01, 0xA6EC343F),
    (0xDEADBEEF, 0xE628C683),
    (0xFFFFFFFF, 0x6768824A),
]


def _lowbias32_steps(x: int) -> int:
    """The five published steps, one line each, for re-deriving the table."""
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    return x ^ (x >> 16)


@pytest.mark.parametrize("x,y", MIX32_KAT)
def test_mix32_known_answers(oracle, x, y):
    assert _lowbias32_steps(x) == y          # the table is the published function's
    assert oracle.mix32(x) == y
    assert oracle.unmix32(y) == x


def test_hashes_compose_the_finaliser(oracle):
    """mangle(x) = f(x ^ seed_m), H_bv(oip) = f(oip ^ seed_bv) >> (32 - log2 g), H_j(LP) = f(LP ^ seed_j) >>
    (32 - cbn_j): with each input chosen so that the finaliser sees a table entry, the results are
    the table's outputs (top bits for the hashes)."""
    geo = dict(GEO.L2)
    sm, sbv, sva = geo["seed_mangle"], geo["seed_bv"], geo["seed_va"][0]
    for x, y in MIX32_KAT:
        assert oracle.mangle(geo, x ^ sm) == y
        assert oracle.row(geo, x ^ sbv) == y >> (32 - geo["log2_g"])
        assert oracle.va_col(geo, 0, x ^ sva) == y >> (32 - geo["cbn"][geo["n_ra"]])


def test_mix32_avalanche(oracle):
    """Flipping one input bit flips close to half the output bits on average."""
    rng = np.random.default_rng(2)
    flips = []
    for x in rng.integers(0, 1 << 32, 400).tolist():
        y = oracle.mix32(x)
        for b in range(32):
            flips.append(bin(y ^ oracle.mix32(x ^ (1 << b))).count("1"))
    assert 15.0 < np.mean(flips) < 17.0


@pytest.mark.parametrize("name", ["PAPER", "L2", "TINY", "TINY2"])
def test_mangle_roundtrip_and_ranges(oracle, name):
    d = GEO.ALL[name]
    rng = np.random.default_rng(3)
    g, L = 1 << d["log2_g"], 32 - d["r"]
    for ip in [0, 0xFFFFFFFF] + rng.integers(0, 1 << 32, 500).tolist():
        m = oracle.mangle(d, ip)
        assert oracle.unmangle(d, m) == ip
        assert 0 <= oracle.row(d, ip) < g
        lp = m >> d["r"]
        assert lp < (1 << L)
        for i in range(d["n_ra"]):
            assert 0 <= oracle.ra_col(d, i, lp) < (1 << d["cbn"][i])
        for j in range(d["n_va"]):
            assert 0 <= oracle.va_col(d, j, lp) < (1 << d["cbn"][d["n_ra"] + j])


# ------------------------------------------------------------------ column indices (Section III.B/C)

@pytest.mark.parametrize("name", ["PAPER", "L2", "SERVE", "UNDERSIZED", "TINY", "TINY2", "QUAD", "DUO"])
def test_ep_cp_structure(oracle, name):
    """EPs partition LP; CP(i) is the first |CP(i)| bits of the next column; LP is the EP concatenation."""
    d = GEO.ALL[name]
    nra, L = d["n_ra"], 32 - d["r"]
    eps_ = [oracle.ep_len(d, i) for i in range(nra)]
    cps = [oracle.cp_len(d, i) for i in range(nra)]
    assert sum(eps_) == L
    assert all(c >= 0 for c in cps)
    for i in range(nra):
        assert cps[i] <= eps_[(i + 1) % nra]
    rng = np.random.default_rng(4)
    for lp in rng.integers(0, 1 << L, 300).tolist():
        cols = [oracle.ra_col(d, i, lp) for i in range(nra)]
        # bit k of CL(i) is LP bit (off_i + k) mod L, checked bit by bit
        for i in range(nra):
            for k in range(d["cbn"][i]):
                assert (cols[i] >> k) & 1 == (lp >> ((d["ring_off"][i] + k) % L)) & 1
        for i in range(nra):
            nxt = cols[(i + 1) % nra]
            assert cols[i] >> eps_[i] == nxt & ((1 << cps[i]) - 1)
        rebuilt = 0
        for i in range(nra):
            rebuilt |= (cols[i] & ((1 << eps_[i]) - 1)) << d["ring_off"][i]
        assert rebuilt == lp


def test_paper_geometry_memory(oracle):
    """Section V.C: r=4, |RA|=3, |VA|=1, g=2^12, c=2^12 occupies 128 MB."""
    with open(os.path.join(GOLDEN, "paper_geometry.json")) as f:
        gold = json.load(f)
    d = GEO.PAPER
    assert d["r"] == gold["r"] and d["n_ra"] == gold["n_ra"] and d["n_va"] == gold["n_va"]
    assert 1 << d["log2_g"] == gold["g"] and all(1 << c == gold["c"] for c in d["cbn"][:4])
    assert oracle.cube_words(d) * 4 == gold["memory_mib"] * 2 ** 20


# ------------------------------------------------------------------ Alg. 1 invariants

def _tiny_window(seed, n=1 << 16, planted=40, lo=150, hi=600, hosts=2000, bg_max=60):
    spec = T.TrafficSpec(n_packets=n, n_hosts=hosts, n_planted=planted, planted_lo=lo, planted_hi=hi,
                         planted_dist="uniform", bg_mode="per_host", zipf_a=1.2, bg_max=bg_max, seed=seed)
    return T.make_window(spec)


def test_forward_map_sets_every_bit(oracle):
    """Alg. 1 sets bit H_bv(oip) of each of the |RA|+|VA| columns of every packet and nothing else."""
    d = GEO.TINY2
    w = _tiny_window(11, n=1 << 14)
    cube = oracle.build_cube(d, w.pairs)
    W = (1 << d["log2_g"]) // 32
    A = d["n_ra"] + d["n_va"]
    base = np.cumsum([0] + [(1 << d["cbn"][a]) * W for a in range(A)])
    csw = int(base[-1])
    expect = np.zeros_like(cube)
    for iip, oip in w.pairs.tolist():
        m = oracle.mangle(d, iip)
        cs, lp = m & ((1 << d["r"]) - 1), m >> d["r"]
        rw = oracle.row(d, oip)
        cols = [oracle.ra_col(d, i, lp) for i in range(d["n_ra"])] + \
               [oracle.va_col(d, j, lp) for j in range(d["n_va"])]
        for a, col in enumerate(cols):
            expect[cs * csw + int(base[a]) + col * W + rw // 32] |= np.uint32(1 << (rw % 32))
    assert np.array_equal(cube, expect)
    n_flows = len({(a, b) for a, b in w.pairs.tolist()})
    assert int(_popcount_words(cube).sum()) <= A * n_flows


def test_order_independence_and_duplicates(oracle):
    d = GEO.TINY
    w = _tiny_window(12)
    c1 = oracle.build_cube(d, w.pairs)
    perm = np.random.default_rng(5).permutation(w.pairs.shape[0])
    c2 = oracle.build_cube(d, w.pairs[perm])
    c3 = oracle.build_cube(d, np.concatenate([w.pairs, w.pairs[::3]]))
    assert np.array_equal(c1, c2)
    assert np.array_equal(c1, c3)


def test_merge_homomorphism(oracle):
    """Section III.C: OR-merging per-router cubes gives the cube of the union traffic."""
    d = GEO.TINY2
    w = _tiny_window(13)
    whole = oracle.build_cube(d, w.pairs)
    rid, _ = T.split_by_router(w.pairs, 13, 5)
    merged = oracle.new_cube(d)
    for k in range(5):
        oracle.merge(merged, oracle.build_cube(d, w.pairs[rid == k]))
    assert np.array_equal(merged, whole)
    zero = oracle.new_cube(d)
    oracle.merge(zero, oracle.new_cube(d))
    assert not zero.any()


@pytest.mark.parametrize("nthreads", [1, 2, 3, 8])
def test_threaded_build_is_a_merge(oracle, nthreads):
    """The threaded build ORs private cubes of contiguous shares; Alg. 1 only sets bits, so any split
    gives the one-pair-at-a-time cube, including shares that are empty (n < threads) and bits already set."""
    d = GEO.TINY2
    w = _tiny_window(17)
    whole = oracle.build_cube(d, w.pairs)
    assert np.array_equal(oracle.update_threads(d, oracle.new_cube(d), w.pairs, nthreads), whole)
    few = w.pairs[:5]
    assert np.array_equal(oracle.update_threads(d, oracle.new_cube(d), few, nthreads), oracle.build_cube(d, few))
    head, tail = w.pairs[: len(w.pairs) // 3], w.pairs[len(w.pairs) // 3:]
    assert np.array_equal(oracle.update_threads(d, oracle.build_cube(d, head), tail, nthreads), whole)
    assert not oracle.update_threads(d, oracle.new_cube(d), w.pairs[:0], nthreads).any()


# ------------------------------------------------------------------ zero counts, Thm. 1, theta_bn

def test_zero_counts_match_popcount(oracle):
    d = GEO.TINY2
    cube = oracle.build_cube(d, _tiny_window(14).pairs)
    zc, za = oracle.zero_counts(d, cube)
    W = (1 << d["log2_g"]) // 32
    g, S, A = 1 << d["log2_g"], 1 << d["r"], d["n_ra"] + d["n_va"]
    per_cs = cube.reshape(S, -1)
    off = 0
    for a in range(A):
        c = 1 << d["cbn"][a]
        blk = per_cs[:, off:off + c * W].reshape(S, c, W)
        zeros = g - _popcount_words(blk).sum(axis=2)
        assert np.array_equal(zc[:, a, :c].astype(np.int64), zeros)
        assert np.array_equal(za[:, a].astype(np.int64), zeros.sum(axis=1))
        off += c * W


@pytest.mark.parametrize("form", [0, 1])
def test_empty_cube_closed_forms(oracle, form):
    d = GEO.with_form(GEO.PAPER, form)
    cube = oracle.new_cube(d)
    zc, za = oracle.zero_counts(d, cube)
    g = 1 << d["log2_g"]
    assert (zc == g).all() and (za == (1 << 12) * g).all()
    res = oracle.detect(d, cube, 1024)
    assert (res["eps"] == 0.0).all()
    assert (res["zmax"] == math.floor(g * math.exp(-1024 / g))).all()
    assert res["hosts"].size == 0


def test_zmax_agrees_with_estimate_threshold(oracle):
    """Thm-2 form: Z <= Zmax exactly when the Thm. 2 estimate reaches theta."""
    d = GEO.L2
    g = 1 << d["log2_g"]
    for theta in (512, 1024, 2048):
        E = oracle.exp_factor(theta, d["log2_g"])
        assert E == math.exp(-theta / g)
        for eps in (0.0, 1e-6, 0.003, 0.05, 0.3):
            zm = oracle.zmax(d, eps, E)
            est_hi, _ = oracle.estimate(d["log2_g"], zm, eps)
            est_lo, _ = oracle.estimate(d["log2_g"], zm + 1, eps)
            assert est_hi >= theta * (1 - 1e-6)
            assert est_lo < theta * (1 + 1e-6)


def test_printed_threshold_form(oracle):
    """Printed theta_bn = g(1+eps)E - g eps equals the Thm-2 form at eps = 0 and differs by g eps (1 - 2E)."""
    d0, d1 = GEO.L2, GEO.with_form(GEO.L2, 1)
    g = 1 << d0["log2_g"]
    E = oracle.exp_factor(1024, d0["log2_g"])
    assert oracle.zmax(d0, 0.0, E) == oracle.zmax(d1, 0.0, E)
    for eps in (0.01, 0.1, 0.3):
        t0 = g * (1 - eps) * E
        t1 = g * (1 + eps) * E - g * eps
        assert abs((t1 - t0) - g * eps * (2 * E - 1)) < 1e-9
        assert oracle.zmax(d1, eps, E) in (math.floor(t1), math.floor(t1) - 1, math.floor(t1) + 1)


# ------------------------------------------------------------------ Eq. 1 / Thm. 2 estimator

def test_estimator_special_cases(oracle):
    lg = 10
    g = 1 << lg
    # eps = 0 is linear counting (Eq. 1); it inverts the expected zero count g exp(-n/g)
    for n in (50, 700, 1024, 3000):
        z = g * math.exp(-n / g)
        zi = int(round(z))
        est, fl = oracle.estimate(lg, zi, 0.0)
        assert fl == 0
        assert abs(est - (-g * math.log(zi / g))) <= 1e-6 * max(1.0, est)
        assert abs(est - n) < g * abs(math.log(zi / z)) + 1e-3
    # Thm. 2: the correction is the same as replacing Z by Z_r = Z / (1 - eps)
    for eps in (0.01, 0.2):
        for z in (10, 200, 600):
            a, _ = oracle.estimate(lg, z, eps)
            b = -g * math.log((z / (1 - eps)) / g)
            assert abs(a - b) <= 1e-5 * max(1.0, abs(b))
    # saturation and clamping
    est, fl = oracle.estimate(lg, 0, 0.1)
    assert fl == 1 and abs(est - (-g * math.log(1 / (g * 0.9)))) < 1e-2
    est, fl = oracle.estimate(lg, g, 0.1)
    assert est == 0.0 and fl == 0


def test_single_host_in_empty_cube(oracle):
    """One host alone: Z_U = g - |distinct rows|, eps = (d/(c g))^A, est from Thm. 2."""
    d = GEO.L2
    g, c, A = 1 << d["log2_g"], 1 << 12, 4
    rng = np.random.default_rng(6)
    for n_peers in (1, 37, 900, 2500):
        host = int(rng.integers(0, 1 << 32))
        peers = rng.choice(1 << 32, size=n_peers, replace=False).astype(np.uint32)
        pairs = np.stack([np.full(n_peers, host, np.uint32), peers], axis=1)
        cube = oracle.build_cube(d, pairs)
        rows = {oracle.row(d, int(p)) for p in peers}
        z = oracle.union_zeros(d, cube, host)
        assert z == g - len(rows)
        res = oracle.detect(d, cube, 1024)
        cs = oracle.mangle(d, host) & ((1 << d["r"]) - 1)
        p1 = len(rows) / (c * g)
        assert res["eps"][cs] == p1 * p1 * p1 * p1
        detected = res["hosts"]["ip"].tolist()
        assert (host in detected) == (z <= res["zmax"][cs])
        if host in detected:
            h = res["hosts"][res["hosts"]["ip"] == host][0]
            assert h["z"] == z
            want = -g * math.log(z / (g - g * res["eps"][cs]))
            assert abs(h["est"] - want) <= 1e-6 * want


def test_linear_counting_expectation(oracle):
    """E[Z] = g (1 - 1/g)^n for n distinct peers hashed into g rows (the estimator of Eq. 1)."""
    d = GEO.L2
    g = 1 << d["log2_g"]
    n = 1024
    zs = []
    for s in range(40):
        rng = np.random.default_rng(100 + s)
        peers = rng.choice(1 << 32, size=n, replace=False)
        rows = {oracle.row(d, int(p)) for p in peers}
        zs.append(g - len(rows))
    mean = np.mean(zs)
    expect = g * (1 - 1 / g) ** n
    var = g * (1 - 1 / g) ** n + g * (g - 1) * (1 - 2 / g) ** n - expect ** 2
    assert abs(mean - expect) < 4 * math.sqrt(var / len(zs))


# ------------------------------------------------------------------ Alg. 2 + Alg. 3 vs the plain definition

CASES = [("TINY", 128, 0, 21), ("TINY", 96, 1, 22), ("TINY2", 128, 0, 23), ("QUAD", 128, 0, 24),
         ("DUO", 128, 1, 25)]


@pytest.mark.parametrize("name,theta,form,seed", CASES)
def test_restore_equals_bruteforce(oracle, name, theta, form, seed):
    """Alg. 2 + Alg. 3 return exactly {ip : Z_U(ip) <= Zmax(cs)} over all 2^32 addresses."""
    d = GEO.with_form(GEO.ALL[name], form)
    g = 1 << d["log2_g"]
    w = _tiny_window(seed, n=1 << 18, planted=300, lo=int(1.2 * theta), hi=5 * theta,
                     hosts=3000, bg_max=g // 2)
    cube = oracle.build_cube(d, w.pairs)
    res = oracle.detect(d, cube, theta)
    brute = oracle.bruteforce(d, cube, res["zmax"])
    got = res["hosts"]["ip"]
    assert np.unique(got).size == got.size
    assert np.array_equal(np.sort(got), brute)
    assert got.size >= 250         # most planted hosts are there
    for h in res["hosts"][:50]:
        assert oracle.union_zeros(d, cube, int(h["ip"])) == h["z"]


# ------------------------------------------------------------------ detection on the 1M-packet window

def test_planted_hosts_detected_on_1m_window(oracle):
    d = GEO.PAPER
    w = T.make_window(T.spec_window_1m())
    cube = oracle.build_cube(d, w.pairs)
    res = oracle.detect(d, cube, 1024)
    det = set(res["hosts"]["ip"].tolist())
    assert set(w.planted_ips.tolist()) <= det
    ips, cnt = oracle.exact_counts(w.pairs)
    card = dict(zip(ips.tolist(), cnt.tolist()))
    assert all(card.get(ip, 0) >= 1000 for ip in det)
    fnr, fpr, nH = oracle.fnr_fpr(res["hosts"]["ip"], ips, cnt, 1024)
    assert nH == 20 and fnr == 0.0 and fpr <= 0.1
    for h in res["hosts"]:
        assert abs(h["est"] - card[int(h["ip"])]) < 0.15 * card[int(h["ip"])]


# ------------------------------------------------------------------ exact baseline and Eq. 2 / Eq. 3

def test_exact_counts_against_sets(oracle):
    rng = np.random.default_rng(7)
    pairs = np.stack([rng.integers(0, 50, 5000), rng.integers(0, 300, 5000)], axis=1).astype(np.uint32)
    ips, cnt = oracle.exact_counts(pairs)
    ref = {}
    for a, b in pairs.tolist():
        ref.setdefault(a, set()).add(b)
    assert ips.tolist() == sorted(ref)
    assert cnt.tolist() == [len(ref[k]) for k in sorted(ref)]


def test_fnr_fpr_definitions(oracle):
    ips = np.array([1, 2, 3, 4, 5], np.uint32)
    cnt = np.array([2000, 1024, 1023, 10, 5000], np.uint32)
    # H = {1, 2, 5}; detected {1, 3, 9}: FN = {2, 5}, FP = {3, 9 (never seen)}
    fnr, fpr, nH = oracle.fnr_fpr(np.array([1, 3, 9]), ips, cnt, 1024)
    assert nH == 3 and fnr == pytest.approx(2 / 3) and fpr == pytest.approx(2 / 3)


# ------------------------------------------------------------------ the inner/outer model (Section III)

def _ip(s: str) -> int:
    return int.from_bytes(bytes(int(x) for x in s.split(".")), "big")


def test_orient_cases_from_section_iii(oracle):
    """Hand-derived from Section III: a packet between NI and NO keeps its inner address first,
    whichever direction it travels; internal (both in NI) and transit (neither) packets are not
    between NI and NO.  Prefix edges: 172.16.0.0/12 spans 172.16.0.0 .. 172.31.255.255."""
    ni = [(_ip("10.0.0.0"), 8), (_ip("172.16.0.0"), 12), (_ip("192.0.2.7"), 32)]
    cases = [(("10.1.2.3", "8.8.8.8"), ("10.1.2.3", "8.8.8.8")),
             (("8.8.8.8", "10.1.2.3"), ("10.1.2.3", "8.8.8.8")),
             (("10.0.0.1", "10.200.0.2"), None),
             (("1.1.1.1", "2.2.2.2"), None),
             (("172.31.255.255", "172.32.0.0"), ("172.31.255.255", "172.32.0.0")),
             (("172.32.0.0", "172.16.0.0"), ("172.16.0.0", "172.32.0.0")),
             (("172.15.255.255", "172.32.0.0"), None),
             (("192.0.2.8", "192.0.2.7"), ("192.0.2.7", "192.0.2.8")),
             (("11.0.0.0", "9.255.255.255"), None)]
    raw = np.array([[_ip(a), _ip(b)] for (a, b), _ in cases], dtype=np.uint32)
    want = np.array([[_ip(a), _ip(b)] for _, w in cases if w for a, b in [w]], dtype=np.uint32)
    assert np.array_equal(oracle.orient(raw, ni), want)


def test_orient_edge_prefixes_and_direction_blindness(oracle):
    rng = np.random.default_rng(12)
    pairs = rng.integers(0, 1 << 32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    assert oracle.orient(pairs, [(0, 0)]).shape == (0, 2)          # /0: every address inner
    assert oracle.orient(pairs, []).shape == (0, 2)                # empty NI: every address outer
    ni = [(_ip("10.0.0.0"), 8)]
    inner = (_ip("10.0.0.0") | (rng.integers(0, 1 << 24, 5000))).astype(np.uint32)
    outer = rng.integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    outer = outer[(outer >> 24) != 10]
    inner = inner[: outer.size]
    fwd = np.stack([inner, outer], axis=1)
    flip = rng.random(inner.size) < 0.5
    raw = fwd.copy()
    raw[flip] = raw[flip][:, ::-1]
    assert np.array_equal(oracle.orient(raw, ni), fwd)
    assert np.array_equal(oracle.orient(fwd, ni), fwd)


def test_host_with_peers_in_both_directions(oracle):
    """Def. 1 counts peers a host sends to or receives from: one host in an empty cube whose
    peers arrive half as destinations, half as sources, plus internal and transit noise,
    has Z_U = g - |distinct rows of its peers|."""
    d = GEO.L2
    g = 1 << d["log2_g"]
    ni = [(_ip("10.20.0.0"), 16)]
    rng = np.random.default_rng(13)
    host = _ip("10.20.3.4")
    peers = rng.choice(np.arange(1 << 31, 1 << 32, dtype=np.uint64), size=700, replace=False).astype(np.uint32)
    out_dir = np.stack([np.full(350, host, np.uint32), peers[:350]], axis=1)
    in_dir = np.stack([peers[350:], np.full(350, host, np.uint32)], axis=1)
    internal = np.array([[host, _ip("10.20.9.9")]] * 40, dtype=np.uint32)
    transit = np.stack([peers[:40], peers[40:80]], axis=1)
    raw = np.concatenate([out_dir, in_dir, internal, transit])
    raw = raw[rng.permutation(raw.shape[0])]
    cube = oracle.build_cube(d, oracle.orient(raw, ni))
    rows = {oracle.row(d, int(p)) for p in peers}
    assert oracle.union_zeros(d, cube, host) == g - len(rows)
    assert int(np.count_nonzero(cube)) <= 4 * (g // 32)          # only the host's A columns are touched
