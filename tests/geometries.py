"""Named cube geometries used by the tests and the benchmark (plain data).

Fields follow Section III.A/B of the paper: r CS-selector bits, |RA| restoring
and |VA| validating arrays, g = 2^log2_g rows per column, c_a = 2^cbn[a]
columns per array, ring_off[i] = CL_bs(i) - r (the offset of RA i's column
index inside the left part LP).  Offsets split LP into efficient parts as
evenly as possible, larger parts first.  Seeds are arbitrary constants.
"""

SEEDS = dict(seed_mangle=0x3C6EF372, seed_bv=0xA54FF53A,
             seed_va=[0x510E527F, 0x9B05688C, 0x1F83D9AB, 0x5BE0CD19, 0, 0, 0, 0])


def _geo(r, n_ra, n_va, log2_g, cbn, ring_off, form=0):
    d = dict(r=r, n_ra=n_ra, n_va=n_va, log2_g=log2_g,
             cbn=list(cbn) + [0] * (8 - len(cbn)),
             ring_off=list(ring_off) + [0] * (8 - len(ring_off)),
             threshold_form=form)
    d.update(SEEDS)
    d["seed_va"] = list(SEEDS["seed_va"])
    return d


# The paper's setting (Section V.C): r=4, |RA|=3, |VA|=1, g=2^12, c=2^12 -> 128 MiB.
# L = 28: EP = (10, 9, 9), CP = (2, 3, 3).
PAPER = _geo(4, 3, 1, 12, [12, 12, 12, 12], [0, 10, 19])

# L2-resident geometry for the 64M-packet window: r=5, 3+1, g=2^10, c=2^12 -> 64 MiB.
# L = 27: EP = (9, 9, 9), CP = (3, 3, 3).
L2 = _geo(5, 3, 1, 10, [12, 12, 12, 12], [0, 9, 18])

# Serving geometry: r=6, 3+1, g=2^10, c=2^13 -> 256 MiB.  L = 26: EP = (9, 9, 8), CP = (4, 4, 5).
SERVE = _geo(6, 3, 1, 10, [13, 13, 13, 13], [0, 9, 18])

# Undersized geometry for the saturated regime: r=6, 3+1, g=2^10, c=2^11 -> 64 MiB.
# L = 26: EP = (9, 9, 8), CP = (2, 2, 3).
UNDERSIZED = _geo(6, 3, 1, 10, [11, 11, 11, 11], [0, 9, 18])

# Tiny geometry for the brute-force check over all 2^32 addresses:
# r=6, 3+1, g=2^7, c=2^10 -> 4 MiB.  L = 26: EP = (9, 9, 8), CP = (1, 1, 2).
TINY = _geo(6, 3, 1, 7, [10, 10, 10, 10], [0, 9, 18])

# A second tiny shape with two VAs, unequal column widths and a longer CP:
# r=8, |RA|=3, |VA|=2, g=2^7, cbn=(9, 9, 10 | 7, 8).  L = 24: EP = (8, 8, 8), CP = (1, 1, 2).
TINY2 = _geo(8, 3, 2, 7, [9, 9, 10, 7, 8], [0, 8, 16])

# Four restoring arrays (three join stages; the middle ones both extend and prune):
# r=6, |RA|=4, |VA|=1, g=2^7, cbn=(10, 10, 10, 10 | 9).  L = 26: EP = (7, 7, 6, 6), CP = (3, 3, 4, 4).
QUAD = _geo(6, 4, 1, 7, [10, 10, 10, 10, 9], [0, 7, 14, 20])

# Two restoring arrays (one join stage that both opens and closes the ring) and two VAs:
# r=6, |RA|=2, |VA|=2, g=2^7, cbn=(14, 14 | 10, 11).  L = 26: EP = (13, 13), CP = (1, 1).
DUO = _geo(6, 2, 2, 7, [14, 14, 10, 11], [0, 13])

ALL = dict(PAPER=PAPER, L2=L2, SERVE=SERVE, UNDERSIZED=UNDERSIZED, TINY=TINY, TINY2=TINY2, QUAD=QUAD, DUO=DUO)


def with_form(d, form):
    e = dict(d)
    e["threshold_form"] = form
    return e
