/*
 * CBAA CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow restatement of the Cube of Bit Arrays
 * Algorithm of Xu, Ding and Hu, "GPU based Real-time Super Hosts Detection at
 * Distributed Edge Routers" (arXiv 1901.06207).  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this file; the
 * product path never does.  It shares no code, header, table or constant
 * generator with the CUDA library: everything below is written out again
 * from the paper.
 *
 * The cube is built one pair at a time (oracle_update) or by OpenMP threads
 * on private cubes that are OR-ed afterwards (oracle_update_threads); the
 * brute-force restoration check also runs on OpenMP threads.
 *
 * Each function names the passage it follows.  Where the paper is silent or
 * garbled the reading used is stated at the function.  Floating point is
 * IEEE double with every operation written out in a fixed order; build with
 * -ffp-contract=off so no multiply-add is fused.
 *
 * Geometry (Section III.A/B, Fig. 2):
 *   S = 2^r cardinality sketches (CS); each CS holds n_ra restoring arrays
 *   (RA) followed by n_va validating arrays (VA); array a has c_a = 2^cbn[a]
 *   columns of g = 2^log2_g bits.
 * Memory format of the cube: uint32 words, array-major inside a CS:
 *   word index of (cs, a, col, w) = cs*cs_words + arr_base(a) + col*W + w,
 *   with W = g/32, arr_base(a) = sum_{b<a} c_b*W, cs_words = sum_a c_a*W;
 *   row `row` of a column lives in word row/32, bit row%32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_ARRAYS 8

typedef struct {
    uint32_t r;            /* CS selector width: the right r bits of the mangled ip */
    uint32_t n_ra;         /* |RA| */
    uint32_t n_va;         /* |VA| */
    uint32_t log2_g;       /* g = 2^log2_g bits per column */
    uint32_t cbn[OR_MAX_ARRAYS];       /* column-index widths, RA first then VA */
    uint32_t ring_off[OR_MAX_ARRAYS];  /* RA only: CL_bs(i) - r, offset of CL(i) inside LP */
    uint32_t seed_mangle;
    uint32_t seed_bv;
    uint32_t seed_va[OR_MAX_ARRAYS];   /* VA j uses seed_va[j] */
    uint32_t threshold_form;           /* 0: Thm-2 consistent, 1: as printed in Section III.C */
} oracle_geometry;

/* ------------------------------------------------------------------------ */
/* Hashing.  The paper mangles ip addresses with a reversible function
 * (Section III.A, citing reversible sketches) and uses unnamed hash
 * functions H_bv (row) and H_j (VA column) (Alg. 1).  Project definition:
 * the 32-bit "lowbias32" finaliser published by C. Wellons (hash-prospector):
 *   x ^= x>>16; x *= 0x7feb352d; x ^= x>>15; x *= 0x846ca68b; x ^= x>>16.
 * Every step is a bijection of the 32-bit words, so the whole map is one. */

static uint32_t or_mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

/* Multiplicative inverse modulo 2^32 of an odd number, by Newton's iteration
 * y <- y*(2 - a*y), which doubles the number of correct low bits each step. */
static uint32_t or_inverse_odd(uint32_t a)
{
    uint32_t y = a;                 /* correct to 3 bits for odd a */
    for (int i = 0; i < 5; ++i)
        y = y * (2u - a * y);
    return y;
}

/* Inverse of x ^= x >> s for 0 < s < 32: repeat the xor-shift until the
 * shifted term vanishes. */
static uint32_t or_unxorshift(uint32_t y, unsigned s)
{
    uint32_t x = y;
    for (unsigned k = s; k < 32; k += s)
        x = y ^ (x >> s);
    return x;
}

static uint32_t or_unmix32(uint32_t y)
{
    y = or_unxorshift(y, 16);
    y *= or_inverse_odd(0x846ca68bu);
    y = or_unxorshift(y, 15);
    y *= or_inverse_odd(0x7feb352du);
    y = or_unxorshift(y, 16);
    return y;
}

uint32_t oracle_mix32(uint32_t x) { return or_mix32(x); }
uint32_t oracle_unmix32(uint32_t y) { return or_unmix32(y); }

/* mangle / unmangle (Section III.A) */
uint32_t oracle_mangle(const oracle_geometry *G, uint32_t ip) { return or_mix32(ip ^ G->seed_mangle); }
uint32_t oracle_unmangle(const oracle_geometry *G, uint32_t m) { return or_unmix32(m) ^ G->seed_mangle; }

/* bvIdx = H_bv(oip), a row in [0, g) (Alg. 1) */
uint32_t oracle_row(const oracle_geometry *G, uint32_t oip)
{
    return or_mix32(oip ^ G->seed_bv) >> (32u - G->log2_g);
}

/* CL(j) = H_j(LP) in [0, c_j) for validating array j (Alg. 1) */
uint32_t oracle_va_col(const oracle_geometry *G, uint32_t j, uint32_t lp)
{
    uint32_t a = G->n_ra + j;
    return or_mix32(lp ^ G->seed_va[j]) >> (32u - G->cbn[a]);
}

/* CL(i) for restoring array i (Section III.B, Fig. 3): cbn(i) consecutive
 * bits of the left part LP starting at CL_bs(i).  Bit numbering: bit 0 is
 * the least significant; LP has L = 32 - r bits, and a run that passes the
 * top of LP continues at LP bit 0 (the paper's "module ... base 32", read as
 * a wrap inside LP, which is what makes CP(last) the first bits of EP(0)).
 * Bit k of CL(i) is LP bit (ring_off[i] + k) mod L: read from LP written
 * twice in a row, so a run past the top continues at bit 0. */
uint32_t oracle_ra_col(const oracle_geometry *G, uint32_t i, uint32_t lp)
{
    uint32_t L = 32u - G->r;
    uint64_t ring = (uint64_t)lp | ((uint64_t)lp << L);   /* LP followed by LP again */
    uint64_t mask = (1ull << G->cbn[i]) - 1ull;
    return (uint32_t)((ring >> G->ring_off[i]) & mask);
}

/* |EP(i)| = CL_bs((i+1) mod |RA|) - CL_bs(i), taken modulo L so that the
 * last array's efficient part runs up to the top of LP (Section III.C). */
uint32_t oracle_ep_len(const oracle_geometry *G, uint32_t i)
{
    uint32_t L = 32u - G->r;
    uint32_t nxt = G->ring_off[(i + 1) % G->n_ra];
    return (nxt + L - G->ring_off[i]) % L;
}

/* |CP(i)| = cbn(i) - |EP(i)| (Section III.C; Alg. 3 prints "CL(i)", a typo). */
uint32_t oracle_cp_len(const oracle_geometry *G, uint32_t i)
{
    return G->cbn[i] - oracle_ep_len(G, i);
}

/* ------------------------------------------------------------------------ */
/* Cube format helpers */

static uint64_t or_words_per_col(const oracle_geometry *G) { return (1ull << G->log2_g) / 32ull; }

static uint64_t or_arr_base(const oracle_geometry *G, uint32_t a)
{
    uint64_t base = 0;
    for (uint32_t b = 0; b < a; ++b)
        base += (1ull << G->cbn[b]) * or_words_per_col(G);
    return base;
}

static uint64_t or_cs_words(const oracle_geometry *G)
{
    return or_arr_base(G, G->n_ra + G->n_va);
}

uint64_t oracle_cube_words(const oracle_geometry *G)
{
    return (1ull << G->r) * or_cs_words(G);
}

/* Word offsets of the format above, computed once per call. */
typedef struct {
    uint64_t W;                          /* words per column */
    uint64_t arr_base[OR_MAX_ARRAYS + 1];
    uint64_t cs_words;
} or_layout;

static or_layout or_make_layout(const oracle_geometry *G)
{
    or_layout Ly;
    uint32_t A = G->n_ra + G->n_va;
    Ly.W = or_words_per_col(G);
    for (uint32_t a = 0; a <= A && a <= OR_MAX_ARRAYS; ++a)
        Ly.arr_base[a] = or_arr_base(G, a);
    Ly.cs_words = Ly.arr_base[A];
    return Ly;
}

static uint64_t or_col_word0(const or_layout *Ly, uint32_t cs, uint32_t a, uint32_t col)
{
    return (uint64_t)cs * Ly->cs_words + Ly->arr_base[a] + (uint64_t)col * Ly->W;
}

static void or_set_bit(const or_layout *Ly, uint32_t *cube, uint32_t cs, uint32_t a,
                       uint32_t col, uint32_t row)
{
    uint64_t w = or_col_word0(Ly, cs, a, col) + row / 32u;
    cube[w] |= 1u << (row % 32u);
}

static int or_get_bit(const or_layout *Ly, const uint32_t *cube, uint32_t cs, uint32_t a,
                      uint32_t col, uint32_t row)
{
    uint64_t w = or_col_word0(Ly, cs, a, col) + row / 32u;
    return (int)((cube[w] >> (row % 32u)) & 1u);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: update the cube with IP pairs <iip, oip>, one pair at a time.
 * pairs holds n records {iip, oip}. */
void oracle_update(const oracle_geometry *G, uint32_t *cube, const uint32_t *pairs, uint64_t n)
{
    uint32_t smask = (1u << G->r) - 1u;
    or_layout Ly = or_make_layout(G);
    for (uint64_t p = 0; p < n; ++p) {
        uint32_t iip = pairs[2 * p];
        uint32_t oip = pairs[2 * p + 1];
        uint32_t bv = oracle_row(G, oip);
        uint32_t m = oracle_mangle(G, iip);
        uint32_t cs = m & smask;          /* right r bits select the CS */
        uint32_t lp = m >> G->r;          /* left 32-r bits */
        for (uint32_t i = 0; i < G->n_ra; ++i)
            or_set_bit(&Ly, cube, cs, i, oracle_ra_col(G, i, lp), bv);
        for (uint32_t j = 0; j < G->n_va; ++j)
            or_set_bit(&Ly, cube, cs, G->n_ra + j, oracle_va_col(G, j, lp), bv);
    }
}

/* Section III.C: the global server merges same-structure cubes by bitwise OR.
 * (Section IV.B's "all ones, AND" contradicts this and is not followed.) */
void oracle_merge(uint32_t *dst, const uint32_t *src, uint64_t words)
{
    for (uint64_t w = 0; w < words; ++w)
        dst[w] |= src[w];
}

/* Alg. 1 run by nthreads threads, each on a private cube built from its own
 * contiguous share of the pairs, the private cubes then OR-ed into `cube`
 * (the multi-router model of Section III.C: every router keeps a cube of the
 * same structure and the global cube is their OR).  Alg. 1 only sets bits, so
 * the result equals oracle_update over all n pairs for any split; the test
 * suite checks exactly that, which makes this both a second build mode and a
 * merge test.  `cube` may already hold bits; they are kept. */
int oracle_update_threads(const oracle_geometry *G, uint32_t *cube, const uint32_t *pairs, uint64_t n,
                          int nthreads)
{
    uint64_t words = oracle_cube_words(G);
    if (nthreads < 1) nthreads = 1;
    uint32_t **priv = (uint32_t **)calloc((size_t)nthreads, sizeof(uint32_t *));
    if (!priv) return -1;
    int ok = 1;
    for (int t = 0; t < nthreads; ++t) {
        priv[t] = (uint32_t *)calloc((size_t)words, sizeof(uint32_t));
        if (!priv[t]) ok = 0;
    }
    if (ok) {
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
        for (int t = 0; t < nthreads; ++t) {
            uint64_t lo = n * (uint64_t)t / (uint64_t)nthreads;
            uint64_t hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
            oracle_update(G, priv[t], pairs + 2 * lo, hi - lo);
        }
        /* the OR of Section III.C, word by word, the words split across the threads */
#pragma omp parallel for num_threads(nthreads) schedule(static)
        for (int64_t w = 0; w < (int64_t)words; ++w)
            for (int t = 0; t < nthreads; ++t)
                cube[w] |= priv[t][w];
    }
    for (int t = 0; t < nthreads; ++t)
        free(priv[t]);
    free(priv);
    return ok ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* Zero bits of each column (the "z" of Eq. 1), by a bit loop, and the zero
 * total of each array.  zc holds S*A*c_max entries indexed
 * ((cs*A + a) * c_max + col); za holds S*A entries. */
void oracle_zero_counts(const oracle_geometry *G, const uint32_t *cube, uint32_t *zc, uint64_t *za)
{
    uint32_t S = 1u << G->r, A = G->n_ra + G->n_va, g = 1u << G->log2_g;
    uint32_t cmax = 0;
    for (uint32_t a = 0; a < A; ++a)
        if ((1u << G->cbn[a]) > cmax) cmax = 1u << G->cbn[a];
    or_layout Ly = or_make_layout(G);
    for (uint32_t cs = 0; cs < S; ++cs)
        for (uint32_t a = 0; a < A; ++a) {
            uint64_t tot = 0;
            for (uint32_t col = 0; col < (1u << G->cbn[a]); ++col) {
                const uint32_t *cw = cube + or_col_word0(&Ly, cs, a, col);
                uint32_t z = 0;
                for (uint32_t row = 0; row < g; ++row)
                    z += ((cw[row / 32u] >> (row % 32u)) & 1u) ? 0u : 1u;
                zc[((uint64_t)cs * A + a) * cmax + col] = z;
                tot += z;
            }
            za[(uint64_t)cs * A + a] = tot;
        }
}

/* Thm. 1: probability that a union-column bit is set by other flows,
 * eps = prod_a P1(a), where P1(a) is the probability that a bit of array a
 * is one.  The paper writes P1(a) = 1 - exp(-eta/(c(a) g)) but never says
 * how eta is known at the end of a window; the reading used here measures
 * P1(a) directly as the fraction of one bits in array a of this CS (which
 * is Eq. 1 applied to the whole array).  Product taken in array order. */
double oracle_eps(const oracle_geometry *G, const uint64_t *za, uint32_t cs)
{
    uint32_t A = G->n_ra + G->n_va;
    double eps = 1.0;
    for (uint32_t a = 0; a < A; ++a) {
        uint64_t bits = (1ull << G->cbn[a]) << G->log2_g;
        uint64_t ones = bits - za[(uint64_t)cs * A + a];
        double p1 = (double)ones / (double)bits;
        eps = eps * p1;
    }
    return eps;
}

/* E = exp(-theta/g), the zero fraction a host of exactly theta peers leaves
 * in an unshared column (Eq. 1 solved for z). */
double oracle_exp_factor(uint32_t theta, uint32_t log2_g)
{
    double q = (double)theta / (double)(1u << log2_g);
    return exp(-q);
}

/* Hot-column bound theta_bn (Section III.C) and its integer form.
 *  form 1 (as printed):     theta_bn = g(1+eps)E - g*eps
 *  form 0 (Thm-2 solved for est >= theta): theta_bn = g(1-eps)E
 * A count z is "no more than theta_bn" iff z <= floor(theta_bn). */
int64_t oracle_zmax(const oracle_geometry *G, double eps, double E)
{
    double g = (double)(1u << G->log2_g);
    double t;
    if (G->threshold_form == 1) {
        double a = g * (1.0 + eps);
        double b = a * E;
        double c = g * eps;
        t = b - c;
    } else {
        double a = 1.0 - eps;
        double b = g * a;
        t = b * E;
    }
    return (int64_t)floor(t);
}

/* Thm. 2: est = -g ln(Z / (g - g*eps)).  Saturation (Z = 0) is not covered
 * by the paper; read: use Z = 1 and report it.  A negative estimate (Z above
 * g - g*eps) is clamped to 0. */
float oracle_estimate(uint32_t log2_g, uint32_t z, double eps, uint32_t *flags)
{
    double g = (double)(1u << log2_g);
    uint32_t zs = z;
    *flags = 0;
    if (zs == 0) { zs = 1; *flags = 1u; }
    double den = g - g * eps;
    double est = -g * log((double)zs / den);
    if (est < 0.0) est = 0.0;
    return (float)est;
}

/* ------------------------------------------------------------------------ */
/* Restoration on one CS (Alg. 2 then Alg. 3).
 * out records are {ip, z, est (float bits), flags}.  Returns the number of
 * detected hosts (even beyond cap, in which case only cap are written). */

typedef struct { uint32_t ip, z, est_bits, flags; } oracle_host;

static uint32_t or_zero_count_union(const oracle_geometry *G, const uint32_t *cube, uint32_t cs,
                                    const uint32_t *cols)
{
    uint32_t A = G->n_ra + G->n_va, g = 1u << G->log2_g, z = 0;
    or_layout Ly = or_make_layout(G);
    for (uint32_t row = 0; row < g; ++row) {
        int one = 1;
        for (uint32_t a = 0; a < A; ++a)
            one = one & or_get_bit(&Ly, cube, cs, a, cols[a], row);
        z += one ? 0u : 1u;
    }
    return z;
}

uint64_t oracle_detect(const oracle_geometry *G, const uint32_t *cube, uint32_t theta,
                       oracle_host *out, uint64_t cap,
                       double *eps_out, int64_t *zmax_out, uint64_t *n_hot_out)
{
    uint32_t S = 1u << G->r, A = G->n_ra + G->n_va, nra = G->n_ra;
    uint32_t cmax = 0;
    for (uint32_t a = 0; a < A; ++a)
        if ((1u << G->cbn[a]) > cmax) cmax = 1u << G->cbn[a];
    uint32_t *zc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)S * A * cmax);
    uint64_t *za = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S * A);
    oracle_zero_counts(G, cube, zc, za);
    double E = oracle_exp_factor(theta, G->log2_g);
    uint64_t n = 0;

    uint32_t *hc[OR_MAX_ARRAYS];
    uint32_t nhc[OR_MAX_ARRAYS];
    for (uint32_t i = 0; i < nra; ++i)
        hc[i] = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)1 << G->cbn[i]));

    for (uint32_t cs = 0; cs < S; ++cs) {
        double eps = oracle_eps(G, za, cs);
        int64_t zmax = oracle_zmax(G, eps, E);
        if (eps_out) eps_out[cs] = eps;
        if (zmax_out) zmax_out[cs] = zmax;

        /* Alg. 2: HC(i) = columns j in [0, c(i)-1] with no more than theta_bn
         * zero bits (the printed range [0, c(i)] overruns by one). */
        for (uint32_t i = 0; i < nra; ++i) {
            nhc[i] = 0;
            for (uint32_t j = 0; j < (1u << G->cbn[i]); ++j)
                if ((int64_t)zc[((uint64_t)cs * A + i) * cmax + j] <= zmax)
                    hc[i][nhc[i]++] = j;
            if (n_hot_out) n_hot_out[(uint64_t)cs * nra + i] = nhc[i];
        }

        /* Alg. 3 on every tuple of the Cartesian product HC(0) x ... x HC(|RA|-1). */
        int empty = 0;
        for (uint32_t i = 0; i < nra; ++i)
            if (nhc[i] == 0) empty = 1;
        if (empty) continue;
        uint32_t idx[OR_MAX_ARRAYS] = {0};
        for (;;) {
            uint32_t t[OR_MAX_ARRAYS];
            for (uint32_t i = 0; i < nra; ++i)
                t[i] = hc[i][idx[i]];

            /* step 1: CP(i) of hc_i must equal the first |CP(i)| bits of hc_(i+1 mod |RA|) */
            int ok = 1;
            for (uint32_t i = 0; i < nra && ok; ++i) {
                uint32_t ep = oracle_ep_len(G, i), cp = oracle_cp_len(G, i);
                uint32_t mask = (cp == 32u) ? 0xFFFFFFFFu : ((1u << cp) - 1u);
                uint32_t cp_bits = t[i] >> ep;
                uint32_t next_first = t[(i + 1) % nra] & mask;
                if (cp_bits != next_first) ok = 0;
            }
            if (ok) {
                /* step 2: LP is the concatenation of every column's EP */
                uint32_t lp = 0;
                for (uint32_t i = 0; i < nra; ++i) {
                    uint32_t ep = oracle_ep_len(G, i);
                    uint32_t part = t[i] & ((1u << ep) - 1u);
                    lp |= part << G->ring_off[i];
                }
                /* step 3: union column = AND of the RA columns and the VA columns H_j(LP) */
                uint32_t cols[OR_MAX_ARRAYS];
                for (uint32_t i = 0; i < nra; ++i) cols[i] = t[i];
                for (uint32_t j = 0; j < G->n_va; ++j) cols[nra + j] = oracle_va_col(G, j, lp);
                uint32_t z = or_zero_count_union(G, cube, cs, cols);
                /* step 4: keep LP unless the union has more than theta_bn zeros */
                if ((int64_t)z <= zmax) {
                    if (n < cap) {
                        uint32_t m = (lp << G->r) | cs;     /* LP || RP, RP = CS id */
                        oracle_host h;
                        float est;
                        h.ip = oracle_unmangle(G, m);
                        h.z = z;
                        est = oracle_estimate(G->log2_g, z, eps, &h.flags);
                        memcpy(&h.est_bits, &est, sizeof est);
                        out[n] = h;
                    }
                    ++n;
                }
            }
            /* odometer over the tuple space */
            uint32_t k = 0;
            while (k < nra) {
                if (++idx[k] < nhc[k]) break;
                idx[k] = 0;
                ++k;
            }
            if (k == nra) break;
        }
    }
    for (uint32_t i = 0; i < nra; ++i) free(hc[i]);
    free(zc);
    free(za);
    return n;
}

/* ------------------------------------------------------------------------ */
/* The plain definition the restoration must reach: every 32-bit address
 * whose union column has at most Zmax(cs) zero bits.  Brute force over the
 * whole mangled space, one address at a time; the walk goes CS by CS (all
 * 2^L left parts of a CS in a row) and threads only split the range.
 * Returns the count; writes up to cap addresses, unsorted. */
uint64_t oracle_bruteforce(const oracle_geometry *G, const uint32_t *cube, const int64_t *zmax,
                           uint32_t *out, uint64_t cap, int nthreads)
{
    uint64_t found = 0;
    uint32_t nra = G->n_ra, A = nra + G->n_va;
    uint32_t S = 1u << G->r, L = 32u - G->r;
    or_layout Ly = or_make_layout(G);
    uint64_t chunks_per_cs = (L > 12) ? (1ull << (L - 12)) : 1ull;
    uint64_t chunk_len = (1ull << L) / chunks_per_cs;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
    for (int64_t t = 0; t < (int64_t)(S * chunks_per_cs); ++t) {
        uint32_t cs = (uint32_t)((uint64_t)t / chunks_per_cs);
        uint64_t lp0 = ((uint64_t)t % chunks_per_cs) * chunk_len;
        if (zmax[cs] < 0) continue;
        for (uint64_t lp64 = lp0; lp64 < lp0 + chunk_len; ++lp64) {
            uint32_t lp = (uint32_t)lp64;
            uint64_t w0[OR_MAX_ARRAYS];
            for (uint32_t i = 0; i < nra; ++i)
                w0[i] = or_col_word0(&Ly, cs, i, oracle_ra_col(G, i, lp));
            for (uint32_t j = 0; j < G->n_va; ++j)
                w0[nra + j] = or_col_word0(&Ly, cs, nra + j, oracle_va_col(G, j, lp));
            uint32_t z = 0;
            for (uint64_t w = 0; w < Ly.W; ++w) {
                uint32_t acc = 0xFFFFFFFFu;
                for (uint32_t a = 0; a < A; ++a)
                    acc &= cube[w0[a] + w];
                z += 32u - (uint32_t)__builtin_popcount(acc);
            }
            if ((int64_t)z <= zmax[cs]) {
                uint64_t slot;
#pragma omp atomic capture
                slot = found++;
                if (slot < cap) out[slot] = oracle_unmangle(G, (lp << G->r) | cs);
            }
        }
    }
    return found;
}

/* ------------------------------------------------------------------------ */
/* Exact cardinalities (Section V.A: the exact baseline keeps every host's
 * opposite addresses and counts them).  Plain version: sort the 64-bit keys
 * iip<<32 | oip, drop repeated keys, and count the run of each iip.
 * keys is scratch of n entries.  Writes (ip, |OP(ip)|) for each distinct
 * iip in ascending ip order and returns how many there are. */
static int or_cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

uint64_t oracle_exact_counts(const uint32_t *pairs, uint64_t n, uint64_t *keys,
                             uint32_t *ips_out, uint32_t *counts_out)
{
    for (uint64_t p = 0; p < n; ++p)
        keys[p] = ((uint64_t)pairs[2 * p] << 32) | (uint64_t)pairs[2 * p + 1];
    qsort(keys, (size_t)n, sizeof(uint64_t), or_cmp_u64);
    uint64_t hosts = 0;
    for (uint64_t p = 0; p < n; ++p) {
        if (p > 0 && keys[p] == keys[p - 1])
            continue;                              /* same flow seen again */
        uint32_t ip = (uint32_t)(keys[p] >> 32);
        if (hosts == 0 || ips_out[hosts - 1] != ip) {
            ips_out[hosts] = ip;
            counts_out[hosts] = 0;
            ++hosts;
        }
        counts_out[hosts - 1] += 1;
    }
    return hosts;
}

/* Union-column zero count of one given address (the quantity Thm. 2 turns
 * into an estimate), straight from the forward map of Alg. 1. */
uint32_t oracle_union_zeros(const oracle_geometry *G, const uint32_t *cube, uint32_t ip)
{
    uint32_t m = oracle_mangle(G, ip);
    uint32_t cs = m & ((1u << G->r) - 1u);
    uint32_t lp = m >> G->r;
    uint32_t cols[OR_MAX_ARRAYS];
    for (uint32_t i = 0; i < G->n_ra; ++i) cols[i] = oracle_ra_col(G, i, lp);
    for (uint32_t j = 0; j < G->n_va; ++j) cols[G->n_ra + j] = oracle_va_col(G, j, lp);
    return or_zero_count_union(G, cube, cs, cols);
}
