// Internal definitions shared by the libcbaa translation units (sm_103a).
//
// Geo is the derived, by-value kernel parameter form of cbaa_params: every
// quantity a kernel needs (EP/CP lengths of Section III.C, array word
// offsets of the cube format) is computed once on the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cbaa.h"

namespace cbaa {

struct Geo {
    uint32_t r, L, smask;          // CS bits, LP width, 2^r - 1
    uint32_t n_ra, n_va, A;        // |RA|, |VA|, |RA| + |VA|
    uint32_t log2_g, g, W;         // rows per column, words per column
    uint32_t cmax;                 // max columns of any array
    uint32_t form;                 // threshold form
    uint32_t cbn[CBAA_MAX_ARRAYS];
    uint32_t ring_off[CBAA_MAX_ARRAYS];
    uint32_t ep[CBAA_MAX_ARRAYS];  // |EP(i)| (RA only)
    uint32_t cp[CBAA_MAX_ARRAYS];  // |CP(i)| (RA only)
    uint32_t seed_m, seed_bv;
    uint32_t seed_va[CBAA_MAX_ARRAYS];
    uint32_t arr_base[CBAA_MAX_ARRAYS + 1];  // word offset of array a inside a CS
    uint32_t col_base[CBAA_MAX_ARRAYS + 1];  // arr_base / W: first column of array a among a CS's columns
    uint32_t cs_words;                       // words of one CS
    uint64_t cube_words;
    uint32_t n_inner;                        // NI prefixes (0: pairs arrive as {iip, oip})
    uint32_t inner_net[CBAA_MAX_INNER];      // prefix addresses, masked
    uint32_t inner_mask[CBAA_MAX_INNER];     // prefix masks
};

// Builds Geo from validated params (host).
Geo make_geo(const cbaa_params &p);

// ---------------------------------------------------------------------------
// Hashing (Section III.A mangling, Alg. 1 H_bv and H_j).  The same bijective
// 32-bit finaliser serves all three; see cbaa.h.

__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// mix32 without its last step, for callers that keep only bits 16..31 of the
// result: the last step XORs x >> 16 into bits 0..15 and leaves bits 16..31
// as they are, so mix32(x) >> s == mix32_top(x) >> s for every s >= 16.  The
// row hash keeps the top log2 g <= 15 bits and the VA hash the top cbn <= 16.
// The steps of mix32 after its first one (x ^= x >> 16), without the last.
__host__ __device__ __forceinline__ uint32_t mix32_mid(uint32_t x) {
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    return x;
}
__host__ __device__ __forceinline__ uint32_t mix32_top(uint32_t x) { return mix32_mid(x ^ (x >> 16)); }

// Inverse multipliers modulo 2^32 (a * a^-1 == 1), fixed at compile time by
// Newton's iteration on the host compiler.
constexpr uint32_t inv_odd(uint32_t a) {
    uint32_t y = a;
    for (int i = 0; i < 5; ++i) y = y * (2u - a * y);
    return y;
}
constexpr uint32_t kInvMul1 = inv_odd(0x7feb352du);
constexpr uint32_t kInvMul2 = inv_odd(0x846ca68bu);
static_assert(0x7feb352du * kInvMul1 == 1u, "inverse of the first multiplier");
static_assert(0x846ca68bu * kInvMul2 == 1u, "inverse of the second multiplier");

__host__ __device__ __forceinline__ uint32_t unmix32(uint32_t y) {
    y ^= y >> 16;                 // x ^= x>>16 is its own inverse
    y *= kInvMul2;
    y ^= (y >> 15) ^ (y >> 30);   // inverse of x ^= x>>15
    y *= kInvMul1;
    y ^= y >> 16;
    return y;
}

__host__ __device__ __forceinline__ uint32_t mangle(const Geo &G, uint32_t ip) { return mix32(ip ^ G.seed_m); }
__host__ __device__ __forceinline__ uint32_t unmangle(const Geo &G, uint32_t m) { return unmix32(m) ^ G.seed_m; }

// bvIdx = H_bv(oip): top log2_g bits of the finaliser.
__host__ __device__ __forceinline__ uint32_t row_of(const Geo &G, uint32_t oip) {
    return mix32_top(oip ^ G.seed_bv) >> (32u - G.log2_g);     // shift >= 17
}

// CL(j) = H_j(LP) for validating array j (array index n_ra + j).
__host__ __device__ __forceinline__ uint32_t va_col(const Geo &G, uint32_t j, uint32_t lp) {
    return mix32_top(lp ^ G.seed_va[j]) >> (32u - G.cbn[G.n_ra + j]);   // shift >= 16
}

// CL(i) for restoring array i: cbn(i) bits of the L-bit ring LP starting at
// ring_off[i].  The low part comes from lp >> off, the wrapped part from
// lp << (L - off); bits above 32 are never needed because cbn <= L.
__host__ __device__ __forceinline__ uint32_t ra_col(const Geo &G, uint32_t i, uint32_t lp) {
    const uint32_t off = G.ring_off[i];
    uint32_t v = (lp >> off) | (lp << (G.L - off));   // L - off in [1, 31] since r >= 1
    return v & ((1u << G.cbn[i]) - 1u);
}

// Section III: a packet between NI and NO carries exactly one inner address.
// Puts it first ({iip, oip}) and returns true; returns false for a packet
// with both or neither address in NI.  Only called when G.n_inner > 0.
__host__ __device__ __forceinline__ bool orient(const Geo &G, uint32_t &a, uint32_t &b) {
    bool ia = false, ib = false;
    for (uint32_t k = 0; k < G.n_inner; ++k) {
        ia |= ((a & G.inner_mask[k]) == G.inner_net[k]);
        ib |= ((b & G.inner_mask[k]) == G.inner_net[k]);
    }
    if (ia == ib) return false;
    if (ib) {
        const uint32_t t = a;
        a = b;
        b = t;
    }
    return true;
}

#ifdef __CUDACC__
// Sets a bit of a shared-memory tile that only ever gains bits while it is
// assembled.  A bit that a plain read already shows set stays set, so the
// atomic is issued only for bits still clear: under duplicate packets and
// heavy sources most sets land on set bits, and the read is far cheaper
// than the shared-memory atomic.
__device__ __forceinline__ void tile_set_bit(uint32_t *w, uint32_t bit) {
    if (!(*reinterpret_cast<volatile uint32_t *>(w) & bit)) atomicOr(w, bit);
}
#endif

__host__ __device__ __forceinline__ uint32_t col_word0(const Geo &G, uint32_t cs, uint32_t a, uint32_t col) {
    return cs * G.cs_words + G.arr_base[a] + col * G.W;
}

}  // namespace cbaa

// Host-side launchers implemented in the .cu files.
namespace cbaa {
// CBAA_OK for cudaSuccess, else CBAA_ERR_CUDA with the error remembered for
// cbaa_last_cuda_error() on this host thread.  Every CBAA_ERR_CUDA that the
// library returns goes through it.
int cuda_status(cudaError_t e);
int num_sms();   // SM count of the current device (cached on first use)
// Opts kernel `fn` into `bytes` of dynamic shared memory on the current
// device, once per (kernel, device) and again only when more is asked for,
// so launches on the hot path (and launches recorded into a CUDA graph) do
// not repeat the attribute call.
cudaError_t allow_smem_fn(const void *fn, size_t bytes);
template <typename K>
inline cudaError_t allow_smem(K kernel, size_t bytes) {
    return allow_smem_fn(reinterpret_cast<const void *>(kernel), bytes);
}
cudaError_t launch_update(const Geo &G, uint32_t *cube, const uint32_t *pairs, size_t n, uint32_t blocks_per_sm,
                          cudaStream_t s);
// dst |= OR(srcs); assign: dst = OR(srcs) (dst is not read).
cudaError_t launch_merge(uint32_t *dst, const uint32_t *const *srcs, int k, uint64_t words, cudaStream_t s,
                         bool assign = false);
// Zero counts, ε and Zmax of the sketches [cs_lo, cs_hi) (cs_hi = 0: all).
// za_zeroed: the caller has already zeroed za (else it is zeroed here).
cudaError_t launch_column_stats(const Geo &G, const uint32_t *cube, uint16_t *zc, uint64_t *za,
                                double *eps, int64_t *zmax, double E, cudaStream_t s, uint32_t cs_lo = 0,
                                uint32_t cs_hi = 0, uint32_t *done = nullptr, bool za_zeroed = false);
}  // namespace cbaa
