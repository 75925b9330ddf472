// Partitioned (binned) update: tile-space description, workspace, launch.
#pragma once

#include <cmath>
#include <stddef.h>
#include <stdint.h>

#include "cbaa_internal.cuh"

namespace cbaa {

constexpr uint32_t kBinTileBits = 15;     // one tile = 2^15 cube words (128 KiB)
constexpr uint32_t kMaxBins = 4096;       // tile id fits the top 12 bits of a code: <= 512 MiB of cubes
constexpr uint32_t kMaxRouters = 16;      // cubes fed by one pass
constexpr uint32_t kMaxSegs = 32;         // packet segments of one pass

inline uint32_t tiles_per_cube(const Geo &G) {
    return (uint32_t)((G.cube_words + (1ull << kBinTileBits) - 1) >> kBinTileBits);
}

// Packets of one pass: segment j holds packets [start[j], start[j+1]) of the
// flattened pass, read from pairs[j], and feeds cube[router[j]].
struct BinSegs {
    const uint32_t *pairs[kMaxSegs];
    uint64_t start[kMaxSegs + 1];
    uint32_t router[kMaxSegs];
    uint32_t *cube[kMaxRouters];
    uint32_t *merge;          // or null: every word ORed into a cube is ORed here too (the global cube)
    uint32_t k;               // segments
    uint32_t n_routers;       // cubes
    uint32_t tiles_per_seg;   // tiles per cube
    uint32_t seg_words;       // tiles_per_seg << kBinTileBits: offset between cubes in the tile space
};

inline size_t bin_align(size_t x) { return (x + 255) / 256 * 256; }

// Heavy-source split of a single-cube pass (update_heavy.cu).  The sources
// of most packets of a window are few (super hosts and the head of a Zipf
// law); all |RA|+|VA| columns of a source receive the same row bits (Alg. 1),
// so a heavy source's packets are gathered in one row bitmap of W words in
// shared memory and ORed into its columns once.  Tables:
//   a sample table of 2^15 slots (count, a key) indexed by the top 15 bits of
//   the source key (a multiplicative bijection of the inner address), the
//   heavy sources' keys, their row bitmaps, and counters.  Each split block
//   builds its own lookup image of 2^14 entries (top 14 bits of the key ->
//   its low 18 bits << 14 | heavy index) in shared memory.
constexpr uint32_t kHeavyCountBits = 15;
constexpr uint32_t kHeavyTabBits = 14;
constexpr uint32_t kHeavyTagBits = 32 - kHeavyTabBits;            // 18
constexpr uint32_t kHeavyIdxMask = (1u << kHeavyTabBits) - 1u;     // index field of an entry
constexpr uint32_t kHeavyEmpty = 0xFFFFFFFFu;                      // index field all ones: no source
constexpr uint32_t kHeavyMax = 1024;                               // heavy sources per pass at most
constexpr uint32_t kHeavyBitmapMax = 128u << 10;                   // bytes of row bitmaps per block at most
uint32_t rowtile_bins(const Geo &G, uint32_t n_cubes);             // row tiles of n_cubes cubes
constexpr uint32_t kHeavyMaxRegions = 1024;                        // split blocks (residual regions) at most
// counters: [0], [1] heavy sources taken at or above the threshold and in the
// bin below it, [32 + b] histogram of sample counts by quarter octave, then the
// entries of each residual region
constexpr uint32_t kHeavyCtrHist = 32;                             // 128 bins: quarter octaves
constexpr uint32_t kHeavyHistBins = 128;
constexpr uint32_t kHeavyCtrRegions = kHeavyCtrHist + kHeavyHistBins;
constexpr uint32_t kHeavyCtrWords = kHeavyCtrRegions + kHeavyMaxRegions;
constexpr uint32_t kHeavyRegionAlign = 16384;                      // region capacity unit (largest routing block)

struct HeavyWs {
    uint32_t *count, *key;        // sample table [2^kHeavyCountBits]
    uint32_t *list;               // key of heavy source h [kHeavyMax]
    uint32_t *bits;               // row bitmaps [kHeavyMax][W]
    uint32_t *ctr;                // counters [kHeavyCtrWords]
    uint32_t *rcount() const { return ctr + kHeavyCtrRegions; }
};
// Bytes from HeavyWs::count to the end of HeavyWs::ctr (cleared at the start of a pass).
inline size_t heavy_clear_bytes(const Geo &G) {
    return bin_align(sizeof(uint32_t) << kHeavyCountBits) + bin_align(sizeof(uint32_t) * (size_t)kHeavyMax * G.W) +
           sizeof(uint32_t) * kHeavyCtrWords;
}

inline size_t heavy_ws_bytes(const Geo &G) {
    return 2 * bin_align(sizeof(uint32_t) << kHeavyCountBits) + bin_align(sizeof(uint32_t) * kHeavyMax) + bin_align(sizeof(uint32_t) * (size_t)kHeavyMax * G.W) +
           bin_align(sizeof(uint32_t) * kHeavyCtrWords);
}

struct BinWs {
    uint32_t *counts, *offsets, *cursors, *item_start, *nchunk, *codes;
    size_t max_pairs;                     // packets routed per pass (codes hold A per packet)
    uint64_t words;                       // words of the codes buffer (A + 2 per packet sized for)
    HeavyWs heavy;
};

// Five tables of nb + 2 words: per-tile counts (counts[nb] and counts[nb + 1]
// are counters of the row-tile path), offsets, cursors, item starts, chunks.
inline size_t bin_ws_tables_bytes(uint32_t nb) { return 5 * bin_align(sizeof(uint32_t) * ((size_t)nb + 2)); }

// Row tiles (update_rowtile.cu): one per (cube, sketch, row word), each
// holding one word of every column of its sketch.
constexpr uint32_t kMaxRowTiles = 8192;          // shared-memory tables of the routing kernel
constexpr uint32_t kMaxRowTileWords = 32768;     // 128 KiB tile in shared memory
inline uint32_t rowtile_bins_host(const Geo &G, uint32_t n_cubes) { return n_cubes * (G.smask + 1) * G.W; }
inline bool rowtile_ok(const Geo &G, uint32_t n_cubes) {
    return rowtile_bins_host(G, n_cubes) <= kMaxRowTiles && G.cs_words / G.W <= kMaxRowTileWords;
}

// Tables are sized for whichever tiling is used.
inline uint32_t bin_ws_tables(const Geo &G, uint32_t n_cubes) {
    const uint32_t col = n_cubes * tiles_per_cube(G);
    const uint32_t row = rowtile_ok(G, n_cubes) ? rowtile_bins_host(G, n_cubes) : 0;
    return col > row ? col : row;
}

// Words of the code buffer per packet a workspace is sized for: A codes
// (column tiles), or a residual entry {key, row} of the heavy split
// (2 words) plus a record and an overflow entry of the row-tile pass.
inline size_t bin_ws_words_per_pair(const Geo &G) { return (size_t)G.A + 2; }

inline size_t bin_ws_fixed(const Geo &G, uint32_t nb) { return bin_ws_tables_bytes(nb) + heavy_ws_bytes(G); }

inline size_t bin_ws_bytes(const Geo &G, uint32_t n_cubes, size_t max_pairs) {
    return bin_ws_fixed(G, bin_ws_tables(G, n_cubes)) +
           bin_align(sizeof(uint32_t) * bin_ws_words_per_pair(G) * max_pairs);
}

// Carve `bytes` at `base` into a BinWs for n_cubes cubes; false if not even one packet fits.
inline bool bin_ws_make(const Geo &G, uint32_t n_cubes, void *base, size_t bytes, BinWs *W) {
    const uint32_t nb = bin_ws_tables(G, n_cubes);
    const size_t fixed = bin_ws_fixed(G, nb);
    const size_t per = bin_ws_words_per_pair(G);
    if (bytes < fixed + sizeof(uint32_t) * per) return false;
    uint64_t words = (bytes - fixed) / sizeof(uint32_t);
    if (words > (1ull << 31)) words = 1ull << 31;            // code offsets stay 32-bit
    char *b = static_cast<char *>(base);
    const size_t step = bin_align(sizeof(uint32_t) * ((size_t)nb + 2));
    W->counts = reinterpret_cast<uint32_t *>(b);
    W->offsets = reinterpret_cast<uint32_t *>(b + step);
    W->cursors = reinterpret_cast<uint32_t *>(b + 2 * step);
    W->item_start = reinterpret_cast<uint32_t *>(b + 3 * step);
    W->nchunk = reinterpret_cast<uint32_t *>(b + 4 * step);
    // what a pass clears first (sample counts, row bitmaps, counters) lies in one run
    char *h = b + bin_ws_tables_bytes(nb);
    W->heavy.count = reinterpret_cast<uint32_t *>(h);
    h += bin_align(sizeof(uint32_t) << kHeavyCountBits);
    W->heavy.bits = reinterpret_cast<uint32_t *>(h);
    h += bin_align(sizeof(uint32_t) * (size_t)kHeavyMax * G.W);
    W->heavy.ctr = reinterpret_cast<uint32_t *>(h);
    h += bin_align(sizeof(uint32_t) * kHeavyCtrWords);
    W->heavy.key = reinterpret_cast<uint32_t *>(h);
    h += bin_align(sizeof(uint32_t) << kHeavyCountBits);
    W->heavy.list = reinterpret_cast<uint32_t *>(h);
    W->codes = reinterpret_cast<uint32_t *>(b + fixed);
    W->words = words;
    W->max_pairs = words / G.A;                               // column tiles: A codes per packet
    return true;
}

// assign (one cube): the cube's words become the pass's bits alone (zeroed
// by the heavy split's blocks, or by a memset first on the other paths).
cudaError_t launch_update_segments(const Geo &G, const BinSegs &S, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                   cudaStream_t s, bool assign = false);
cudaError_t launch_update_rowtile(const Geo &G, const BinSegs &S, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                  cudaStream_t s);
// Source key of an inner address, by which the heavy split looks sources up:
// x * an odd constant is a bijection of the 32-bit words, and its top bits mix
// all bits of x (Knuth's multiplicative hashing).  The expansion turns a key
// back into its address.
constexpr uint32_t kHeavyKeyMul = 0x9E3779B1u;
constexpr uint32_t kHeavyKeyInv = inv_odd(kHeavyKeyMul);
static_assert(kHeavyKeyMul * kHeavyKeyInv == 1u, "inverse of the key multiplier");
__host__ __device__ __forceinline__ uint32_t heavy_key(uint32_t ip) { return ip * kHeavyKeyMul; }

// The heavy sources of a split pass, whose row bitmaps the residual's
// counting kernel ORs into their columns (list null: nothing to expand).
struct HeavyExpand {
    const uint32_t *list;          // key of heavy source h
    const uint32_t *ctr;           // [0], [1]: sources taken (see split_select)
    const uint32_t *bits;          // row bitmaps, W words per source
    uint32_t kmax;
};

// Heavy sources taken: the upper ones plus the lower ones that found room.
__host__ __device__ __forceinline__ uint32_t heavy_count(const uint32_t *ctr, uint32_t kmax) {
    const uint32_t t = ctr[0] + ctr[1];
    return t < kmax ? t : kmax;
}

#ifdef __CUDACC__
// Part `part` of `parts` equal parts (blocks of whole warps) of the
// expansion: one warp per (heavy source, array), the source's row bitmap ORed
// into its column of that array, one reduction per non-zero word.
__device__ __forceinline__ void heavy_expand_part(const Geo &G, uint32_t *cube, const HeavyExpand &X, uint32_t part,
                                                  uint32_t parts) {
    const uint32_t nh = heavy_count(X.ctr, X.kmax);
    const uint32_t lane = threadIdx.x & 31u, wpb = blockDim.x / 32;
    const uint32_t warps = parts * wpb;
    for (uint32_t t = part * wpb + threadIdx.x / 32; t < nh * G.A; t += warps) {
        const uint32_t h = t / G.A, a = t - h * G.A;
        const uint32_t m = mangle(G, X.list[h] * kHeavyKeyInv), cs = m & G.smask, lp = m >> G.r;
        const uint32_t col = a < G.n_ra ? ra_col(G, a, lp) : va_col(G, a - G.n_ra, lp);
        uint32_t *dst = cube + (size_t)cs * G.cs_words + G.arr_base[a] + (size_t)col * G.W;
        const uint32_t *src = X.bits + (size_t)h * G.W;
        for (uint32_t w = lane; w < G.W; w += 32) {
            const uint32_t x = src[w];
            if (x) asm volatile("red.global.or.b32 [%0], %1;" :: "l"(dst + w), "r"(x) : "memory");
        }
    }
}
#endif

// Residual of the heavy split: region b holds rcount[b] entries {key, row}
// from entry b * rcap on (rcap a multiple of kHeavyRegionAlign), nreg regions.
struct Residual {
    const uint2 *entries;
    const uint32_t *rcount;
    uint64_t rcap;
    uint32_t nreg;
    HeavyExpand x;                 // done by the residual pass's counting kernel
};
// One row-tile pass over the residual entries of the heavy split (m of them
// at most), with run capacities from a sample when `sampled`; W.codes /
// W.words: the room after the residual regions.  W.counts[0 .. nb] must be
// zero already (the split's histogram kernel clears them).
cudaError_t rowtile_pass_residual(const Geo &G, uint32_t *cube, const Residual &R, uint64_t m, const BinWs &W,
                                  const cbaa_tuning &T, bool sampled, cudaStream_t s);
// Words a row-tile pass of m packets needs in the code buffer (sampled run
// capacities with their overflow list, or exact counts).
uint64_t rowtile_pass_words(const Geo &G, uint64_t m, bool sampled);
constexpr uint64_t kRowTileMinSampled = 8ull << 20;  // below this every packet is counted
// Heavy-source split in front of the row tiles (single cube, update_heavy.cu).
// assign: the split's blocks of the first pass zero the cube first.
cudaError_t launch_update_heavy(const Geo &G, uint32_t *cube, const uint32_t *pairs, uint64_t n, const BinWs &W,
                                const cbaa_tuning &T, cudaStream_t s, bool assign = false);
// Whether the split serves a pass over these cubes with this tuning.
bool heavy_enabled(const Geo &G, uint32_t n_cubes, uint64_t n, const cbaa_tuning &T);
cudaError_t launch_bin_scan(uint32_t *counts, uint32_t nb, uint32_t ch, const BinWs &W, cudaStream_t s,
                            uint32_t samp = 1);

// Run capacity of a tile from its count c in a 1-in-samp sample of the
// packets: the estimate c*samp, plus 1/8 of it, plus four standard
// deviations of the sampled estimate (samp*sqrt(c+1)), plus 256.  Only
// time depends on it: records beyond a run's capacity take the overflow
// path.  sample_capacity_bound() bounds the sum over all tiles.
__host__ __device__ inline uint32_t sample_capacity(uint32_t c, uint32_t samp) {
    const uint64_t est = (uint64_t)c * samp;
    const uint64_t c1 = (uint64_t)c + 1;                  // r = ceil(sqrt(c + 1)), exact
    uint32_t r = (uint32_t)sqrtf((float)c1);
    while ((uint64_t)r * r < c1) ++r;
    while (r > 1 && (uint64_t)(r - 1) * (r - 1) >= c1) --r;
    const uint64_t cap = est + est / 8 + 4ull * samp * r + 256;
    return cap > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)cap;
}

#ifdef __CUDACC__
// Exclusive scan of in[0..n) into out[0..n) by one block (blockDim a
// multiple of 32, at most 1024; in == out allowed); returns the total.
// `tmp` is 32 words of shared memory.
__device__ inline uint32_t block_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *tmp) {
    const uint32_t T = blockDim.x, t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t per = (n + T - 1) / T;
    const uint32_t b0 = t * per < n ? t * per : n;
    const uint32_t b1 = b0 + per < n ? b0 + per : n;
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i) s += in[i];
    uint32_t x = s;                                   // inclusive warp scan of thread sums
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < T / 32 ? tmp[lane] : 0u;
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        tmp[lane] = v;                                // inclusive over warps
    }
    __syncthreads();
    uint32_t run = (warp ? tmp[warp - 1] : 0u) + x - s;
    const uint32_t total = tmp[T / 32 - 1];
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t v = in[i];
        out[i] = run;
        run += v;
    }
    __syncthreads();
    return total;
}

// By one block: offsets = exclusive scan of counts (offsets[nb] = total),
// cursors = offsets, items = exclusive scan of ceil(counts / ch)
// (item_start[nb] = total), and the assembly's queue counters nchunk[nb] and
// nchunk[nb + 1] = 0.
// samp > 1: counts are those of a 1-in-samp sample of the packets and are
// first replaced by run capacities (sample_capacity).
__device__ inline void bin_scan_block(uint32_t *counts, uint32_t nb, uint32_t ch, uint32_t *offsets, uint32_t *cursors,
                                      uint32_t *item_start, uint32_t *nchunk, uint32_t samp, uint32_t *tmp) {
    if (samp > 1) {
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) counts[i] = sample_capacity(counts[i], samp);
        __syncthreads();
    }
    const uint32_t total = block_exclusive_scan(counts, offsets, nb, tmp);
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        cursors[i] = offsets[i];
        nchunk[i] = (counts[i] + ch - 1) / ch;
    }
    if (threadIdx.x == 0) offsets[nb] = total;
    __syncthreads();
    const uint32_t items = block_exclusive_scan(nchunk, item_start, nb, tmp);
    if (threadIdx.x == 0) {
        item_start[nb] = items;
        nchunk[nb] = 0;
        nchunk[nb + 1] = 0;
    }
}
#endif

// Upper bound of sum_b sample_capacity(c_b, samp) when m packets are
// sampled in tiles of `tile` (sum_b c_b <= m/samp + tile): the estimates sum
// to at most m + samp*tile, and sum_b sqrt(c_b + 1) <= sqrt(nb * sum(c_b + 1))
// (Cauchy-Schwarz), plus one per tile for the ceiling.
inline uint64_t sample_capacity_bound(uint64_t m, uint32_t nb, uint32_t samp, uint32_t tile) {
    const uint64_t est = m + (uint64_t)samp * tile;
    const double rt = std::sqrt((double)nb * ((double)est / samp + (double)tile + nb)) + nb;
    return est + est / 8 + (uint64_t)(4.0 * samp * rt) + 4ull * samp + 257ull * nb;
}

}  // namespace cbaa
