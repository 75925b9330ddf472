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
    uint32_t k;               // segments
    uint32_t n_routers;       // cubes
    uint32_t tiles_per_seg;   // tiles per cube
    uint32_t seg_words;       // tiles_per_seg << kBinTileBits: offset between cubes in the tile space
};

struct BinWs {
    uint32_t *counts, *offsets, *cursors, *item_start, *nchunk, *codes;
    size_t max_pairs;                     // packets routed per pass (codes hold A per packet)
};

inline size_t bin_align(size_t x) { return (x + 255) / 256 * 256; }

// Five tables of nb + 2 words: per-tile counts (counts[nb] and counts[nb + 1]
// are counters of the row-tile path), offsets, cursors, item starts, chunks.
inline size_t bin_ws_fixed(uint32_t nb) { return 5 * bin_align(sizeof(uint32_t) * ((size_t)nb + 2)); }

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

inline size_t bin_ws_bytes(const Geo &G, uint32_t n_cubes, size_t max_pairs) {
    return bin_ws_fixed(bin_ws_tables(G, n_cubes)) + bin_align(sizeof(uint32_t) * (size_t)G.A * max_pairs);
}

// Carve `bytes` at `base` into a BinWs for n_cubes cubes; false if not even one packet fits.
inline bool bin_ws_make(const Geo &G, uint32_t n_cubes, void *base, size_t bytes, BinWs *W) {
    const uint32_t nb = bin_ws_tables(G, n_cubes);
    const size_t fixed = bin_ws_fixed(nb);
    if (bytes < fixed + sizeof(uint32_t) * G.A) return false;
    size_t m = (bytes - fixed) / (sizeof(uint32_t) * G.A);
    const size_t cap = (size_t)(1u << 31) / G.A;            // code offsets stay 32-bit
    if (m > cap) m = cap;
    char *b = static_cast<char *>(base);
    const size_t step = bin_align(sizeof(uint32_t) * ((size_t)nb + 2));
    W->counts = reinterpret_cast<uint32_t *>(b);
    W->offsets = reinterpret_cast<uint32_t *>(b + step);
    W->cursors = reinterpret_cast<uint32_t *>(b + 2 * step);
    W->item_start = reinterpret_cast<uint32_t *>(b + 3 * step);
    W->nchunk = reinterpret_cast<uint32_t *>(b + 4 * step);
    W->codes = reinterpret_cast<uint32_t *>(b + fixed);
    W->max_pairs = m;
    return true;
}

cudaError_t launch_update_segments(const Geo &G, const BinSegs &S, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                   cudaStream_t s);
cudaError_t launch_update_rowtile(const Geo &G, const BinSegs &S, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                  cudaStream_t s);
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
