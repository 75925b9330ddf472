// Workspace of the partitioned (binned) update: host arithmetic + pointers.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "cbaa_internal.cuh"

namespace cbaa {

constexpr uint32_t kBinTileBits = 15;     // one tile = 2^15 cube words (128 KiB)
constexpr uint32_t kMaxBins = 4096;       // tile id fits the top 12 bits of a code: cube <= 512 MiB

inline uint32_t bin_count(const Geo &G) {
    return (uint32_t)((G.cube_words + (1ull << kBinTileBits) - 1) >> kBinTileBits);
}

struct BinWs {
    uint32_t *counts, *offsets, *cursors, *item_start, *nchunk, *codes;
    size_t max_pairs;                     // packets routed per pass (codes hold A per packet)
};

inline size_t bin_align(size_t x) { return (x + 255) / 256 * 256; }

inline size_t bin_ws_fixed(uint32_t nb) { return 5 * bin_align(sizeof(uint32_t) * ((size_t)nb + 1)); }

inline size_t bin_ws_bytes(const Geo &G, size_t max_pairs) {
    return bin_ws_fixed(bin_count(G)) + bin_align(sizeof(uint32_t) * (size_t)G.A * max_pairs);
}

// Carve `bytes` at `base` into a BinWs; false if not even one packet fits.
inline bool bin_ws_make(const Geo &G, void *base, size_t bytes, BinWs *W) {
    const uint32_t nb = bin_count(G);
    const size_t fixed = bin_ws_fixed(nb);
    if (bytes < fixed + sizeof(uint32_t) * G.A) return false;
    size_t m = (bytes - fixed) / (sizeof(uint32_t) * G.A);
    const size_t cap = (size_t)(1u << 31) / G.A;            // code offsets stay 32-bit
    if (m > cap) m = cap;
    char *b = static_cast<char *>(base);
    const size_t step = bin_align(sizeof(uint32_t) * ((size_t)nb + 1));
    W->counts = reinterpret_cast<uint32_t *>(b);
    W->offsets = reinterpret_cast<uint32_t *>(b + step);
    W->cursors = reinterpret_cast<uint32_t *>(b + 2 * step);
    W->item_start = reinterpret_cast<uint32_t *>(b + 3 * step);
    W->nchunk = reinterpret_cast<uint32_t *>(b + 4 * step);
    W->codes = reinterpret_cast<uint32_t *>(b + fixed);
    W->max_pairs = m;
    return true;
}

cudaError_t launch_update_binned(const Geo &G, uint32_t *cube, const uint32_t *pairs, size_t n, const BinWs &W,
                                 cudaStream_t s);

}  // namespace cbaa
