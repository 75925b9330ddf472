// Alg. 1 by partition over row tiles: a third way to set the cube's bits,
// with one routed record per packet instead of one per bit.
//
// A row tile is the pair (sketch cs, row word w): for every array a and
// column col it holds the word w of column (cs, a, col) -- sum_a c_a words,
// at most 128 KiB.  All |RA|+|VA| bits of a packet fall into the same row
// tile (they share the sketch and the row, Alg. 1), so a packet is routed
// once, as a record {LP, bit position} (4 bytes when r >= 5, else the
// 8 bytes {mangled iip, row}); the tile assembly recomputes its columns (the
// ring reads and the VA hash of Alg. 1) and sets its bits with shared-memory
// atomics, then ORs every non-zero word into the cube (the words of a row
// tile are one per column, W words apart in the cube).
//
//   1. k_rt_count   : packets per row tile (one shared-memory atomic per
//                     packet), of every packet or of a 1-in-16 sample
//      k_bin_scan   : (shared with the column-tile path) the runs' offsets
//                     (or sampled capacities) and the assembly items
//   2. k_rt_scatter : a block stages its packets' records grouped by row tile
//                     and writes each run out coalesced; with sampled
//                     capacities, records past a run's capacity go to an
//                     overflow list
//   3. k_rt_apply   : per item, assemble the row tile in shared memory and
//                     flush it; then the overflow list, by direct reductions
// Traffic per packet: 8 B read once (plus 8 B more when every packet is
// counted), a 4-byte (r >= 5) or 8-byte record written and read once.
#include <cstring>

#include "cbaa_internal.cuh"
#include "update_binned.h"

namespace cbaa {


namespace {

constexpr uint32_t kCountThreads = 256;
constexpr uint32_t kApplyThreads = 1024;

__device__ __forceinline__ uint2 ld_pair(const uint32_t *p) {
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.global.or.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_or64(uint32_t *p, uint64_t v) {   // p 8-byte aligned
    asm volatile("red.global.or.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t seg_of(const BinSegs &S, uint64_t p) {
    uint32_t s = 0;
    while (s + 1 < S.k && p >= S.start[s + 1]) ++s;
    return s;
}

// Row tile of a packet: router r's tiles come first-to-last as (cs, w).
__device__ __forceinline__ uint32_t row_tile(const Geo &G, uint32_t router, uint32_t m, uint32_t row) {
    return (router * (G.smask + 1) + (m & G.smask)) * G.W + (row >> 5);
}

// A block's own tile numbering.  Its packets lie in consecutive segments
// [s_lo, s_lo + span); when span x (tiles per router) fits nb, tile t of
// segment s is numbered (s - s_lo) x tpr + t, so a block that meets one or
// two routers of many scans, zeroes and reserves only their tiles; otherwise
// the global numbering router x tpr + t is kept.  unit(s) is the multiplier
// of tpr for segment s in either case.
struct BlockTiles {
    uint32_t s_lo, nbl, tpr;
    bool local;
    __device__ uint32_t unit(const BinSegs &S, uint32_t s) const { return local ? s - s_lo : S.router[s]; }
    __device__ uint32_t global(const BinSegs &S, uint32_t lb) const {
        return local ? S.router[s_lo + lb / tpr] * tpr + lb % tpr : lb;
    }
};

__device__ __forceinline__ BlockTiles block_tiles(const Geo &G, const BinSegs &S, uint64_t first, uint64_t last,
                                                   uint32_t nb) {
    BlockTiles B;
    B.tpr = (G.smask + 1) * G.W;
    B.s_lo = seg_of(S, first);
    const uint32_t span = seg_of(S, last) - B.s_lo + 1;
    B.local = (uint64_t)span * B.tpr <= nb;
    B.nbl = B.local ? span * B.tpr : nb;
    return B;
}

// Offset of (array a, column col) inside a row tile.
__device__ __forceinline__ uint32_t tile_off(const Geo &G, uint32_t a, uint32_t col) {
    return G.col_base[a] + col;
}


__device__ __forceinline__ uint4 ld_quad(const uint32_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// MULTI (a pass over several cubes): block b counts the contiguous packets
// [b chunk, (b+1) chunk), chunk a multiple of kCountTile, so that it meets
// few segments and numbers only their tiles (BlockTiles).  Otherwise blocks
// take tiles of kCountTile packets in turn.  A tile that lies inside one
// segment at a 16-byte aligned address (the usual case) is read as two
// 16-byte loads (two packets each) per thread with the segment looked up
// once; any other tile packet by packet.
constexpr uint32_t kCountTile = 4 * kCountThreads;

// ORIENT (the cube has an inner network): packets are raw {src, dst} (orient()).
// RESID: the input is the residual of the heavy split, entries {key, row}
// already oriented (key = heavy_key(iip), so iip = key * kHeavyKeyInv), one segment of regions of rcap entries whose first
// rcount[r] are valid (rcap a multiple of every tile and block size).
// samp > 1: only every samp-th tile of kCountTile packets is counted (a
// sample for run capacities, see sample_capacity).  The first ncount blocks
// count; a residual pass's blocks after them OR the heavy sources' bitmaps
// into their columns (X).
template <bool MULTI, bool ORIENT, bool RESID>
__global__ void __launch_bounds__(kCountThreads) k_rt_count(const Geo G, const BinSegs S, uint64_t n, uint32_t nb,
                                                            uint32_t *__restrict__ counts, uint32_t samp,
                                                            const uint32_t *__restrict__ rcount, uint64_t rcap,
                                                            uint32_t ncount, const HeavyExpand X) {
    extern __shared__ uint32_t hist[];
    if (RESID && blockIdx.x >= ncount) {              // whole blocks: no barrier below is reached
        heavy_expand_part(G, S.cube[0], X, blockIdx.x - ncount, gridDim.x - ncount);
        return;
    }
    uint64_t lo, hi, step;
    if (MULTI) {
        const uint64_t tiles = (n + kCountTile - 1) / kCountTile;
        const uint64_t per = ((tiles + ncount - 1) / ncount + samp - 1) / samp * samp;
        lo = (uint64_t)blockIdx.x * per * kCountTile;
        hi = lo + per * kCountTile < n ? lo + per * kCountTile : n;
        if (lo > hi) lo = hi;                              // a block past the end counts nothing
        step = (uint64_t)kCountTile * samp;
    } else {
        lo = (uint64_t)blockIdx.x * kCountTile * samp;
        hi = n;
        step = (uint64_t)ncount * kCountTile * samp;
    }
    BlockTiles B;
    if (MULTI && lo < hi) {
        B = block_tiles(G, S, lo, hi - 1, nb);
    } else {
        B.s_lo = 0; B.nbl = MULTI ? 0u : nb; B.tpr = (G.smask + 1) * G.W; B.local = false;
    }
    for (uint32_t i = threadIdx.x; i < B.nbl; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint64_t base = lo; base < hi; base += step) {
        uint64_t thi = hi;                            // end of this tile's valid packets
        if (RESID) {
            const uint64_t r = base / rcap, ve = r * rcap + rcount[r];
            if (ve < thi) thi = ve;
            if (base >= thi) continue;
        }
        const uint32_t s = seg_of(S, base);
        const uint32_t *ptr = S.pairs[s] + 2 * (base - S.start[s]);
        const bool fast = base + kCountTile <= thi && base + kCountTile <= S.start[s + 1] &&
                          (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0;
        if (fast) {
            const uint4 q0 = ld_quad(ptr + 4 * threadIdx.x);
            const uint4 q1 = ld_quad(ptr + 4 * (threadIdx.x + kCountThreads));
            const uint32_t rb = B.unit(S, s) * B.tpr;
            uint32_t ip[4] = {q0.x, q0.z, q1.x, q1.z}, oip[4] = {q0.y, q0.w, q1.y, q1.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!RESID && ORIENT && !orient(G, ip[u], oip[u])) continue;      // raw {src, dst} against NI
                const uint32_t row = RESID ? oip[u] : row_of(G, oip[u]);
                const uint32_t iip = RESID ? ip[u] * kHeavyKeyInv : ip[u];
                atomicAdd(&hist[rb + row_tile(G, 0, mangle(G, iip), row)], 1u);
            }
        } else {
            const uint64_t end = base + kCountTile < thi ? base + kCountTile : thi;
            for (uint64_t p = base + threadIdx.x; p < end; p += kCountThreads) {
                const uint32_t sp = seg_of(S, p);
                uint2 v = ld_pair(S.pairs[sp] + 2 * (p - S.start[sp]));
                if (!RESID && ORIENT && !orient(G, v.x, v.y)) continue;
                const uint32_t row = RESID ? v.y : row_of(G, v.y);
                atomicAdd(&hist[row_tile(G, B.unit(S, sp), mangle(G, RESID ? v.x * kHeavyKeyInv : v.x), row)], 1u);
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < B.nbl; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[B.global(S, i)], hist[i]);
}

// SHORT records (r >= 5): lp << 5 | bit in 4 bytes; else {mangled ip, row}.
// Shapes of up to 8 packets per thread are held to 32 registers (4-byte
// records: 2048 threads per SM, measured ~8 % faster) or 42 (8-byte records).
template <int THREADS, int PPT, bool SHORT, bool MULTI, bool ORIENT, bool RESID>
__global__ void __launch_bounds__(THREADS, PPT > 8 ? 1 : (SHORT ? 2048 : 1536) / THREADS) k_rt_scatter(const Geo G, const BinSegs S, uint64_t n, uint32_t nb,
                                                        uint32_t *__restrict__ cursors, void *__restrict__ recs_out,
                                                        const uint32_t *__restrict__ offsets, uint2 *__restrict__ ovf,
                                                        uint32_t *__restrict__ ovf_count, uint32_t ovf_cap,
                                                        const uint32_t *__restrict__ rcount, uint64_t rcap) {
    extern __shared__ uint32_t sm[];
    if (RESID) {                                     // the valid part of this block's residual region
        const uint64_t p0 = (uint64_t)blockIdx.x * THREADS * PPT, r = p0 / rcap, ve = r * rcap + rcount[r];
        if (ve < n) n = ve;
        if (p0 >= n) return;
    }
    uint32_t *hist = sm;
    uint32_t *first = sm + nb;     // exclusive start of each tile's run in `staged`
    uint32_t *delta = sm + 2 * nb;
    uint2 *staged = reinterpret_cast<uint2 *>(sm + ((3 * nb + 1) & ~1u));
    uint32_t *staged1 = reinterpret_cast<uint32_t *>(staged);
    uint32_t *sbin = SHORT ? staged1 + THREADS * PPT : reinterpret_cast<uint32_t *>(staged + THREADS * PPT);
    __shared__ uint32_t tmp[32];
    constexpr uint32_t P = THREADS * PPT;
    const uint64_t p0 = (uint64_t)blockIdx.x * P;
    const uint32_t np = (uint32_t)((n - p0) < P ? (n - p0) : P);
    __shared__ BlockTiles sB;                         // MULTI: kept in shared memory, registers are short here
    if (MULTI) {
        if (threadIdx.x == 0) sB = block_tiles(G, S, p0, p0 + np - 1, nb);
        __syncthreads();
    }
    BlockTiles one;                                   // one cube: the global numbering, folded at compile time
    one.s_lo = 0; one.nbl = nb; one.tpr = (G.smask + 1) * G.W; one.local = false;
    const BlockTiles &B = MULTI ? sB : one;
    for (uint32_t i = threadIdx.x; i < B.nbl; i += THREADS) hist[i] = 0;
    __syncthreads();
    uint2 rec[PPT];
    uint32_t rt[PPT];                                 // the packet's unit (BlockTiles), or none
    // every load issued before any hashing; a block inside one segment at a
    // 16-byte aligned address reads two packets per 16-byte load
    const uint32_t s0 = seg_of(S, p0);
    const uint32_t *ptr0 = S.pairs[s0] + 2 * (p0 - S.start[s0]);
    if (np == P && p0 + P <= S.start[s0 + 1] && (reinterpret_cast<uintptr_t>(ptr0) & 15u) == 0) {
#pragma unroll
        for (uint32_t j = 0; j < PPT / 2; ++j) {
            const uint4 q = ld_quad(ptr0 + 4 * (threadIdx.x + j * THREADS));
            rec[2 * j] = make_uint2(q.x, q.y);
            rec[2 * j + 1] = make_uint2(q.z, q.w);
            rt[2 * j] = rt[2 * j + 1] = B.unit(S, s0);
        }
    } else {
#pragma unroll
        for (uint32_t k = 0; k < PPT; ++k) {
            const uint32_t p = threadIdx.x + k * THREADS;
            rt[k] = 0xFFFFFFFFu;
            if (p < np) {
                const uint64_t gp = p0 + p;
                const uint32_t s = seg_of(S, gp);
                rt[k] = B.unit(S, s);
                rec[k] = __ldg(reinterpret_cast<const uint2 *>(S.pairs[s] + 2 * (gp - S.start[s])));
            }
        }
    }
    // per packet: its record and tile << 16 | its place in the tile's run (tiles < 2^16)
    uint32_t slot[PPT];
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {
        slot[k] = 0xFFFFFFFFu;
        if (rt[k] != 0xFFFFFFFFu) {
            if (!RESID && ORIENT && !orient(G, rec[k].x, rec[k].y)) continue;      // raw {src, dst} against NI
            const uint32_t m = mangle(G, RESID ? rec[k].x * kHeavyKeyInv : rec[k].x);   // RESID: {key, row}
            const uint32_t row = RESID ? rec[k].y : row_of(G, rec[k].y);
            const uint32_t b = row_tile(G, rt[k], m, row);
            if (SHORT) rec[k].x = ((m >> G.r) << 5) | (row & 31u);
            else rec[k] = make_uint2(m, row);
            slot[k] = (b << 16) | atomicAdd(&hist[b], 1u);
        }
    }
    __syncthreads();
    const uint32_t total = block_exclusive_scan(hist, first, B.nbl, tmp);
    // Run reservations in the record buffer.  Only the copy-out needs them:
    // with registers to spare (16 packets per thread) the first KB bins'
    // atomics are issued before the staging and their results wait in
    // registers, so the staging hides their round trip.
    constexpr bool EARLY = PPT > 8;
    constexpr uint32_t KB = EARLY ? 4 : 1;
    uint32_t base[KB];
    // A run reserved at `at`: delta maps staging positions to the record
    // buffer.  With sampled capacities (ovf set) hist[b] becomes the end, in
    // staging positions, of the part of the run that fits before its tile's
    // capacity ends; the rest overflows.
    bool spill = false;                               // some record of this thread's bins overflows
    auto reserved = [&](uint32_t b, uint32_t c, uint32_t at) {
        delta[b] = at - first[b];
        if (ovf) {
            const uint32_t end = offsets[B.global(S, b) + 1];
            const uint32_t room = end > at ? end - at : 0u;
            hist[b] = first[b] + (c < room ? c : room);
            spill |= room < c;
        }
    };
    if (EARLY) {
#pragma unroll
        for (uint32_t k = 0; k < KB; ++k) {
            const uint32_t b = threadIdx.x + k * THREADS;
            const uint32_t c = b < B.nbl ? hist[b] : 0u;
            base[k] = c ? atomicAdd(&cursors[B.global(S, b)], c) : 0u;
        }
    } else {
        for (uint32_t b = threadIdx.x; b < B.nbl; b += THREADS) {
            const uint32_t c = hist[b];
            if (c) reserved(b, c, atomicAdd(&cursors[B.global(S, b)], c));
        }
    }
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {             // first[] is complete after the scan
        if (slot[k] != 0xFFFFFFFFu) {
            const uint32_t b = slot[k] >> 16;
            const uint32_t pos = first[b] + (slot[k] & 0xFFFFu);
            if (SHORT) staged1[pos] = rec[k].x;
            else staged[pos] = rec[k];
            sbin[pos] = b;
        }
    }
    if (EARLY) {
#pragma unroll
        for (uint32_t k = 0; k < KB; ++k) {
            const uint32_t b = threadIdx.x + k * THREADS;
            if (b < B.nbl) {
                const uint32_t c = hist[b];
                if (c) reserved(b, c, base[k]);
            }
        }
        for (uint32_t b = threadIdx.x + KB * THREADS; b < B.nbl; b += THREADS) {
            const uint32_t c = hist[b];
            if (c) reserved(b, c, atomicAdd(&cursors[B.global(S, b)], c));
        }
    }
    const bool any_spill = __syncthreads_or(spill);
    if (!any_spill) {                                 // nothing overflows: the plain copy-out
        if (SHORT) {
            uint32_t *recs = static_cast<uint32_t *>(recs_out);
            for (uint32_t t = threadIdx.x; t < total; t += THREADS) recs[delta[sbin[t]] + t] = staged1[t];
        } else {
            uint2 *recs = static_cast<uint2 *>(recs_out);
            for (uint32_t t = threadIdx.x; t < total; t += THREADS) recs[delta[sbin[t]] + t] = staged[t];
        }
        return;
    }
    // sampled capacities: records past their run's capacity go to the overflow list as
    // {record, tile} (4-byte records) or {mangled ip, row | cube << 16}
    for (uint32_t t = threadIdx.x; t < total; t += THREADS) {
        const uint32_t b = sbin[t];
        if (t < hist[b]) {
            if (SHORT) static_cast<uint32_t *>(recs_out)[delta[b] + t] = staged1[t];
            else static_cast<uint2 *>(recs_out)[delta[b] + t] = staged[t];
        } else {
            const uint32_t gb = B.global(S, b);
            const uint2 e = SHORT ? make_uint2(staged1[t], gb)
                                  : make_uint2(staged[t].x, staged[t].y | ((gb / B.tpr) << 16));
            const uint32_t at = atomicAdd(ovf_count, 1u);
            if (at < ovf_cap) ovf[at] = e;
        }
    }
}

// One overflow entry of a sampled pass: a record that did not fit its run's
// capacity sets its |RA|+|VA| bits straight in the cube (one L2 reduction per
// bit, as the direct update does).  Entries are {record, tile} for 4-byte
// records, {mangled ip, row | cube << 16} otherwise.
template <bool SHORT>
__device__ __forceinline__ void overflow_entry(const Geo &G, const BinSegs &S, uint2 e) {
    const uint32_t tpr = (G.smask + 1) * G.W;
    uint32_t lp, bit, router, cs, w;
    if (SHORT) {
        lp = e.x >> 5;
        bit = e.x & 31u;
        router = e.y / tpr;
        const uint32_t rem = e.y - router * tpr;
        cs = rem / G.W;
        w = rem - cs * G.W;
    } else {
        const uint32_t row = e.y & 0xFFFFu;
        router = e.y >> 16;
        cs = e.x & G.smask;
        lp = e.x >> G.r;
        w = row >> 5;
        bit = row & 31u;
    }
    const size_t off = (size_t)cs * G.cs_words + w;
    for (uint32_t a = 0; a < G.A; ++a) {
        const uint32_t col = a < G.n_ra ? ra_col(G, a, lp) : va_col(G, a - G.n_ra, lp);
        const size_t o = off + G.arr_base[a] + (size_t)col * G.W;
        red_or(S.cube[router] + o, 1u << bit);
        if (S.merge) red_or(S.merge + o, 1u << bit);
    }
}

// Items (a row tile's records, cut into chunks of ch only when a tile holds
// more than ch) are taken from a queue, so blocks that drew small tiles take
// more of them.
// NRA/NVA > 0 fix the array counts at compile time (the 3+1 layout); 0 reads them from G.
// TEST: read a tile word before its atomic and skip bits already set (where
// most sets land on set bits: duplicates and heavy sources); else one
// shared-memory OR per bit (the heavy split's residual: light sources, whose
// bits are mostly still clear).
template <bool TEST>
__device__ __forceinline__ void rt_set(uint32_t *w, uint32_t bit) {
    if (TEST) tile_set_bit(w, bit);
    else atomicOr(w, bit);
}

template <int NRA, int NVA, bool TEST = true>
__device__ __forceinline__ void rt_apply_lp(const Geo &G, uint32_t *tile, uint32_t lp, uint32_t bit) {
    const uint32_t nra = NRA ? NRA : G.n_ra, nva = NRA ? NVA : G.n_va;
#pragma unroll
    for (uint32_t i = 0; i < (NRA ? NRA : CBAA_MAX_RA); ++i) {
        if (NRA == 0 && i >= nra) break;
        rt_set<TEST>(&tile[tile_off(G, i, ra_col(G, i, lp))], bit);
    }
#pragma unroll
    for (uint32_t j = 0; j < (NRA ? NVA : CBAA_MAX_ARRAYS); ++j) {
        if (NRA == 0 && j >= nva) break;
        rt_set<TEST>(&tile[tile_off(G, nra + j, va_col(G, j, lp))], bit);
    }
}

template <int NRA, int NVA, bool TEST = true>
__device__ __forceinline__ void rt_apply_rec(const Geo &G, uint32_t *tile, uint2 rv) {
    rt_apply_lp<NRA, NVA, TEST>(G, tile, rv.x >> G.r, 1u << (rv.y & 31u));
}

template <int NRA, int NVA, bool TEST = true>
__device__ __forceinline__ void rt_apply_rec(const Geo &G, uint32_t *tile, uint32_t rv) {
    rt_apply_lp<NRA, NVA, TEST>(G, tile, rv >> 5, 1u << (rv & 31u));
}

template <int NRA, int NVA, typename Rec>
__global__ void __launch_bounds__(kApplyThreads) k_rt_apply(const Geo G, const BinSegs S,
                                                            const Rec *__restrict__ recs,
                                                            const uint32_t *__restrict__ offsets,
                                                            const uint32_t *__restrict__ item_start, uint32_t nb,
                                                            uint32_t ch, uint32_t tile_words,
                                                            uint32_t *__restrict__ queue,
                                                            const uint32_t *__restrict__ cursors,
                                                            const uint2 *__restrict__ ovf,
                                                            const uint32_t *__restrict__ ovf_count, uint32_t ovf_cap) {
    extern __shared__ __align__(16) uint32_t tile[];
    __shared__ uint32_t s_item;
    const uint32_t items = item_start[nb];
    const uint32_t tiles_per_router = (G.smask + 1) * G.W;
    uint4 *tile4 = reinterpret_cast<uint4 *>(tile);
    const uint32_t quads = tile_words / 4;             // arrays start at multiples of 32 words
    // zeroed once: each flush leaves the words it read zero again
    for (uint32_t q = threadIdx.x; q < quads; q += blockDim.x) tile4[q] = make_uint4(0u, 0u, 0u, 0u);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= items) break;
        uint32_t lo = 0, hi = nb;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_start[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t b = lo;
        const uint32_t c0 = offsets[b] + (item - item_start[b]) * ch;
        // records written: up to the run's end, or fewer when its capacity came from a sample
        const uint32_t cend = offsets[b + 1] < cursors[b] ? offsets[b + 1] : cursors[b];
        const uint32_t c1 = c0 + ch < cend ? c0 + ch : cend;
        if (c0 >= c1) {                                   // an empty item (sampled capacities)
            __syncthreads();                              // s_item is read by every thread first
            continue;
        }
        uint32_t c = c0 + threadIdx.x;
        for (; c + 3 * blockDim.x < c1; c += 4 * blockDim.x) {        // four records in flight
            Rec rv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) rv[u] = __ldcs(recs + c + u * blockDim.x);
#pragma unroll
            for (int u = 0; u < 4; ++u) rt_apply_rec<NRA, NVA>(G, tile, rv[u]);
        }
        for (; c < c1; c += blockDim.x) rt_apply_rec<NRA, NVA>(G, tile, __ldcs(recs + c));
        __syncthreads();
        const uint32_t router = b / tiles_per_router;
        const uint32_t rem = b - router * tiles_per_router;
        const uint32_t cs = rem / G.W, w = rem - cs * G.W;
        uint32_t *cube = S.cube[router] + (size_t)cs * G.cs_words + w;
        // four tile words (four consecutive columns of one array) per step
        for (uint32_t q = threadIdx.x; q < quads; q += blockDim.x) {
            const uint4 v = tile4[q];
            if (!(v.x | v.y | v.z | v.w)) continue;
            const uint32_t t = 4 * q;
            uint32_t a = 0;                                   // array of tile words t .. t+3
            while (a + 1 < G.A && t >= G.col_base[a + 1]) ++a;
            uint32_t *dst = cube + G.arr_base[a] + (size_t)(t - G.col_base[a]) * G.W;
            if (v.x) red_or(dst, v.x);
            if (v.y) red_or(dst + G.W, v.y);
            if (v.z) red_or(dst + 2 * G.W, v.z);
            if (v.w) red_or(dst + 3 * G.W, v.w);
            if (S.merge) {                                    // the global server's OR, in the same pass
                uint32_t *mdst = S.merge + (dst - S.cube[router]);
                if (v.x) red_or(mdst, v.x);
                if (v.y) red_or(mdst + G.W, v.y);
                if (v.z) red_or(mdst + 2 * G.W, v.z);
                if (v.w) red_or(mdst + 3 * G.W, v.w);
            }
            tile4[q] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
    }
    // a sampled pass: blocks leaving the item queue take chunks of the overflow list
    if (!ovf) return;
    const uint32_t n_ovf = *ovf_count < ovf_cap ? *ovf_count : ovf_cap;
    constexpr bool SHORT = sizeof(Rec) == 4;
    for (;;) {
        __syncthreads();                                  // every thread has read the previous chunk
        if (threadIdx.x == 0) s_item = atomicAdd(queue + 1, 1u);
        __syncthreads();
        const uint64_t c0 = (uint64_t)s_item * blockDim.x;
        if (c0 >= n_ovf) break;
        const uint64_t c = c0 + threadIdx.x;
        if (c < n_ovf) overflow_entry<SHORT>(G, S, ovf[c]);
    }
}

// Tiles (cs, 2k) and (cs, 2k + 1) of one cube as one item (item k): both are
// assembled in shared memory, then each column's two row words, adjacent in
// the cube (W is even), are ORed in with one 64-bit reduction, which halves
// the flush's reductions.  For passes whose tiles are of similar size (the
// heavy split's residual), where whole-pair items balance well.
template <int NRA, int NVA, typename Rec>
__global__ void __launch_bounds__(kApplyThreads, 1) k_rt_apply_pair(const Geo G, const BinSegs S,
                                                                    const Rec *__restrict__ recs,
                                                                    const uint32_t *__restrict__ offsets,
                                                                    const uint32_t *__restrict__ cursors,
                                                                    uint32_t npairs, uint32_t tile_words,
                                                                    uint32_t *__restrict__ queue,
                                                                    const uint2 *__restrict__ ovf,
                                                                    const uint32_t *__restrict__ ovf_count,
                                                                    uint32_t ovf_cap) {
    extern __shared__ __align__(16) uint32_t tile[];   // tile 2k, then tile 2k + 1
    __shared__ uint32_t s_item;
    uint32_t *t1 = tile + tile_words;
    const uint4 *a4 = reinterpret_cast<const uint4 *>(tile), *b4 = reinterpret_cast<const uint4 *>(t1);
    const uint32_t quads = tile_words / 4;                 // arrays start at multiples of 32 words
    for (uint32_t q = threadIdx.x; q < 2 * quads; q += blockDim.x)
        reinterpret_cast<uint4 *>(tile)[q] = make_uint4(0u, 0u, 0u, 0u);
    // An item's records as one stream: tile 2k's run, then tile 2k + 1's (records written: up to
    // the run's end, or fewer when its capacity came from a sample).  Items are fetched one
    // ahead, so that the next item's first records load while the current one is flushed.
    struct Stream {
        uint32_t a0, len_a, b0, len;
    };
    auto stream_of = [&](uint32_t kk) {
        Stream st{0u, 0u, 0u, 0u};
        if (kk < npairs) {
            const uint32_t b = 2 * kk;
            const uint32_t a1 = offsets[b + 1] < cursors[b] ? offsets[b + 1] : cursors[b];
            const uint32_t b1 = offsets[b + 2] < cursors[b + 1] ? offsets[b + 2] : cursors[b + 1];
            st.a0 = offsets[b];
            st.len_a = a1 > st.a0 ? a1 - st.a0 : 0u;
            st.b0 = offsets[b + 1];
            st.len = st.len_a + (b1 > st.b0 ? b1 - st.b0 : 0u);
        }
        return st;
    };
    auto rec_at = [&](const Stream &st, uint32_t q) {
        return recs + (q < st.len_a ? st.a0 + q : st.b0 + (q - st.len_a));
    };
    constexpr uint32_t U = 8;                          // records in flight per thread (and the next U)
    const uint32_t T = blockDim.x;
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
    __syncthreads();
    uint32_t k = s_item;
    Stream st = stream_of(k);
    uint32_t pos = threadIdx.x;
    Rec rv[U];
    bool full = pos + (U - 1) * T < st.len;
    if (full) {
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) rv[u] = __ldcs(rec_at(st, pos + u * T));
    }
    while (k < npairs) {
        __syncthreads();                              // the previous flush's zeros are written; s_item read
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1u);
        while (full) {
            const uint32_t pn = pos + U * T;
            const bool next = pn + (U - 1) * T < st.len;
            Rec rn[U];
            if (next) {
#pragma unroll
                for (uint32_t u = 0; u < U; ++u) rn[u] = __ldcs(rec_at(st, pn + u * T));
            }
#pragma unroll
            for (uint32_t u = 0; u < U; ++u)
                rt_apply_rec<NRA, NVA, false>(G, pos + u * T < st.len_a ? tile : t1, rv[u]);
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) rv[u] = rn[u];
            pos = pn;
            full = next;
        }
        for (; pos < st.len; pos += T)
            rt_apply_rec<NRA, NVA, false>(G, pos < st.len_a ? tile : t1, __ldcs(rec_at(st, pos)));
        __syncthreads();                              // the item's tiles are complete
        const uint32_t kn = s_item;
        const Stream sn = stream_of(kn);
        // the next item's first records, in flight during the flush
        pos = threadIdx.x;
        full = pos + (U - 1) * T < sn.len;
        if (full) {
#pragma unroll
            for (uint32_t u = 0; u < U; ++u) rv[u] = __ldcs(rec_at(sn, pos + u * T));
        }
        if (st.len) {                                 // the same for every thread
            const uint32_t cs = (2 * k) / G.W, w = 2 * k - cs * G.W;
            uint32_t *cube = S.cube[0] + (size_t)cs * G.cs_words + w;
            for (uint32_t q = threadIdx.x; q < quads; q += blockDim.x) {
                const uint4 va = a4[q], vb = b4[q];
                if (!(va.x | va.y | va.z | va.w | vb.x | vb.y | vb.z | vb.w)) continue;
                const uint32_t t = 4 * q;
                uint32_t a = 0;                               // array of tile words t .. t+3
                while (a + 1 < G.A && t >= G.col_base[a + 1]) ++a;
                uint32_t *dst = cube + G.arr_base[a] + (size_t)(t - G.col_base[a]) * G.W;
                const uint32_t lo[4] = {va.x, va.y, va.z, va.w}, hi[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (lo[j] | hi[j]) red_or64(dst + j * G.W, ((uint64_t)hi[j] << 32) | lo[j]);
                reinterpret_cast<uint4 *>(tile)[q] = make_uint4(0u, 0u, 0u, 0u);
                reinterpret_cast<uint4 *>(t1)[q] = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        k = kn;
        st = sn;
    }
    // a sampled pass: blocks leaving the item queue take chunks of the overflow list
    if (!ovf) return;
    const uint32_t n_ovf = *ovf_count < ovf_cap ? *ovf_count : ovf_cap;
    constexpr bool SHORT = sizeof(Rec) == 4;
    for (;;) {
        __syncthreads();                                  // every thread has read the previous chunk
        if (threadIdx.x == 0) s_item = atomicAdd(queue + 1, 1u);
        __syncthreads();
        const uint64_t c0 = (uint64_t)s_item * blockDim.x;
        if (c0 >= n_ovf) break;
        const uint64_t c = c0 + threadIdx.x;
        if (c < n_ovf) overflow_entry<SHORT>(G, S, ovf[c]);
    }
}

// Overflow list of a sampled pass (null: exact counts, no overflow).
struct Overflow {
    uint2 *list;
    uint32_t *count;
    uint32_t cap;
};

// Tile tables of a routing block in a pass over several cubes.  A block
// numbers only the tiles of the router segments its packets meet
// (BlockTiles), so its shared-memory tables need span x tiles-per-cube
// entries, span the most segments any block of P packets meets -- one,
// unless a segment starts inside the block's range -- and never more than
// the pass's nb tiles.  Sizing the tables for that instead of nb lets more
// blocks share an SM.
uint32_t routing_table_tiles(const Geo &G, const BinSegs &S, uint32_t nb, uint64_t P) {
    const uint64_t tpr = (uint64_t)(G.smask + 1) * G.W;
    uint64_t span_max = 1;
    for (uint32_t j = 1; j < S.k; ++j) {              // the block holding segment j's first packet
        const uint64_t lo = S.start[j] / P * P, hi = lo + P;
        uint64_t span = 0;
        for (uint32_t t = 0; t < S.k; ++t)
            if (S.start[t] < hi && S.start[t + 1] > lo) ++span;
        if (span > span_max) span_max = span;
    }
    return span_max * tpr < nb ? (uint32_t)(span_max * tpr) : nb;
}

template <int THREADS, int PPT, bool SHORT, bool MULTI, bool ORIENT, bool RESID>
cudaError_t launch_rt_scatter(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W,
                              const Overflow &O, const uint32_t *rcount, uint64_t rcap, cudaStream_t s) {
    // several cubes: every block numbers its own tiles within tables of nbt entries
    const uint32_t nbt = MULTI ? routing_table_tiles(G, S, nb, (uint64_t)THREADS * PPT) : nb;
    const size_t per = SHORT ? 2 : 3;                 // staged record words + bin word per packet
    const size_t smem = sizeof(uint32_t) * (((3 * (size_t)nbt + 1) & ~(size_t)1) + per * THREADS * PPT);
    auto k = k_rt_scatter<THREADS, PPT, SHORT, MULTI, ORIENT, RESID>;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((m + THREADS * PPT - 1) / (THREADS * PPT));
    k<<<blocks, THREADS, smem, s>>>(G, S, m, nbt, W.cursors, W.codes, W.offsets, O.list, O.count, O.cap, rcount,
                                    rcap);
    return cudaGetLastError();
}

template <bool SHORT, bool MULTI, bool ORIENT, bool RESID>
cudaError_t launch_rt_scatter_shape(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W,
                                    const Overflow &O, uint32_t shape, const uint32_t *rcount, uint64_t rcap,
                                    cudaStream_t s) {
    switch (shape) {
        case 1: return launch_rt_scatter<512, 4, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 2: return launch_rt_scatter<1024, 4, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 3: return launch_rt_scatter<256, 8, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 4: return launch_rt_scatter<256, 4, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 5: return launch_rt_scatter<1024, 8, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 6: return launch_rt_scatter<512, 16, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 7: return launch_rt_scatter<256, 16, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        case 8: {
            // 1024 x 16 stages 16Ki records: with 8-byte records or many tiles it exceeds shared memory
            const uint32_t nbt = MULTI ? routing_table_tiles(G, S, nb, 16384) : nb;
            const size_t need = sizeof(uint32_t) * ((((size_t)3 * nbt + 1) & ~(size_t)1) + (SHORT ? 2 : 3) * 16384);
            if (need + 1024 > 227u * 1024u)
                return launch_rt_scatter<512, 16, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
            return launch_rt_scatter<1024, 16, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
        }
        default: return launch_rt_scatter<512, 8, SHORT, MULTI, ORIENT, RESID>(G, S, m, nb, W, O, rcount, rcap, s);
    }
}

template <bool MULTI, bool ORIENT>
cudaError_t launch_rt_scatter_kind(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W,
                                   const Overflow &O, uint32_t shape, cudaStream_t s) {
    return G.r >= 5 ? launch_rt_scatter_shape<true, MULTI, ORIENT, false>(G, S, m, nb, W, O, shape, nullptr, 1, s)
                    : launch_rt_scatter_shape<false, MULTI, ORIENT, false>(G, S, m, nb, W, O, shape, nullptr, 1, s);
}

// Tile pairs fit one block's shared memory.
bool pair_ok(const Geo &G) { return 2ull * sizeof(uint32_t) * G.col_base[G.A] <= 200u * 1024u; }

template <typename Rec>
cudaError_t launch_rt_apply_pair(const Geo &G, const BinSegs &S, const BinWs &W, uint32_t nb, uint32_t tw, int sms,
                                 const uint2 *ovf, const uint32_t *ovf_count, uint32_t ovf_cap, cudaStream_t s) {
    const bool three_one = G.n_ra == 3 && G.n_va == 1;
    auto k = three_one ? k_rt_apply_pair<3, 1, Rec> : k_rt_apply_pair<0, 0, Rec>;
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)tw;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)sms, kApplyThreads, smem, s>>>(G, S, reinterpret_cast<const Rec *>(W.codes), W.offsets, W.cursors,
                                                 nb / 2, tw, W.nchunk + nb, ovf, ovf_count, ovf_cap);
    return cudaGetLastError();
}

template <typename Rec>
cudaError_t launch_rt_apply(const Geo &G, const BinSegs &S, const BinWs &W, uint32_t nb, uint32_t ch, uint32_t tw,
                            size_t smem, int sms, const uint2 *ovf, const uint32_t *ovf_count, uint32_t ovf_cap,
                            cudaStream_t s) {
    const bool three_one = G.n_ra == 3 && G.n_va == 1;
    auto kapply = three_one ? k_rt_apply<3, 1, Rec> : k_rt_apply<0, 0, Rec>;
    cudaError_t e = allow_smem(kapply, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kapply, kApplyThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    kapply<<<(unsigned)(sms * per_sm), kApplyThreads, smem, s>>>(G, S, reinterpret_cast<const Rec *>(W.codes),
                                                                 W.offsets, W.item_start, nb, ch, tw, W.nchunk + nb,
                                                                 W.cursors, ovf, ovf_count, ovf_cap);
    return cudaGetLastError();
}

}  // namespace

uint32_t rowtile_bins(const Geo &G, uint32_t n_cubes) { return n_cubes * (G.smask + 1) * G.W; }
uint32_t rowtile_words(const Geo &G) { return G.col_base[G.A]; }

constexpr uint32_t kSample = 16;                  // sampled passes count 1 tile in 16
constexpr uint64_t kMinSampled = kRowTileMinSampled;

// Words of a sampled pass of m packets: records up to the capacity bound,
// then an overflow list with room for every packet.
static uint64_t sampled_words(uint64_t m, uint32_t nb, uint64_t rec_words) {
    return ((rec_words * sample_capacity_bound(m, nb, kSample, kCountTile) + 3) & ~3ull) + 2 * m + 8;
}

uint64_t rowtile_pass_words(const Geo &G, uint64_t m, bool sampled) {
    const uint64_t rec_words = G.r >= 5 ? 1 : 2;
    return sampled ? sampled_words(m, rowtile_bins(G, 1), rec_words) : rec_words * m;
}

// Largest sampled pass (at most `want` packets) that fits the workspace.
static uint64_t sampled_pass_max(const BinWs &W, uint32_t nb, uint64_t rec_words, uint64_t want) {
    const uint64_t cap_words = W.words;
    if (sampled_words(want, nb, rec_words) <= cap_words) return want;
    uint64_t lo = 0, hi = want;
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (sampled_words(mid, nb, rec_words) <= cap_words) lo = mid; else hi = mid;
    }
    return lo;
}

// One pass over m packets (RESID: the residual regions R, m entries at most,
// the input spans R->nreg * R->rcap positions): counts (or sampled
// capacities), scan, routing, assembly.
template <bool MULTI, bool ORIENT, bool RESID>
static cudaError_t rowtile_pass(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W,
                                const cbaa_tuning &T, bool sampled, const Residual *R, cudaStream_t s) {
    const uint32_t tw = rowtile_words(G);
    const int sms = num_sms();
    const size_t apply_smem = sizeof(uint32_t) * tw;
    const bool short_rec = G.r >= 5;                  // lp (32 - r bits) and the bit fit one word
    const uint64_t rec_words = short_rec ? 1 : 2;
    const uint32_t count_bps = T.count_blocks_per_sm ? T.count_blocks_per_sm : 8;
    const uint32_t apply_ips = T.apply_items_per_sm ? T.apply_items_per_sm : 8;
    const uint32_t samp = sampled ? kSample : 1u;
    auto kcount = k_rt_count<MULTI, ORIENT, RESID>;
    cudaError_t e;
    if ((e = allow_smem(kcount, sizeof(uint32_t) * nb)) != cudaSuccess) return e;
    // counts[nb] is the overflow counter of a sampled pass (a residual pass finds them zeroed by the split)
    if (!RESID && (e = cudaMemsetAsync(W.counts, 0, sizeof(uint32_t) * (nb + 1), s)) != cudaSuccess) return e;
    const uint64_t span = RESID ? (uint64_t)R->nreg * R->rcap : m;      // positions the kernels walk
    const uint32_t *rcount = RESID ? R->rcount : nullptr;
    const uint64_t rcap = RESID ? R->rcap : 1;
    const uint64_t want = (span + (uint64_t)kCountTile * samp - 1) / ((uint64_t)kCountTile * samp);
    const uint64_t cap = (uint64_t)sms * count_bps;
    const unsigned cgrid = (unsigned)(want < cap ? want : cap);
    // split a row tile only when it holds more than apply_ips/2 times the average tile
    uint64_t ch = (m * apply_ips / 2 + nb - 1) / nb;
    if (ch < (1u << 12)) ch = 1u << 12;
    // a residual pass: blocks for the heavy bitmaps' expansion after the counting blocks
    const HeavyExpand X = RESID ? R->x : HeavyExpand{nullptr, nullptr, nullptr, 0};
    uint32_t eblocks = 0;
    if (X.list) {
        const uint64_t ew = (uint64_t)X.kmax * G.A * 32;
        const uint64_t eb = (ew + kCountThreads - 1) / kCountThreads, ecap = (uint64_t)sms * 8;
        eblocks = (uint32_t)(eb < ecap ? eb : ecap);
    }
    kcount<<<cgrid + eblocks, kCountThreads, sizeof(uint32_t) * nb, s>>>(G, S, span, nb, W.counts, samp, rcount,
                                                                          rcap, cgrid, X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_bin_scan(W.counts, nb, (uint32_t)ch, W, s, samp)) != cudaSuccess) return e;
    Overflow O{nullptr, nullptr, 0};
    if (sampled) {
        const uint64_t rec_region = (rec_words * sample_capacity_bound(m, nb, kSample, kCountTile) + 3) & ~3ull;
        O = Overflow{reinterpret_cast<uint2 *>(W.codes + rec_region), W.counts + nb, (uint32_t)m};
    }
    if (RESID)
        e = short_rec ? launch_rt_scatter_shape<true, false, false, true>(G, S, span, nb, W, O, T.scatter_shape, rcount,
                                                                          rcap, s)
                      : launch_rt_scatter_shape<false, false, false, true>(G, S, span, nb, W, O, T.scatter_shape,
                                                                           rcount, rcap, s);
    else
        e = launch_rt_scatter_kind<MULTI, ORIENT>(G, S, m, nb, W, O, T.scatter_shape, s);
    if (e != cudaSuccess) return e;
    if (RESID && pair_ok(G))                         // residual tiles are of similar size: whole pairs
        return short_rec ? launch_rt_apply_pair<uint32_t>(G, S, W, nb, tw, sms, O.list, O.count, O.cap, s)
                         : launch_rt_apply_pair<uint2>(G, S, W, nb, tw, sms, O.list, O.count, O.cap, s);
    return short_rec ? launch_rt_apply<uint32_t>(G, S, W, nb, (uint32_t)ch, tw, apply_smem, sms, O.list, O.count,
                                                 O.cap, s)
                     : launch_rt_apply<uint2>(G, S, W, nb, (uint32_t)ch, tw, apply_smem, sms, O.list, O.count, O.cap,
                                              s);
}

cudaError_t rowtile_pass_residual(const Geo &G, uint32_t *cube, const Residual &R, uint64_t m, const BinWs &W,
                                  const cbaa_tuning &T, bool sampled, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    BinSegs S;
    memset(&S, 0, sizeof S);
    S.pairs[0] = reinterpret_cast<const uint32_t *>(R.entries);
    S.start[0] = 0;
    S.start[1] = (uint64_t)R.nreg * R.rcap;
    S.router[0] = 0;
    S.cube[0] = cube;
    S.k = 1;
    S.n_routers = 1;
    return rowtile_pass<false, false, true>(G, S, m, rowtile_bins(G, 1), W, T, sampled, &R, s);
}

cudaError_t launch_update_rowtile(const Geo &G, const BinSegs &S0, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t nb = rowtile_bins(G, S0.n_routers);
    const bool multi = S0.n_routers > 1, ori = G.n_inner > 0;
    const uint64_t rec_words = G.r >= 5 ? 1 : 2;
    const uint64_t max_pairs = W.words / rec_words;            // counted passes: one record per packet
    // tile_kind 3: run capacities from a 1-in-16 sample of the packets (records
    // past a capacity take the overflow path), where the workspace allows it
    // tile_kind 0 (the default) samples passes of at least kMinSampled packets
    uint64_t max_sampled = 0;
    if (T.tile_kind == 3 || (T.tile_kind == 0 && n >= kMinSampled)) {
        max_sampled = sampled_pass_max(W, nb, rec_words, n);
        // kind 3: any pass of a useful size; kind 0: only where it takes no more passes than counting
        const uint64_t counted = n < max_pairs ? n : max_pairs;
        const uint64_t least = T.tile_kind == 3 ? (n < (1u << 16) ? n : (1u << 16)) : counted;
        if (max_sampled < least) max_sampled = 0;
    }
    const bool sampled = max_sampled > 0;
    for (uint64_t done = 0; done < n;) {
        const uint64_t lim = sampled ? max_sampled : max_pairs;
        const uint64_t m = (n - done) < lim ? (n - done) : lim;
        BinSegs S = S0;
        S.k = 0;
        for (uint32_t j = 0; j < S0.k; ++j) {
            const uint64_t a = S0.start[j] > done ? S0.start[j] : done;
            const uint64_t b = S0.start[j + 1] < done + m ? S0.start[j + 1] : done + m;
            if (a >= b) continue;
            S.pairs[S.k] = S0.pairs[j] + 2 * (a - S0.start[j]);
            S.start[S.k] = a - done;
            S.router[S.k] = S0.router[j];
            ++S.k;
        }
        S.start[S.k] = m;
        cudaError_t e;
        if (multi)
            e = ori ? rowtile_pass<true, true, false>(G, S, m, nb, W, T, sampled, nullptr, s)
                    : rowtile_pass<true, false, false>(G, S, m, nb, W, T, sampled, nullptr, s);
        else
            e = ori ? rowtile_pass<false, true, false>(G, S, m, nb, W, T, sampled, nullptr, s)
                    : rowtile_pass<false, false, false>(G, S, m, nb, W, T, sampled, nullptr, s);
        if (e != cudaSuccess) return e;
        done += m;
    }
    return cudaSuccess;
}

}  // namespace cbaa
