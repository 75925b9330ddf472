// Alg. 1 by partition: the same cube bits as the direct update, set without
// L2 atomics on hot columns.  One pass can feed several cubes of the same
// geometry (the routers of Section III.C), each from its own packet segments.
//
// Why: Alg. 1 sets |RA|+|VA| single bits per packet.  Done as reductions
// straight into an L2-resident cube, heavy sources (a Zipf head of
// millions of packets) aim all their bits at the same few columns -- a few
// L2 lines -- and the reductions on one line serialise.  Here each bit set
// becomes a 4-byte code routed to the 128 KiB cube tile that holds its
// word; each tile is then assembled in shared memory, where a hot column's
// 32 words sit in 32 different banks, and ORed into its cube with one
// coalesced reduction per non-zero word.
//
// Tiles: router cube r owns tiles [r*T, (r+1)*T) with T = ceil(cube words /
// 2^15); a column never straddles a tile (columns start at multiples of W,
// tiles are multiples of W words), so a bit's tile depends on the source
// address only.
//
//   1. k_bin_count   : histogram of codes per tile (shared-memory counters)
//   2. k_bin_scan    : exclusive scans -> code offsets per tile, and apply
//                      items (a tile's codes cut into chunks of `ch`)
//   3. k_bin_scatter : each block routes the codes of one chunk of packets
//                      (kept in registers): counts them per tile, reserves
//                      one run per tile in the code buffer, stages them
//                      grouped by tile in shared memory and writes the runs
//                      out coalesced
//   4. k_bin_apply   : per item: zero a shared tile, set the item's bits
//                      with shared-memory atomics, OR the non-zero words
//                      into the tile's cube
// Traffic per packet: 8 B read twice (count, scatter), 4 B per code
// written and read once.
#include "cbaa_internal.cuh"
#include "update_binned.h"

namespace cbaa {

namespace {

constexpr uint32_t kTileBits = kBinTileBits;          // 2^15 words = 128 KiB per tile
constexpr uint32_t kTileWords = 1u << kTileBits;
constexpr uint32_t kCountThreads = 256;
constexpr uint32_t kApplyThreads = 1024;

__device__ __forceinline__ uint2 ld_pair(const uint32_t *p) {
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint4 ld_stream_v4(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void apply_code(uint32_t *tile, uint32_t v) {
    tile_set_bit(&tile[(v >> 5) & (kTileWords - 1u)], 1u << (v & 31u));
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.global.or.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Segment of flattened packet p (segments are few; a linear walk).
__device__ __forceinline__ uint32_t seg_of(const BinSegs &S, uint64_t p) {
    uint32_t s = 0;
    while (s + 1 < S.k && p >= S.start[s + 1]) ++s;
    return s;
}

// Word in the tile space (router r's words start at r * seg_words) of each
// of the pair's |RA|+|VA| bits (Alg. 1), and the bit.
template <int NRA, int NVA>
__device__ __forceinline__ uint32_t pair_targets(const Geo &G, uint32_t seg_base, uint32_t iip, uint32_t oip,
                                                 uint32_t (&w)[NRA ? NRA + NVA : CBAA_MAX_ARRAYS], uint32_t &bit) {
    const uint32_t nra = NRA ? NRA : G.n_ra;
    const uint32_t nva = NRA ? NVA : G.n_va;
    const uint32_t row = row_of(G, oip);
    const uint32_t m = mangle(G, iip);
    const uint32_t cs = m & G.smask;
    const uint32_t lp = m >> G.r;
    const uint32_t base = seg_base + cs * G.cs_words + (row >> 5);
#pragma unroll
    for (uint32_t i = 0; i < (NRA ? NRA : CBAA_MAX_RA); ++i) {
        if (NRA == 0 && i >= nra) break;
        w[i] = base + G.arr_base[i] + ra_col(G, i, lp) * G.W;
    }
#pragma unroll
    for (uint32_t j = 0; j < (NRA ? NVA : CBAA_MAX_ARRAYS); ++j) {
        if (NRA == 0 && j >= nva) break;
        w[nra + j] = base + G.arr_base[nra + j] + va_col(G, j, lp) * G.W;
    }
    bit = row & 31u;
    return nra + nva;
}

// Tile of each of the pair's bits (source address only, see above).
template <int NRA, int NVA>
__device__ __forceinline__ uint32_t source_tiles(const Geo &G, uint32_t seg_base, uint32_t iip,
                                                 uint32_t (&t)[NRA ? NRA + NVA : CBAA_MAX_ARRAYS]) {
    const uint32_t nra = NRA ? NRA : G.n_ra;
    const uint32_t nva = NRA ? NVA : G.n_va;
    const uint32_t m = mangle(G, iip);
    const uint32_t cs = m & G.smask;
    const uint32_t lp = m >> G.r;
    const uint32_t base = seg_base + cs * G.cs_words;
#pragma unroll
    for (uint32_t i = 0; i < (NRA ? NRA : CBAA_MAX_RA); ++i) {
        if (NRA == 0 && i >= nra) break;
        t[i] = (base + G.arr_base[i] + ra_col(G, i, lp) * G.W) >> kTileBits;
    }
#pragma unroll
    for (uint32_t j = 0; j < (NRA ? NVA : CBAA_MAX_ARRAYS); ++j) {
        if (NRA == 0 && j >= nva) break;
        t[nra + j] = (base + G.arr_base[nra + j] + va_col(G, j, lp) * G.W) >> kTileBits;
    }
    return nra + nva;
}

template <int NRA, int NVA>
__global__ void __launch_bounds__(kCountThreads) k_bin_count(const Geo G, const BinSegs S, uint64_t n, uint32_t nb,
                                                             uint32_t *__restrict__ counts) {
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // four packets in flight per thread
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < n; p0 += 4 * stride) {
        uint32_t iip[4], seg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t p = p0 + u * stride;
            seg[u] = 0xFFFFFFFFu;
            if (p < n) {
                seg[u] = seg_of(S, p);
                const uint32_t *pp = S.pairs[seg[u]] + 2 * (p - S.start[seg[u]]);
                if (G.n_inner) {                          // raw {src, dst} against NI (Section III)
                    uint2 v = ld_pair(pp);
                    if (orient(G, v.x, v.y)) iip[u] = v.x;
                    else seg[u] = 0xFFFFFFFFu;
                } else {
                    iip[u] = ld_stream_u32(pp);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (seg[u] == 0xFFFFFFFFu) continue;
            uint32_t t[NRA ? NRA + NVA : CBAA_MAX_ARRAYS];
            const uint32_t A = source_tiles<NRA, NVA>(G, S.router[seg[u]] * S.seg_words, iip[u], t);
#pragma unroll
            for (uint32_t a = 0; a < (NRA ? NRA + NVA : CBAA_MAX_ARRAYS); ++a) {
                if (NRA == 0 && a >= A) break;
                atomicAdd(&hist[t[a]], 1u);
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// One block: bin_scan_block.
__global__ void __launch_bounds__(1024) k_bin_scan(uint32_t *__restrict__ counts, uint32_t nb, uint32_t ch,
                                                   uint32_t *__restrict__ offsets, uint32_t *__restrict__ cursors,
                                                   uint32_t *__restrict__ item_start, uint32_t *__restrict__ nchunk,
                                                   uint32_t samp) {
    __shared__ uint32_t tmp[32];
    bin_scan_block(counts, nb, ch, offsets, cursors, item_start, nchunk, samp, tmp);
}

// THREADS x PPT packets per block.
template <int NRA, int NVA, int THREADS, int PPT>
__global__ void __launch_bounds__(THREADS) k_bin_scatter(const Geo G, const BinSegs S, uint64_t n, uint32_t nb,
                                                         uint32_t *__restrict__ cursors,
                                                         uint32_t *__restrict__ codes) {
    extern __shared__ uint32_t sm[];
    uint32_t *hist = sm;             // per-tile count
    uint32_t *fill = sm + nb;        // next free slot of each tile's run in `staged`
    uint32_t *delta = sm + 2 * nb;   // run start in `codes` minus run start in `staged`
    uint32_t *staged = sm + 3 * nb;  // codes of this block, grouped by tile
    __shared__ uint32_t tmp[32];
    constexpr uint32_t AM = NRA ? NRA + NVA : CBAA_MAX_ARRAYS;
    constexpr uint32_t P = THREADS * PPT;
    const uint64_t p0 = (uint64_t)blockIdx.x * P;
    const uint32_t np = (uint32_t)((n - p0) < P ? (n - p0) : P);

    for (uint32_t i = threadIdx.x; i < nb; i += THREADS) hist[i] = 0;
    __syncthreads();
    // codes packed as tile << (kTileBits + 5) | word-in-tile << 5 | bit, kept in registers
    uint32_t code[PPT][AM];
    bool ok[PPT];
    uint32_t A = G.A;
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {
        const uint32_t p = threadIdx.x + k * THREADS;
        ok[k] = false;
        if (p < np) {
            const uint64_t gp = p0 + p;
            const uint32_t s = seg_of(S, gp);
            uint2 v = ld_pair(S.pairs[s] + 2 * (gp - S.start[s]));
            if (G.n_inner && !orient(G, v.x, v.y)) continue;   // raw {src, dst} against NI (Section III)
            ok[k] = true;
            uint32_t w[AM], bit;
            A = pair_targets<NRA, NVA>(G, S.router[s] * S.seg_words, v.x, v.y, w, bit);
#pragma unroll
            for (uint32_t a = 0; a < AM; ++a) {
                if (NRA == 0 && a >= A) break;
                const uint32_t b = w[a] >> kTileBits;
                code[k][a] = (b << (kTileBits + 5)) | ((w[a] & (kTileWords - 1u)) << 5) | bit;
                atomicAdd(&hist[b], 1u);
            }
        }
    }
    __syncthreads();
    const uint32_t total = block_exclusive_scan(hist, fill, nb, tmp);
    for (uint32_t b = threadIdx.x; b < nb; b += THREADS) {
        const uint32_t c = hist[b];
        if (c) delta[b] = atomicAdd(&cursors[b], c) - fill[b];
    }
    __syncthreads();
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {
        if (ok[k]) {
#pragma unroll
            for (uint32_t a = 0; a < AM; ++a) {
                if (NRA == 0 && a >= A) break;
                const uint32_t v = code[k][a];
                staged[atomicAdd(&fill[v >> (kTileBits + 5)], 1u)] = v;
            }
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < total; t += THREADS) {
        const uint32_t v = staged[t];
        codes[delta[v >> (kTileBits + 5)] + t] = v;
    }
}

__global__ void __launch_bounds__(kApplyThreads) k_bin_apply(const BinSegs S, uint64_t cube_words,
                                                             const uint32_t *__restrict__ codes,
                                                             const uint32_t *__restrict__ offsets,
                                                             const uint32_t *__restrict__ item_start, uint32_t nb,
                                                             uint32_t ch) {
    extern __shared__ uint32_t tile[];
    const uint32_t items = item_start[nb];
    for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
        uint32_t lo = 0, hi = nb;                        // last b with item_start[b] <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (item_start[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t b = lo;
        const uint32_t c0 = offsets[b] + (item - item_start[b]) * ch;
        const uint32_t cend = offsets[b + 1];
        const uint32_t c1 = c0 + ch < cend ? c0 + ch : cend;
        uint4 *t4 = reinterpret_cast<uint4 *>(tile);
        for (uint32_t i = threadIdx.x; i < kTileWords / 4; i += blockDim.x) t4[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
        // scalar head up to a 16-byte boundary, vector body, scalar tail
        const uint32_t up4 = (c0 + 3u) & ~3u;
        const uint32_t a0 = up4 < c1 ? up4 : c1;
        const uint32_t a1 = a0 + ((c1 - a0) & ~3u);
        for (uint32_t c = c0 + threadIdx.x; c < a0; c += blockDim.x) apply_code(tile, ld_stream_u32(codes + c));
        const uint4 *q = reinterpret_cast<const uint4 *>(codes + a0);
        const uint32_t nq = (a1 - a0) / 4;
        uint32_t i = threadIdx.x;
        for (; i + blockDim.x < nq; i += 2 * blockDim.x) {
            const uint4 x = ld_stream_v4(q + i), y = ld_stream_v4(q + i + blockDim.x);
            apply_code(tile, x.x); apply_code(tile, x.y); apply_code(tile, x.z); apply_code(tile, x.w);
            apply_code(tile, y.x); apply_code(tile, y.y); apply_code(tile, y.z); apply_code(tile, y.w);
        }
        for (; i < nq; i += blockDim.x) {
            const uint4 x = ld_stream_v4(q + i);
            apply_code(tile, x.x); apply_code(tile, x.y); apply_code(tile, x.z); apply_code(tile, x.w);
        }
        for (uint32_t c = a1 + threadIdx.x; c < c1; c += blockDim.x) apply_code(tile, ld_stream_u32(codes + c));
        __syncthreads();
        const uint32_t r = b / S.tiles_per_seg;
        const uint64_t base = (uint64_t)(b - r * S.tiles_per_seg) << kTileBits;   // inside cube r
        const uint32_t lim = (uint32_t)((cube_words - base) < kTileWords ? (cube_words - base) : kTileWords);
        uint32_t *dst = S.cube[r] + base;
        for (uint32_t w = threadIdx.x; w < lim; w += blockDim.x) {
            const uint32_t v = tile[w];
            if (v) {
                red_or(dst + w, v);
                if (S.merge) red_or(S.merge + base + w, v);     // the global server's OR, in the same pass
            }
        }
        __syncthreads();
    }
}

template <int NRA, int NVA, int THREADS, int PPT>
cudaError_t launch_scatter(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W, cudaStream_t s) {
    const size_t smem = sizeof(uint32_t) * (3ull * nb + (size_t)G.A * THREADS * PPT);
    cudaError_t e = allow_smem(k_bin_scatter<NRA, NVA, THREADS, PPT>, smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((m + THREADS * PPT - 1) / (THREADS * PPT));
    k_bin_scatter<NRA, NVA, THREADS, PPT><<<blocks, THREADS, smem, s>>>(G, S, m, nb, W.cursors, W.codes);
    return cudaGetLastError();
}

template <int NRA, int NVA>
cudaError_t launch_scatter_shape(const Geo &G, const BinSegs &S, uint64_t m, uint32_t nb, const BinWs &W,
                                 uint32_t shape, cudaStream_t s) {
    switch (shape) {
        case 1: return launch_scatter<NRA, NVA, 512, 4>(G, S, m, nb, W, s);
        case 2: return launch_scatter<NRA, NVA, 1024, 4>(G, S, m, nb, W, s);
        case 3: return launch_scatter<NRA, NVA, 256, 8>(G, S, m, nb, W, s);
        case 4: return launch_scatter<NRA, NVA, 256, 4>(G, S, m, nb, W, s);
        case 5: return launch_scatter<NRA, NVA, 1024, 8>(G, S, m, nb, W, s);
        case 6: return launch_scatter<NRA, NVA, 512, 16>(G, S, m, nb, W, s);
        case 7: return launch_scatter<NRA, NVA, 256, 16>(G, S, m, nb, W, s);
        case 8: return launch_scatter<NRA, NVA, 512, 8>(G, S, m, nb, W, s);   // 1024 x 16 exceeds shared memory here
        default: return launch_scatter<NRA, NVA, 512, 8>(G, S, m, nb, W, s);
    }
}

template <int NRA, int NVA>
cudaError_t launch_binned_t(const Geo &G, const BinSegs &S0, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                            cudaStream_t s) {
    const uint32_t nb = S0.n_routers * S0.tiles_per_seg;
    const uint32_t A = G.A;
    const int sms = num_sms();
    const size_t apply_smem = sizeof(uint32_t) * kTileWords;
    cudaError_t e;
    if ((e = allow_smem(k_bin_apply, apply_smem)) != cudaSuccess) return e;
    if ((e = allow_smem(k_bin_count<NRA, NVA>, sizeof(uint32_t) * nb)) != cudaSuccess) return e;
    const uint32_t count_bps = T.count_blocks_per_sm ? T.count_blocks_per_sm : 8;
    const uint32_t apply_ips = T.apply_items_per_sm ? T.apply_items_per_sm : 8;
    for (uint64_t done = 0; done < n;) {
        const uint64_t m = (n - done) < W.max_pairs ? (n - done) : W.max_pairs;
        // the segments clipped to flattened packets [done, done + m), re-based at 0
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
        if ((e = cudaMemsetAsync(W.counts, 0, sizeof(uint32_t) * nb, s)) != cudaSuccess) return e;
        const uint64_t want = (m + kCountThreads - 1) / kCountThreads;
        const uint64_t cap = (uint64_t)sms * count_bps;
        const unsigned cblocks = (unsigned)(want < cap ? want : cap);
        k_bin_count<NRA, NVA><<<cblocks, kCountThreads, sizeof(uint32_t) * nb, s>>>(G, S, m, nb, W.counts);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint64_t ch = ((uint64_t)A * m + (uint64_t)sms * apply_ips - 1) / ((uint64_t)sms * apply_ips);
        if (ch < (1u << 14)) ch = 1u << 14;
        k_bin_scan<<<1, 1024, 0, s>>>(W.counts, nb, (uint32_t)ch, W.offsets, W.cursors, W.item_start, W.nchunk, 1u);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_scatter_shape<NRA, NVA>(G, S, m, nb, W, T.scatter_shape, s)) != cudaSuccess) return e;
        k_bin_apply<<<(unsigned)sms, kApplyThreads, apply_smem, s>>>(S, G.cube_words, W.codes, W.offsets,
                                                                     W.item_start, nb, (uint32_t)ch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        done += m;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_bin_scan(uint32_t *counts, uint32_t nb, uint32_t ch, const BinWs &W, cudaStream_t s,
                            uint32_t samp) {
    k_bin_scan<<<1, 1024, 0, s>>>(counts, nb, ch, W.offsets, W.cursors, W.item_start, W.nchunk, samp);
    return cudaGetLastError();
}

cudaError_t launch_update_segments(const Geo &G, const BinSegs &S, uint64_t n, const BinWs &W, const cbaa_tuning &T,
                                   cudaStream_t s, bool assign) {
    if (n == 0) return cudaSuccess;
    if (S.k == 1 && !S.merge && heavy_enabled(G, S.n_routers, n, T))
        return launch_update_heavy(G, S.cube[S.router[0]], S.pairs[0], n, W, T, s, assign);
    if (assign && S.n_routers == 1) {
        const cudaError_t e = cudaMemsetAsync(S.cube[0], 0, G.cube_words * 4u, s);
        if (e != cudaSuccess) return e;
    }
    if (T.tile_kind != 1 && rowtile_ok(G, S.n_routers)) return launch_update_rowtile(G, S, n, W, T, s);
    if (G.n_ra == 3 && G.n_va == 1) return launch_binned_t<3, 1>(G, S, n, W, T, s);
    return launch_binned_t<0, 0>(G, S, n, W, T, s);
}

}  // namespace cbaa
