// Alg. 1 by partition: the same cube as the direct update, built without
// L2 atomics on the cube.
//
// Why: Alg. 1 sets |RA|+|VA| single bits per packet.  Done as reductions
// straight into an L2-resident cube, heavy sources (a Zipf head of
// millions of packets) aim all their bits at the same few columns -- a few
// L2 lines -- and the reductions on one line serialise.  Here each bit set
// becomes a 4-byte code routed to the 128 KiB cube tile that holds its
// word; each tile is then assembled in shared memory, where a hot column's
// 32 words sit in 32 different banks, and ORed into the cube with one
// coalesced reduction per non-zero word.
//
//   1. k_bin_count   : histogram of codes per tile (shared-memory counters;
//                      the tile depends on the source address only)
//   2. k_bin_scan    : exclusive scans -> code offsets per tile, and apply
//                      items (a tile's codes cut into chunks of `ch`)
//   3. k_bin_scatter : each block routes the codes of 4096 packets (kept in
//                      registers): counts them per tile, reserves one run per
//                      tile in the code buffer, stages them grouped by tile
//                      in shared memory and writes the runs out coalesced
//   4. k_bin_apply   : per item: zero a shared tile, set the item's bits
//                      with shared-memory atomics, OR the non-zero words
//                      into the cube
// Traffic per packet: 8 B read twice (count, scatter), 4 B per code
// written and read once.
#include "cbaa_internal.cuh"
#include "update_binned.h"

namespace cbaa {

namespace {

constexpr uint32_t kTileBits = kBinTileBits;          // 2^15 words = 128 KiB per tile
constexpr uint32_t kTileWords = 1u << kTileBits;
constexpr uint32_t kScatterThreads = 512;
constexpr uint32_t kScatterPairs = 4096;               // packets per scatter block
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
    atomicOr(&tile[(v >> 5) & (kTileWords - 1u)], 1u << (v & 31u));
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.global.or.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Word index of each of the pair's |RA|+|VA| bits (Alg. 1) and the bit.
template <int NRA, int NVA>
__device__ __forceinline__ uint32_t pair_targets(const Geo &G, uint32_t iip, uint32_t oip,
                                                 uint32_t (&w)[NRA ? NRA + NVA : CBAA_MAX_ARRAYS], uint32_t &bit) {
    const uint32_t nra = NRA ? NRA : G.n_ra;
    const uint32_t nva = NRA ? NVA : G.n_va;
    const uint32_t row = row_of(G, oip);
    const uint32_t m = mangle(G, iip);
    const uint32_t cs = m & G.smask;
    const uint32_t lp = m >> G.r;
    const uint32_t base = cs * G.cs_words + (row >> 5);
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

// Tile of each of the pair's bits.  A column never straddles a tile (columns
// start at multiples of W and a tile is a multiple of W words), so the tile
// depends on the source address only and the row hash is not needed here.
template <int NRA, int NVA>
__device__ __forceinline__ uint32_t source_tiles(const Geo &G, uint32_t iip,
                                                 uint32_t (&t)[NRA ? NRA + NVA : CBAA_MAX_ARRAYS]) {
    const uint32_t nra = NRA ? NRA : G.n_ra;
    const uint32_t nva = NRA ? NVA : G.n_va;
    const uint32_t m = mangle(G, iip);
    const uint32_t cs = m & G.smask;
    const uint32_t lp = m >> G.r;
    const uint32_t base = cs * G.cs_words;
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

// Exclusive scan of in[0..n) into out[0..n) by one block (blockDim a
// multiple of 32, at most 1024); returns the total.  `tmp` holds 32 words.
__device__ uint32_t block_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *tmp) {
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

template <int NRA, int NVA>
__global__ void __launch_bounds__(kCountThreads) k_bin_count(const Geo G, const uint32_t *__restrict__ pairs,
                                                             uint64_t n, uint32_t nb, uint32_t *__restrict__ counts) {
    extern __shared__ uint32_t hist[];
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const uint32_t iip = ld_stream_u32(pairs + 2 * p);
        uint32_t t[NRA ? NRA + NVA : CBAA_MAX_ARRAYS];
        const uint32_t A = source_tiles<NRA, NVA>(G, iip, t);
#pragma unroll
        for (uint32_t a = 0; a < (NRA ? NRA + NVA : CBAA_MAX_ARRAYS); ++a) {
            if (NRA == 0 && a >= A) break;
            atomicAdd(&hist[t[a]], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x)
        if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// One block: offsets = exclusive scan of counts, cursors = offsets,
// items = exclusive scan of ceil(counts / ch) (item_start[nb] = total).
__global__ void __launch_bounds__(1024) k_bin_scan(const uint32_t *__restrict__ counts, uint32_t nb, uint32_t ch,
                                                   uint32_t *__restrict__ offsets, uint32_t *__restrict__ cursors,
                                                   uint32_t *__restrict__ item_start, uint32_t *__restrict__ nchunk) {
    __shared__ uint32_t tmp[32];
    const uint32_t total = block_exclusive_scan(counts, offsets, nb, tmp);
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        cursors[i] = offsets[i];
        nchunk[i] = (counts[i] + ch - 1) / ch;
    }
    if (threadIdx.x == 0) offsets[nb] = total;
    __syncthreads();
    const uint32_t items = block_exclusive_scan(nchunk, item_start, nb, tmp);
    if (threadIdx.x == 0) item_start[nb] = items;
}

template <int NRA, int NVA>
__global__ void __launch_bounds__(kScatterThreads) k_bin_scatter(const Geo G, const uint32_t *__restrict__ pairs,
                                                                 uint64_t n, uint32_t nb,
                                                                 uint32_t *__restrict__ cursors,
                                                                 uint32_t *__restrict__ codes) {
    extern __shared__ uint32_t sm[];
    uint32_t *hist = sm;             // per-tile count, then fill position
    uint32_t *lstart = sm + nb;      // start of each tile's run in `staged`
    uint32_t *gbase = sm + 2 * nb;   // start of each tile's run in `codes`
    uint32_t *staged = sm + 3 * nb;  // codes of this block, grouped by tile
    __shared__ uint32_t tmp[32];
    constexpr uint32_t AM = NRA ? NRA + NVA : CBAA_MAX_ARRAYS;
    constexpr uint32_t PPT = kScatterPairs / kScatterThreads;     // packets per thread
    const uint64_t p0 = (uint64_t)blockIdx.x * kScatterPairs;
    const uint32_t np = (uint32_t)((n - p0) < kScatterPairs ? (n - p0) : kScatterPairs);

    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // codes packed as tile << (kTileBits + 5) | word-in-tile << 5 | bit, kept in registers
    uint32_t code[PPT][AM];
    uint32_t A = G.A;
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {
        const uint32_t p = threadIdx.x + k * kScatterThreads;
        if (p < np) {
            const uint2 v = ld_pair(pairs + 2 * (p0 + p));
            uint32_t w[AM], bit;
            A = pair_targets<NRA, NVA>(G, v.x, v.y, w, bit);
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
    const uint32_t total = block_exclusive_scan(hist, lstart, nb, tmp);
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const uint32_t c = hist[b];
        if (c) gbase[b] = atomicAdd(&cursors[b], c);
        hist[b] = 0;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t k = 0; k < PPT; ++k) {
        const uint32_t p = threadIdx.x + k * kScatterThreads;
        if (p < np) {
#pragma unroll
            for (uint32_t a = 0; a < AM; ++a) {
                if (NRA == 0 && a >= A) break;
                const uint32_t v = code[k][a];
                const uint32_t b = v >> (kTileBits + 5);
                staged[lstart[b] + atomicAdd(&hist[b], 1u)] = v;
            }
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < total; t += blockDim.x) {
        const uint32_t v = staged[t];
        const uint32_t b = v >> (kTileBits + 5);
        codes[gbase[b] + (t - lstart[b])] = v;
    }
}

__global__ void __launch_bounds__(kApplyThreads) k_bin_apply(uint32_t *__restrict__ cube, uint64_t cube_words,
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
        for (uint32_t c = c0 + threadIdx.x; c < a0; c += blockDim.x) {
            const uint32_t v = ld_stream_u32(codes + c);
            atomicOr(&tile[(v >> 5) & (kTileWords - 1u)], 1u << (v & 31u));
        }
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
        const uint64_t base = (uint64_t)b << kTileBits;
        const uint32_t lim = (uint32_t)((cube_words - base) < kTileWords ? (cube_words - base) : kTileWords);
        for (uint32_t i = threadIdx.x; i < lim; i += blockDim.x) {
            const uint32_t v = tile[i];
            if (v) red_or(cube + base + i, v);
        }
        __syncthreads();
    }
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NRA, int NVA>
cudaError_t launch_binned_t(const Geo &G, uint32_t *cube, const uint32_t *pairs, size_t n, const BinWs &W,
                            cudaStream_t s) {
    const uint32_t nb = bin_count(G);
    const uint32_t A = G.A;
    const int sms = num_sms();
    const size_t scatter_smem = sizeof(uint32_t) * (3ull * nb + (size_t)A * kScatterPairs);
    const size_t apply_smem = sizeof(uint32_t) * kTileWords;
    cudaError_t e;
    if ((e = allow_smem(k_bin_scatter<NRA, NVA>, scatter_smem)) != cudaSuccess) return e;
    if ((e = allow_smem(k_bin_apply, apply_smem)) != cudaSuccess) return e;
    if ((e = allow_smem(k_bin_count<NRA, NVA>, sizeof(uint32_t) * nb)) != cudaSuccess) return e;
    for (size_t done = 0; done < n;) {
        const size_t m = (n - done) < W.max_pairs ? (n - done) : W.max_pairs;
        const uint32_t *pp = pairs + 2 * done;
        if ((e = cudaMemsetAsync(W.counts, 0, sizeof(uint32_t) * nb, s)) != cudaSuccess) return e;
        const uint64_t want = (m + kCountThreads - 1) / kCountThreads;
        const unsigned cblocks = (unsigned)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
        k_bin_count<NRA, NVA><<<cblocks, kCountThreads, sizeof(uint32_t) * nb, s>>>(G, pp, m, nb, W.counts);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // apply items: about 8 per SM, at least 16 Ki codes each
        uint64_t ch = ((uint64_t)A * m + (uint64_t)sms * 8 - 1) / ((uint64_t)sms * 8);
        if (ch < (1u << 14)) ch = 1u << 14;
        k_bin_scan<<<1, 1024, 0, s>>>(W.counts, nb, (uint32_t)ch, W.offsets, W.cursors, W.item_start, W.nchunk);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const unsigned sblocks = (unsigned)((m + kScatterPairs - 1) / kScatterPairs);
        k_bin_scatter<NRA, NVA><<<sblocks, kScatterThreads, scatter_smem, s>>>(G, pp, m, nb, W.cursors, W.codes);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_bin_apply<<<(unsigned)sms, kApplyThreads, apply_smem, s>>>(cube, G.cube_words, W.codes, W.offsets,
                                                                     W.item_start, nb, (uint32_t)ch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        done += m;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_update_binned(const Geo &G, uint32_t *cube, const uint32_t *pairs, size_t n, const BinWs &W,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (G.n_ra == 3 && G.n_va == 1) return launch_binned_t<3, 1>(G, cube, pairs, n, W, s);
    return launch_binned_t<0, 0>(G, cube, pairs, n, W, s);
}

}  // namespace cbaa
