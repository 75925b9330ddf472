// Alg. 1 with the heavy sources split off: a pre-pass in front of the
// row-tile update for single-cube passes.
//
// All |RA|+|VA| bits that a packet sets share its sketch and its row, and
// its columns depend on its source alone (Alg. 1: the CS and the column
// indices come from the mangled inner address, the row from H_bv of the
// outer one).  So the bits that one source sets over a window are its set
// of rows, the same in each of its columns: a row bitmap of W words.  On
// core-network traffic a few sources carry most packets (super hosts and
// the head of a Zipf law), so:
//
//   1. k_heavy_sample : one tile of 1024 packets in 256 is counted by the top
//                       15 bits of the source key (with a key seen in each
//                       slot)
//   2. k_heavy_hist   : the sample counts' histogram; from it every split
//                       block picks the most counted slots, up to K of them,
//                       as the heavy sources (the same ones in every block)
//                       and builds a lookup table from key to heavy index
//                       (top 14 bits -> low 18 bits as a tag and the index)
//   3. k_heavy_split  : every packet: a heavy source's row bit is set in
//                       its bitmap in shared memory (a bit already set is
//                       only read); any other packet is written out as
//                       {key, row} (the key: the bijection below of iip).  Each block ORs its bitmaps into the
//                       global ones with one bulk reduction.
//   4. the row-tile pass over the residual entries (update_rowtile.cu), whose
//      counting kernel also ORs each heavy bitmap into the source's columns
//      (extra blocks: a launch fewer)
//
// The source key is a multiplicative bijection of the inner address, not its
// mangled form: one multiply instead of the mangle's five steps, and the
// mangle is computed only for the residual packets (by the routing kernel)
// and once per heavy source (by the expansion).  The row is computed for
// every packet, once.  Which sources are heavy only
// decides the path a packet takes, never the cube: every packet's bits are
// set by one of the two paths.
#include <cstring>

#include "cbaa_internal.cuh"
#include "update_binned.h"

namespace cbaa {

namespace {

constexpr uint32_t kSampleThreads = 1024;
constexpr uint32_t kSampleTile = 1024;                 // packets of a sample tile, one per thread
constexpr uint32_t kHeavySampleEvery = 256;            // one sample tile in 256
constexpr uint32_t kHeavyMinCount = 4;                 // sampled packets a heavy source needs at least
constexpr uint64_t kHeavyMinPackets = 4ull << 20;      // default: passes of at least this many packets
constexpr uint32_t kTabWords = 1u << kHeavyTabBits;
constexpr uint32_t kCountSlots = 1u << kHeavyCountBits;
constexpr uint32_t kTagMask = (1u << kHeavyTagBits) - 1u;

__device__ __forceinline__ uint4 ld_quad_nc(const uint32_t *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ uint2 ld_pair_nc(const uint32_t *p) {
    uint2 v;
    asm volatile("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}


// H_bv(oip) with its seed folded in: the finaliser's first step applied to
// oip ^ s is (oip ^ (oip >> 16)) ^ (s ^ (s >> 16)), so with seed_fold =
// s ^ (s >> 16) computed once the seed costs no instruction of its own.
// Equal to row_of(G, oip).
__device__ __forceinline__ uint32_t row_of_folded(const Geo &G, uint32_t oip, uint32_t seed_fold) {
    return mix32_mid(oip ^ (oip >> 16) ^ seed_fold) >> (32u - G.log2_g);
}


// Counts of the sample by slot, first in shared memory (one table per
// block, 2^15 counters), then added to the global table: a heavy source's
// slot gets one global atomic per block instead of one per sampled packet.
// Sampled tile j (1024 consecutive packets, one per thread) starts at packet
// j * 1024 * 128.
template <bool ORIENT>
__global__ void __launch_bounds__(kSampleThreads, 1) k_heavy_sample(const Geo G, const uint32_t *__restrict__ pairs,
                                                                    uint64_t n, uint32_t *__restrict__ count,
                                                                    uint32_t *__restrict__ key) {
    extern __shared__ __align__(16) uint32_t cnt[];
    for (uint32_t i = threadIdx.x; i < kCountSlots / 4; i += kSampleThreads)
        reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const uint64_t tiles = (n + (uint64_t)kSampleTile * kHeavySampleEvery - 1) / ((uint64_t)kSampleTile * kHeavySampleEvery);
    // four sampled tiles per step (tiles j + u * gridDim.x), their loads in flight together
    for (uint64_t j = blockIdx.x; j < tiles; j += 4ull * gridDim.x) {
        uint2 v[4];
        bool have[4];
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint64_t p = (j + (uint64_t)u * gridDim.x) * kSampleTile * kHeavySampleEvery + threadIdx.x;
            have[u] = p < n;
            if (have[u]) v[u] = ld_pair_nc(pairs + 2 * p);
        }
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            if (!have[u]) continue;
            if (ORIENT && !orient(G, v[u].x, v[u].y)) continue;
            const uint32_t m = heavy_key(v[u].x);
            const uint32_t slot = m >> (32 - kHeavyCountBits);
            // the slot keeps a key seen at every 8th count of a block: a slot with
            // one heavy source keeps that source's key with high probability
            if ((atomicAdd(&cnt[slot], 1u) & 7u) == 0u) key[slot] = m;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kCountSlots; i += kSampleThreads) {
        const uint32_t c = cnt[i];
        if (c) atomicAdd(&count[i], c);
    }
}

// Quarter-octave bin of a sample count: 4 floor(log2 c) + the two bits below
// the leading one, or kHeavyHistBins below kHeavyMinCount (4, so e >= 2).
__device__ __forceinline__ uint32_t count_bin(uint32_t c) {
    if (c < kHeavyMinCount) return kHeavyHistBins;
    const uint32_t e = 31 - __clz(c);
    return 4 * e + ((c >> (e - 2)) & 3u);
}
// Smallest count of bin b.
__device__ __forceinline__ uint32_t bin_floor(uint32_t b) { return (4u + (b & 3u)) << ((b >> 2) - 2); }

// Histogram of the sample counts by quarter octave (one slot per thread).
// Also zeroes the residual pass's row-tile counts (nzero words).
__global__ void __launch_bounds__(1024) k_heavy_hist(const uint32_t *__restrict__ count, uint32_t *__restrict__ hist,
                                                     uint32_t *__restrict__ zero, uint32_t nzero) {
    __shared__ uint32_t h[kHeavyHistBins];
    if (threadIdx.x < kHeavyHistBins) h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t b = i < kCountSlots ? count_bin(__ldcg(count + i)) : kHeavyHistBins;
    if (b < kHeavyHistBins) atomicAdd(&h[b], 1u);
    for (uint32_t t = i; t < nzero; t += gridDim.x * blockDim.x) zero[t] = 0u;
    __syncthreads();
    if (threadIdx.x < kHeavyHistBins && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// The heavy sources, chosen again by every split block from the sample
// (1024 threads, 32 slots each kept in registers), so that no launch of its
// own stands between the histogram and the split: thr is the smallest bin
// floor whose bins and the ones above hold at most kmax slots; every slot
// counted at least thr times (and kHeavyMinCount) takes an index in
// [0, acc), in slot order, then slots of the bin below thr take acc, acc + 1,
// ... while room is left.  The indices come from block-wide prefix sums in
// slot order, so every block assigns the same index to the same source, and
// block 0 lists the keys for the expansion (ctr[0], ctr[1]: the upper and
// lower slots taken).  Each block enters the keys into its own lookup image
// in shared memory; two keys whose entries collide: the one that loses the
// CAS stays on the row-tile path in that block (which sources are heavy
// only decides the path of a packet).  Also clears the bitmaps.
template <uint32_t THREADS>
__device__ __forceinline__ void split_select(const uint32_t *__restrict__ count, const uint32_t *__restrict__ key,
                                             const uint32_t *__restrict__ hist_g, uint32_t kmax, uint32_t *tab,
                                             uint32_t *bm, uint32_t kwords, uint32_t *__restrict__ list_g,
                                             uint32_t *__restrict__ ctr_g) {
    static_assert(THREADS * 32 == kCountSlots, "32 sample slots per thread");
    __shared__ uint32_t hist[kHeavyHistBins], s_thr, s_lo, s_acc, s_wu[32], s_wl[32];
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    uint32_t c[32];
#pragma unroll
    for (uint32_t j = 0; j < 32; ++j) c[j] = __ldcg(count + t + THREADS * j);
    if (t < kHeavyHistBins) hist[t] = __ldcg(hist_g + t);
    uint4 *t4 = reinterpret_cast<uint4 *>(tab);
    for (uint32_t i = t; i < kTabWords / 4; i += THREADS) t4[i] = make_uint4(kHeavyEmpty, kHeavyEmpty, kHeavyEmpty, kHeavyEmpty);
    uint4 *b4 = reinterpret_cast<uint4 *>(bm);
    for (uint32_t i = t; i < kwords / 4; i += THREADS) b4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (t == 0) {                                     // from shared memory: no global round trip per bin
        uint32_t acc = 0, thr = 0xFFFFFFFFu, lo = 0xFFFFFFFFu;
        for (int b = (int)kHeavyHistBins - 1; b >= 0; --b) {
            const uint32_t hb = hist[b];
            if (acc + hb > kmax) {                     // this bin only partly, while room is left
                lo = hb ? bin_floor(b) : lo;
                break;
            }
            acc += hb;
            if (hb) thr = bin_floor(b);
        }
        s_thr = thr;
        s_lo = lo < thr ? lo : thr;
        s_acc = acc;
    }
    __syncthreads();
    const uint32_t thr = s_thr, lo = s_lo, acc = s_acc;
    uint32_t mu = 0, ml = 0;                          // bit j: slot t + THREADS j taken (upper / lower)
#pragma unroll
    for (uint32_t j = 0; j < 32; ++j) {
        const bool up = c[j] >= thr && c[j] >= kHeavyMinCount;
        const bool low = !up && c[j] >= lo && c[j] >= kHeavyMinCount;
        mu |= (uint32_t)up << j;
        ml |= (uint32_t)low << j;
    }
    // indices in (thread, j) order: an exclusive prefix of the threads' counts
    const uint32_t nu = __popc(mu), nl = __popc(ml);
    uint32_t xu = nu, xl = nl;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t yu = __shfl_up_sync(0xffffffffu, xu, o), yl = __shfl_up_sync(0xffffffffu, xl, o);
        if (lane >= o) {
            xu += yu;
            xl += yl;
        }
    }
    if (lane == 31) {
        s_wu[warp] = xu;
        s_wl[warp] = xl;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t vu = s_wu[lane], vl = s_wl[lane];
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t yu = __shfl_up_sync(0xffffffffu, vu, o), yl = __shfl_up_sync(0xffffffffu, vl, o);
            if (lane >= o) {
                vu += yu;
                vl += yl;
            }
        }
        s_wu[lane] = vu;                               // inclusive over warps
        s_wl[lane] = vl;
    }
    __syncthreads();
    uint32_t hu = (warp ? s_wu[warp - 1] : 0u) + xu - nu;
    uint32_t hl = acc + (warp ? s_wl[warp - 1] : 0u) + xl - nl;
    if (blockIdx.x == 0 && t == 0) {
        ctr_g[0] = s_wu[31];
        ctr_g[1] = s_wl[31];
    }
    uint32_t sel = mu | ml;
    while (sel) {
        const uint32_t j = __ffs(sel) - 1u;
        sel &= sel - 1u;
        const uint32_t h = ((mu >> j) & 1u) ? hu++ : hl++;
        if (h >= kmax) continue;                       // the partial bin only while room is left
        const uint32_t k = __ldcg(key + t + THREADS * j);
        if (blockIdx.x == 0) list_g[h] = k;
        atomicCAS(&tab[k >> kHeavyTagBits], kHeavyEmpty, ((k & kTagMask) << kHeavyTabBits) | h);
    }
    __syncthreads();
}

// Packets of chunk c (32 lanes x 8 packets, 2 per 16-byte load) into q;
// ok: bit k set when slot k of this lane holds a packet.  Slot 2j + h of lane
// l is packet c * 256 + 2 (l + 32 j) + h.
__device__ __forceinline__ uint32_t split_load(const uint32_t *pairs, uint64_t n, uint32_t c, uint32_t lane,
                                               uint32_t full, uint4 (&q)[4]) {
    const uint64_t c0 = (uint64_t)c * 256;
    if (c < full) {                                   // a whole chunk at a 16-byte aligned address
        const uint32_t *p = pairs + 2 * c0 + 4 * lane;
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) q[j] = ld_quad_nc(p + 128 * j);
        return 0xFFu;
    }
    uint32_t ok = 0;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
        const uint64_t p = c0 + 2 * (lane + 32 * j);
        q[j] = make_uint4(0u, 0u, 0u, 0u);
        if (p < n) {
            const uint2 a = ld_pair_nc(pairs + 2 * p);
            q[j].x = a.x;
            q[j].y = a.y;
            ok |= 1u << (2 * j);
        }
        if (p + 1 < n) {
            const uint2 b = ld_pair_nc(pairs + 2 * (p + 1));
            q[j].z = b.x;
            q[j].w = b.y;
            ok |= 2u << (2 * j);
        }
    }
    return ok;
}

// Shared-memory OR of v into the word at shared address sa, issued by every
// lane (v = 0 where nothing is to be set: no predicate, no branch).
__device__ __forceinline__ void red_or_shared(uint32_t sa, uint32_t v) {
    asm volatile("red.shared.or.b32 [%0], %1;" :: "r"(sa), "r"(v) : "memory");
}

// 8-byte store of {x, y} to `ptr` when `p` (predicated).
__device__ __forceinline__ void st_pair_if(uint2 *ptr, uint32_t x, uint32_t y, uint32_t p) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q st.global.v2.u32 [%0], {%1, %2}; }"
                 :: "l"(ptr), "r"(x), "r"(y), "r"(p) : "memory");
}

// The split of NP packets per lane of a warp (slot k of lane `lane`: a[k],
// b[k], present when bit k of ok is set): rows and lookups; bitmap words of
// the heavy ones (some word for the others), read together; sets of the bits
// still clear; the others' entries {key, row} (oriented; key = heavy_key(iip),
// a bijection) written to `region` at places reserved with one shared-memory
// atomic per warp.  In phases, so that the lanes' shared-memory reads are in
// flight together, and without branches: every lane ORs (0 where nothing is
// to be set), the stores are predicated.  bm_s: the shared address of bm;
// kmask: heavy sources in bm - 1 (a power of two less one); lw: log2 of the
// words per bitmap (W); seed_fold: the row hash's seed folded for
// row_of_folded.
// FULL (every lane holds all NP packets, no inner network): the presence
// bits are known to be set and are not tested.
template <uint32_t NP, bool ORIENT, bool FULL>
__device__ __forceinline__ void split_packets(const Geo &G, const uint32_t *tab, const uint32_t *bm, uint32_t bm_s,
                                              uint32_t kmask, uint32_t lw, uint32_t seed_fold, uint32_t (&a)[NP],
                                              uint32_t (&b)[NP], uint32_t ok, uint2 *region, uint32_t *s_cnt,
                                              uint32_t lane) {
    static_assert(!(FULL && ORIENT), "orientation may drop packets");
    if (FULL) ok = (1u << NP) - 1u;
    uint32_t row[NP], e[NP];
#pragma unroll
    for (uint32_t k = 0; k < NP; ++k) {
        if (ORIENT && ((ok >> k) & 1u) && !orient(G, a[k], b[k])) ok &= ~(1u << k);   // raw {src, dst} vs NI
        row[k] = row_of_folded(G, b[k], seed_fold);
        a[k] = heavy_key(a[k]);                       // the key from here on (a bijection of iip)
        e[k] = tab[a[k] >> kHeavyTagBits];
    }
    // e ^ (key << 14) keeps only the index field exactly when the tags agree;
    // the empty marker's index field is all ones
    uint32_t heavy = 0, wi[NP], wv[NP];
#pragma unroll
    for (uint32_t k = 0; k < NP; ++k) {
        const uint32_t d = e[k] ^ (a[k] << kHeavyTabBits);
        const bool hv = (FULL || ((ok >> k) & 1u)) && d < kHeavyIdxMask;
        heavy |= (uint32_t)hv << k;
        // the bitmap word (W = 2^lw words per source); for a packet that is not heavy some
        // source's word (d & kmask < K), read and never set
        wi[k] = ((d & kmask) << lw) + (row[k] >> 5);
        wv[k] = bm[wi[k]];
    }
    // a stale read only costs an atomic that changes nothing: every set is an OR
#pragma unroll
    for (uint32_t k = 0; k < NP; ++k) {
        const uint32_t bit = __funnelshift_l(0u, 1u, row[k]);      // 1 << (row & 31)
        red_or_shared(bm_s + 4u * wi[k], (((heavy >> k) & 1u) && !(wv[k] & bit)) ? bit : 0u);
    }
    const uint32_t keep = ok & ~heavy;
    const uint32_t cnt = __popc(keep);
    uint32_t x = cnt;                                          // lane prefix, one reservation per warp
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t base = 0;
    if (lane == 31 && x) base = atomicAdd(s_cnt, x);
    base = __shfl_sync(0xffffffffu, base, 31) + x - cnt;
    uint32_t at = base;                                        // this lane's entries, in slot order
#pragma unroll
    for (uint32_t k = 0; k < NP; ++k) {
        const uint32_t kk = (keep >> k) & 1u;
        st_pair_if(region + at, a[k], row[k], kk);
        at += kk;
    }
}

// End of a split block: the region's count, then the block's bitmaps into the
// global ones, one bulk OR reduction (async proxy) after the shared-memory
// writes are made visible to it.
__device__ __forceinline__ void split_flush(const uint32_t *bm, uint32_t kwords, uint32_t *bits_g,
                                            const uint32_t *s_cnt, uint32_t *rcount) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();                                  // every warp's reservations and bit sets are done
    if (threadIdx.x == 0) {
        rcount[blockIdx.x] = *s_cnt;
        constexpr uint32_t kChunk = 32u << 10;
        const uint32_t bytes = kwords * 4u;
        const uint32_t s0 = static_cast<uint32_t>(__cvta_generic_to_shared(bm));
        for (uint32_t off = 0; off < bytes; off += kChunk) {
            const uint32_t len = bytes - off < kChunk ? bytes - off : kChunk;
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.or.b32 [%0], [%1], %2;"
                         :: "l"(reinterpret_cast<char *>(bits_g) + off), "r"(s0 + off), "r"(len) : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

// Every warp walks its own chunks of 256 packets (chunk c for c = global
// warp, + all warps, ...), the next chunk's 16-byte loads in flight in
// registers while it works on the current one (two register sets used in
// turn, so nothing is copied between them).  zero (an assigning update's
// first pass): the blocks first zero the cube's zq 16-byte words, which no
// kernel before the split's end reads or writes.  Shared memory: the lookup
// table (built by split_select), then K row bitmaps of W words (kwords
// words).  Residual entries go
// to this block's region (rcap entries from blockIdx.x * rcap), one
// shared-memory reservation per warp and chunk; the region's count is
// written at the end.
template <uint32_t THREADS, uint32_t MINB, bool ORIENT>
__global__ void __launch_bounds__(THREADS, MINB) k_heavy_split(const Geo G, const uint32_t *__restrict__ pairs,
                                                               uint64_t n, const uint32_t *__restrict__ count,
                                                               const uint32_t *__restrict__ key, uint32_t kmax,
                                                               uint32_t kwords, uint32_t *__restrict__ bits_g,
                                                               uint32_t *__restrict__ list, uint32_t *__restrict__ ctr,
                                                               uint2 *__restrict__ resid, uint64_t rcap,
                                                               uint32_t *__restrict__ rcount, uint4 *__restrict__ zero,
                                                               uint64_t zq) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t *tab = sm;
    uint32_t *bm = sm + kTabWords;
    __shared__ uint32_t s_cnt;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    if (tid == 0) s_cnt = 0;
    split_select<THREADS>(count, key, ctr + kHeavyCtrHist, kmax, tab, bm, kwords, list, ctr);
    __syncthreads();
    uint2 *region = resid + (uint64_t)blockIdx.x * rcap;
    const uint32_t bm_s = static_cast<uint32_t>(__cvta_generic_to_shared(bm));
    const uint32_t kmask = kwords / G.W - 1u;          // heavy sources held: a power of two
    const uint32_t lw = __ffs(G.W) - 1u;               // W = g / 32 words per bitmap, a power of two
    const uint32_t seed_fold = G.seed_bv ^ (G.seed_bv >> 16);
    // chunk numbers fit 32 bits: a pass holds far fewer than 2^40 packets
    const uint32_t chunks = (uint32_t)((n + 255) / 256);
    const uint32_t full = (reinterpret_cast<uintptr_t>(pairs) & 15u) == 0 ? (uint32_t)(n / 256) : 0u;
    const uint32_t nw = gridDim.x * (THREADS / 32);
    uint32_t c = blockIdx.x * (THREADS / 32) + (tid >> 5);
    uint4 q[4], qn[4];
    uint32_t ok = c < chunks ? split_load(pairs, n, c, lane, full, q) : 0u;
    // the cube's zeroing spread over the chunk loop: one 16-byte store per thread every
    // zevery chunks, the rest after the loop
    const uint64_t zstride = (uint64_t)gridDim.x * THREADS;
    uint64_t zi = (uint64_t)blockIdx.x * THREADS + tid;
    const uint32_t wchunks = (chunks + nw - 1) / nw, zper = (uint32_t)((zq + zstride - 1) / zstride);
    const uint32_t zevery = zper ? (wchunks / zper > 1 ? wchunks / zper : 1) : 0xFFFFFFFFu;
    uint32_t zt = 0;
    for (; c < chunks; c += nw) {
        if (++zt >= zevery && zi < zq) {
            zero[zi] = make_uint4(0u, 0u, 0u, 0u);
            zi += zstride;
            zt = 0;
        }
        const uint32_t okn = c + nw < chunks ? split_load(pairs, n, c + nw, lane, full, qn) : 0u;
        uint32_t a[8], b[8];
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            a[k] = (k & 1u) ? q[k / 2].z : q[k / 2].x;
            b[k] = (k & 1u) ? q[k / 2].w : q[k / 2].y;
        }
        if (!ORIENT && __all_sync(0xffffffffu, ok == 0xFFu))      // the same path for the whole warp
            split_packets<8, false, true>(G, tab, bm, bm_s, kmask, lw, seed_fold, a, b, ok, region, &s_cnt, lane);
        else
            split_packets<8, ORIENT, false>(G, tab, bm, bm_s, kmask, lw, seed_fold, a, b, ok, region, &s_cnt, lane);
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) q[j] = qn[j];
        ok = okn;
    }
    for (; zi < zq; zi += zstride) zero[zi] = make_uint4(0u, 0u, 0u, 0u);
    split_flush(bm, kwords, bits_g, &s_cnt, rcount);
}

uint32_t heavy_budget(const cbaa_tuning &T) { return T.heavy == 2 ? (64u << 10) : kHeavyBitmapMax; }

// Heavy sources that fit the bitmap budget (W words each), at most kHeavyMax.
uint32_t heavy_sources(const Geo &G, const cbaa_tuning &T) {
    const uint32_t k = heavy_budget(T) / (4u * G.W);
    return k < kHeavyMax ? k : kHeavyMax;
}

// Split blocks: threads and blocks per SM (the lookup table and the bitmaps
// take most of an SM's shared memory).
struct SplitShape {
    uint32_t threads, per_sm;
};
SplitShape split_shape(const cbaa_tuning &) { return SplitShape{1024, 1}; }

// Residual regions of a split pass over m packets: one per split block,
// each as large as the chunks its warps can take, rounded up to kHeavyRegionAlign.
Residual residual_layout(const cbaa_tuning &T, uint64_t m, const uint32_t *entries_base, const uint32_t *rcount) {
    const SplitShape sh = split_shape(T);
    const uint64_t chunks = (m + 255) / 256;
    const uint64_t wpb = sh.threads / 32;
    // at least a region's worth of packets per block, so that rounding regions up wastes little
    uint64_t blocks = (uint64_t)num_sms() * sh.per_sm;
    if (T.split_blocks && T.split_blocks < blocks) blocks = T.split_blocks;      // SMs left to other streams
    const uint64_t need = (m + kHeavyRegionAlign - 1) / kHeavyRegionAlign;
    if (need < blocks) blocks = need;
    if (blocks > kHeavyMaxRegions) blocks = kHeavyMaxRegions;
    if (blocks == 0) blocks = 1;
    const uint64_t nw = blocks * wpb;
    const uint64_t per_warp = (chunks + nw - 1) / nw;
    const uint64_t rcap = (wpb * per_warp * 256 + kHeavyRegionAlign - 1) / kHeavyRegionAlign * kHeavyRegionAlign;
    return Residual{reinterpret_cast<const uint2 *>(entries_base), rcount, rcap, (uint32_t)blocks,
                    HeavyExpand{nullptr, nullptr, nullptr, 0}};
}

template <uint32_t THREADS, uint32_t MINB, bool ORIENT>
cudaError_t launch_split(const Geo &G, const uint32_t *pairs, uint64_t m, const BinWs &W, uint32_t K,
                         uint32_t kwords, const Residual &R, uint32_t *zero, cudaStream_t s) {
    auto k = k_heavy_split<THREADS, MINB, ORIENT>;
    const size_t smem = sizeof(uint32_t) * ((size_t)kTabWords + kwords);
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<R.nreg, THREADS, smem, s>>>(G, pairs, m, W.heavy.count, W.heavy.key, K, kwords, W.heavy.bits, W.heavy.list,
                                    W.heavy.ctr, const_cast<uint2 *>(R.entries), R.rcap, W.heavy.rcount(),
                                    reinterpret_cast<uint4 *>(zero), zero ? G.cube_words / 4 : 0);
    return cudaGetLastError();
}

template <bool ORIENT>
cudaError_t heavy_pass(const Geo &G, uint32_t *cube, const uint32_t *pairs, uint64_t m, const BinWs &W,
                       const cbaa_tuning &T, bool sampled, bool zero_cube, cudaStream_t s) {
    const uint32_t K = heavy_sources(G, T);
    const uint32_t kwords = K * G.W;
    const int sms = num_sms();
    cudaError_t e;
    if ((e = cudaMemsetAsync(W.heavy.count, 0, heavy_clear_bytes(G), s)) != cudaSuccess) return e;
    const size_t count_smem = sizeof(uint32_t) * kCountSlots;
    if ((e = allow_smem(k_heavy_sample<ORIENT>, count_smem)) != cudaSuccess) return e;
    const uint64_t tiles = (m + (uint64_t)kSampleTile * kHeavySampleEvery - 1) / ((uint64_t)kSampleTile * kHeavySampleEvery);
    // half the SMs: every block scans and flushes its whole 2^15-slot table, so fewer, fuller blocks
    const uint64_t sblocks = (uint64_t)(sms > 1 ? sms / 2 : 1);
    k_heavy_sample<ORIENT><<<(unsigned)(tiles < sblocks ? tiles : sblocks), kSampleThreads, count_smem, s>>>(
        G, pairs, m, W.heavy.count, W.heavy.key);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const uint32_t nb = rowtile_bins(G, 1);
    k_heavy_hist<<<kCountSlots / 1024, 1024, 0, s>>>(W.heavy.count, W.heavy.ctr + kHeavyCtrHist, W.counts, nb + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Residual R = residual_layout(T, m, W.codes, W.heavy.rcount());
    R.x = HeavyExpand{W.heavy.list, W.heavy.ctr, W.heavy.bits, K};
    e = launch_split<1024, 1, ORIENT>(G, pairs, m, W, K, kwords, R, zero_cube ? cube : nullptr, s);
    if (e != cudaSuccess) return e;
    // the residual's row-tile pass in the room after the residual regions
    const uint64_t rw = 2 * (uint64_t)R.nreg * R.rcap;
    BinWs W2 = W;
    W2.codes = W.codes + rw;
    W2.words = W.words - rw;
    return rowtile_pass_residual(G, cube, R, m, W2, T, sampled, s);     // its counts were zeroed by k_heavy_hist
}

}  // namespace

bool heavy_enabled(const Geo &G, uint32_t n_cubes, uint64_t n, const cbaa_tuning &T) {
    if (T.heavy == 1 || n_cubes != 1 || T.tile_kind == 1 || !rowtile_ok(G, 1)) return false;
    if (heavy_sources(G, T) < 16) return false;
    return T.heavy >= 2 || n >= kHeavyMinPackets;
}

cudaError_t launch_update_heavy(const Geo &G, uint32_t *cube, const uint32_t *pairs, uint64_t n, const BinWs &W,
                                const cbaa_tuning &T, cudaStream_t s, bool assign) {
    if (n == 0) return cudaSuccess;
    // Largest pass that fits the code buffer: the residual entries (2 words per
    // packet) and the row-tile pass over them, whose run capacities come from a
    // sample as in the plain row-tile path (tile_kind 3, or 0 for passes of at
    // least kRowTileMinSampled packets) unless that leaves passes too small.
    auto fit = [&](bool sampled) -> uint64_t {
        auto need = [&](uint64_t m) {
            const Residual R = residual_layout(T, m, nullptr, nullptr);
            return 2 * (uint64_t)R.nreg * R.rcap + rowtile_pass_words(G, m, sampled);
        };
        if (need(n) <= W.words) return n;
        uint64_t lo = 0, hi = n;
        while (hi - lo > 1) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (need(mid) <= W.words) lo = mid; else hi = mid;
        }
        return lo >= 1024 ? (lo & ~(uint64_t)1023) : lo;   // whole chunks keep later passes 16-byte aligned
    };
    bool sampled = T.tile_kind == 3 || (T.tile_kind == 0 && n >= kRowTileMinSampled);
    uint64_t mmax = sampled ? fit(true) : 0;
    const uint64_t counted = fit(false);
    if (sampled && mmax < (T.tile_kind == 3 ? (n < (1u << 16) ? n : (1u << 16)) : counted)) sampled = false;
    if (!sampled) mmax = counted;
    if (mmax == 0) return cudaErrorInvalidValue;       // not reached: a workspace holds A + 2 words per packet
    if (assign && (G.cube_words & 3u)) {              // not whole 16-byte words: a memset first
        const cudaError_t e = cudaMemsetAsync(cube, 0, G.cube_words * 4u, s);
        if (e != cudaSuccess) return e;
        assign = false;
    }
    for (uint64_t done = 0; done < n;) {
        const uint64_t m = n - done < mmax ? n - done : mmax;
        // later passes OR into the first one's cube (columns of >= 32 words: whole 16-byte words)
        const bool zero = assign && done == 0;
        const cudaError_t e = G.n_inner > 0 ? heavy_pass<true>(G, cube, pairs + 2 * done, m, W, T, sampled, zero, s)
                                            : heavy_pass<false>(G, cube, pairs + 2 * done, m, W, T, sampled, zero, s);
        if (e != cudaSuccess) return e;
        done += m;
    }
    return cudaSuccess;
}

}  // namespace cbaa
