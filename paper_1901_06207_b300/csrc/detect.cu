// End-of-window restoration (Section III.C): Alg. 2 hot columns, Alg. 3
// tuple checks, Thm. 2 estimates, for sm_103a.
//
// The paper tests every tuple of the product HC(0) x ... x HC(|RA|-1).  Here
// the tuples are built one RA at a time instead, which reaches the same set:
//  * HC(i) for i >= 1 is stored grouped by its low |CP(i-1)| bits, so the
//    only candidates for position i after a partial tuple ending in hc_{i-1}
//    are one bucket: those whose first bits equal CP(i-1) of hc_{i-1}
//    (Alg. 3 step 1, applied as soon as both columns are known);
//  * a partial tuple is dropped as soon as the AND of its columns has more
//    than Zmax zero bits: adding columns to an AND only adds zeros, so such
//    a tuple's union column could never pass Alg. 3 step 4.
// The last stage closes the ring (CP(last) against the first bits of
// hc_0), concatenates the EPs into LP (step 2), ANDs in the VA columns
// H_j(LP) (step 3) and keeps LP when the union has at most Zmax zeros
// (step 4).  One warp owns one partial tuple and holds its running AND in
// registers (g/32 words spread over 32 lanes), so no union-column buffer
// pool is needed.
#include <cmath>
#include <cstddef>

#include "cbaa_internal.cuh"
#include "detect_layout.h"

namespace cbaa {

namespace {

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) { return __reduce_add_sync(0xffffffffu, v); }

static_assert(sizeof(cbaa_host) == 16 && offsetof(cbaa_host, z_union) == 4 && offsetof(cbaa_host, est) == 8 &&
                  offsetof(cbaa_host, flags) == 12,
              "the join stages hosts as 16-byte {ip, z_union, est, flags} records");

// ---------------------------------------------------------------------------
// Alg. 2.  Block (cs, i) lists the columns of RA i of sketch cs with no more
// than Zmax zero bits.  For i = 0 the hot columns become the seed tuples
// (cs, hc_0) of the join; for i >= 1 they are stored key-major (key = low
// |CP(i-1)| bits) with bucket offsets.
__global__ void __launch_bounds__(1024) k_hot_lists(const Geo G, WsPtrs P, uint32_t cs_lo) {
    const uint32_t cs = cs_lo + blockIdx.x, i = blockIdx.y;
    const uint32_t ncol = 1u << G.cbn[i];
    const int64_t zm = P.zmax[cs];
    const uint32_t kb = (i == 0) ? 0u : G.cp[i - 1];
    const uint32_t jb = G.cbn[i] - kb;
    const uint16_t *zc = P.zc + ((size_t)cs * G.A + i) * G.cmax;
    uint16_t *list = P.hc + ((size_t)cs * G.n_ra + i) * P.hc_stride;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr uint32_t CPT = 4;                       // list positions p per thread and chunk

    __shared__ uint32_t warp_tot[32], s_base, s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();

    // list position p holds column ((p mod 2^jb) << kb) | (p >> jb): key-major order
    for (uint32_t p0 = 0; p0 < ncol; p0 += CPT * blockDim.x) {
        uint32_t col[CPT], mine = 0, flags = 0;
#pragma unroll
        for (uint32_t j = 0; j < CPT; ++j) {
            const uint32_t p = p0 + CPT * threadIdx.x + j;
            col[j] = 0;
            if (p < ncol) {
                col[j] = ((p & ((1u << jb) - 1u)) << kb) | (p >> jb);
                if ((int64_t)zc[col[j]] <= zm) {
                    flags |= 1u << j;
                    ++mine;
                }
            }
        }
        uint32_t x = mine;                            // exclusive position of this thread's hot columns
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < blockDim.x / 32 ? warp_tot[lane] : 0u;
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            warp_tot[lane] = v;                       // inclusive over warps
            if (lane == 31) {
                s_base = s_count;
                s_count += v;
                if (i == 0 && v > 0) s_base = atomicAdd(&P.state->stage_count[0], v);
            }
        }
        __syncthreads();
        uint32_t pos = s_base + (warp ? warp_tot[warp - 1] : 0u) + x - mine;
#pragma unroll
        for (uint32_t j = 0; j < CPT; ++j) {
            if (!(flags >> j & 1u)) continue;
            if (i == 0) {
                if (pos < P.m) {
                    Tuple t;
                    t.cs = (uint16_t)cs;
                    t.hc[0] = (uint16_t)col[j];
                    P.tup[0][pos] = t;
                }
            } else {
                list[pos] = (uint16_t)col[j];
            }
            ++pos;
        }
        __syncthreads();
    }
    const uint32_t n = s_count;
    if (threadIdx.x == 0) {
        P.nhc[(size_t)cs * G.n_ra + i] = n;
        if (n) atomicAdd(&P.state->info.n_hot, n);
    }
    if (i == 0) return;
    __syncthreads();   // the list written above is visible to the whole block
    uint32_t *offs = P.boff + ((size_t)cs * G.n_ra + i) * P.boff_stride;
    const uint32_t nkeys = 1u << kb, kmask = nkeys - 1u;
    if (n == 0) {
        for (uint32_t k = threadIdx.x; k <= nkeys; k += blockDim.x) offs[k] = 0;
        return;
    }
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        const uint32_t key = list[t] & kmask;
        const int64_t prev = (t == 0) ? -1 : (int64_t)(list[t - 1] & kmask);
        for (int64_t k = prev + 1; k <= (int64_t)key; ++k) offs[k] = t;
        if (t == n - 1)
            for (uint32_t k = key + 1; k <= nkeys; ++k) offs[k] = n;
    }
}

// Words of one column held by a lane: WPL consecutive words for g >= 1024,
// else lane < W holds word `lane`.
template <int WPL>
__device__ __forceinline__ void load_col(const uint32_t *__restrict__ colp, uint32_t W, uint32_t lane, uint32_t (&v)[WPL]) {
    if (WPL >= 4) {
        const uint4 *p4 = reinterpret_cast<const uint4 *>(colp + lane * WPL);
#pragma unroll
        for (int k = 0; k < WPL / 4; ++k) {
            const uint4 q = p4[k];
            v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
        }
    } else if (WPL == 2) {
        const uint2 q = reinterpret_cast<const uint2 *>(colp)[lane];
        v[0] = q.x; v[WPL - 1] = q.y;
    } else {
        v[0] = (lane < W) ? colp[lane] : 0xFFFFFFFFu;
    }
}

// Join stage s (1 <= s < |RA|): extend each partial tuple (cs, hc_0..hc_{s-1})
// by the hot columns of RA s in its CP bucket.
template <int WPL>
__global__ void __launch_bounds__(256) k_join(const Geo G, const uint32_t *__restrict__ cube, WsPtrs P, uint32_t s) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const bool last = (s == G.n_ra - 1);
    const uint32_t cnt_in = P.state->stage_count[s - 1];
    const uint32_t n_in = cnt_in < P.m ? cnt_in : P.m;
    const Tuple *__restrict__ in = P.tup[(s - 1) & 1];
    Tuple *__restrict__ out = P.tup[s & 1];
    const bool lane_live = (WPL > 1) || lane < G.W;
    // Each warp stages its outputs (tuples, or hosts in the last stage; both
    // 16-byte records) and reserves their slots with one atomic per 32, not
    // one per output: thousands of outputs would otherwise queue on one
    // counter.
    __shared__ uint4 wbuf[8][32];
    uint4 *mybuf = wbuf[threadIdx.x >> 5];
    uint32_t *counter = last ? &P.state->info.n_hosts : &P.state->stage_count[s];
    uint4 *dst = last ? reinterpret_cast<uint4 *>(P.hosts) : reinterpret_cast<uint4 *>(out);
    uint32_t nbuf = 0;                                 // the same in every lane
    auto flush = [&]() {
        __syncwarp();
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(counter, nbuf);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < nbuf && base + lane < P.m) dst[base + lane] = mybuf[lane];
        nbuf = 0;
        __syncwarp();
    };

    for (uint32_t t = gw; t < n_in; t += nw) {
        const Tuple tu = in[t];
        const uint32_t cs = tu.cs;
        const int64_t zm = P.zmax[cs];
        uint32_t acc[WPL];
#pragma unroll
        for (int k = 0; k < WPL; ++k) acc[k] = 0xFFFFFFFFu;
        for (uint32_t i = 0; i < s; ++i) {
            uint32_t v[WPL];
            load_col<WPL>(cube + col_word0(G, cs, i, tu.hc[i]), G.W, lane, v);
#pragma unroll
            for (int k = 0; k < WPL; ++k) acc[k] &= v[k];
        }
        const uint32_t key = (uint32_t)tu.hc[s - 1] >> G.ep[s - 1];
        const uint32_t *offs = P.boff + ((size_t)cs * G.n_ra + s) * P.boff_stride;
        const uint16_t *list = P.hc + ((size_t)cs * G.n_ra + s) * P.hc_stride;
        const uint32_t b0 = offs[key], b1 = offs[key + 1];
        // LP bits already fixed by the EPs of hc_0 .. hc_{s-1}
        uint32_t lp_part = 0;
        if (last)
            for (uint32_t i = 0; i < s; ++i) lp_part |= ((uint32_t)tu.hc[i] & ((1u << G.ep[i]) - 1u)) << G.ring_off[i];
        const uint32_t close_bits = (uint32_t)tu.hc[0] & ((1u << G.cp[s]) - 1u);

        // The bucket is read 32 entries at a time, one per lane, with the ring
        // closure (Alg. 3 step 1, last stage) tested in every lane at once; the
        // surviving candidates are taken U at a time: all their column loads
        // (and, in the last stage, the VA columns, which need only the list
        // entry), then the U reductions.  pending and ok[u] are the same in
        // every lane.
        constexpr int U = WPL >= 4 ? 1 : 4 / WPL;
        for (uint32_t g0 = b0; g0 < b1; g0 += 32) {
            const uint32_t e = g0 + lane;
            const uint32_t mine = e < b1 ? (uint32_t)list[e] : 0u;
            const bool pass = e < b1 && (!last || (mine >> G.ep[s]) == close_bits);
            uint32_t pending = __ballot_sync(0xffffffffu, pass);
            while (pending) {
                uint32_t col[U];
                bool ok[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    ok[u] = pending != 0;
                    const uint32_t l = ok[u] ? (uint32_t)__ffs(pending) - 1 : 0u;
                    col[u] = __shfl_sync(0xffffffffu, mine, l);
                    if (ok[u]) pending &= pending - 1;
                }
                uint32_t v[U][WPL], lp[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (ok[u]) {
                        load_col<WPL>(cube + col_word0(G, cs, s, col[u]), G.W, lane, v[u]);
                    } else {
#pragma unroll
                        for (int k = 0; k < WPL; ++k) v[u][k] = 0u;
                    }
                    lp[u] = lp_part | ((col[u] & ((1u << G.ep[s]) - 1u)) << G.ring_off[s]);   // step 2
                }
                if (last) {
                    for (uint32_t j = 0; j < G.n_va; ++j) {                                     // step 3
                        uint32_t w[U][WPL];
#pragma unroll
                        for (int u = 0; u < U; ++u) {
                            if (ok[u]) {
                                load_col<WPL>(cube + col_word0(G, cs, G.n_ra + j, va_col(G, j, lp[u])), G.W, lane, w[u]);
                            } else {
#pragma unroll
                                for (int k = 0; k < WPL; ++k) w[u][k] = 0u;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u)
#pragma unroll
                            for (int k = 0; k < WPL; ++k) v[u][k] &= w[u][k];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!ok[u]) continue;
                    uint32_t ones = 0;
                    if (lane_live) {
#pragma unroll
                        for (int k = 0; k < WPL; ++k) ones += __popc(v[u][k] & acc[k]);
                    }
                    ones = warp_sum(ones);
                    const uint32_t zeros = G.g - ones;
                    if ((int64_t)zeros > zm) continue;                                   // step 4
                    if (lane == 0) {
                        if (!last) {
                            Tuple o = tu;
                            o.hc[s] = (uint16_t)col[u];
                            mybuf[nbuf] = *reinterpret_cast<const uint4 *>(&o);
                        } else {
                            // Thm. 2 estimate; Z = 0 is reported with Z = 1 and flagged.
                            const double g = (double)G.g;
                            const double eps = P.eps[cs];
                            const uint32_t zs = zeros ? zeros : 1u;
                            const double den = __dsub_rn(g, __dmul_rn(g, eps));
                            double est = __dmul_rn(-g, log(__ddiv_rn((double)zs, den)));
                            if (est < 0.0) est = 0.0;
                            // a cbaa_host record: {ip, z_union, est, flags}
                            mybuf[nbuf] = make_uint4(unmangle(G, (lp[u] << G.r) | cs), zeros,
                                                     __float_as_uint((float)est), zeros ? 0u : CBAA_FLAG_SATURATED);
                        }
                    }
                    if (++nbuf == 32) flush();
                }
            }
        }
    }
    if (nbuf) flush();
}

// Sorting the host list by ip, writing the first min(n, cap) to `out`, and
// settling the status, in one launch.  Lists of up to kRankMax entries are
// sorted by rank: every thread owns one host and counts the hosts with a
// smaller ip (ties broken by index), which is its place in the output; the
// keys are read tile by tile through shared memory.  Longer lists go through
// a bitonic network over (ip << 32 | index) keys in block 0 (in shared memory
// up to kSmemKeys keys, else in the workspace).  The status depends only on
// the stage counts, which are final when this kernel runs; block 0 writes it.
constexpr uint32_t kRankMax = 1u << 16;
constexpr uint32_t kRankThreads = 256;
constexpr uint32_t kRankLanes = 8;               // lanes sharing one host's count
constexpr uint32_t kRankTile = 4096;
constexpr uint32_t kSmemKeys = 4096;

__device__ void bitonic_out(WsPtrs P, uint32_t n, cbaa_host *__restrict__ out, uint64_t cap,
                            unsigned long long *skeys) {
    uint32_t N = 1;
    while (N < n) N <<= 1;
    unsigned long long *keys = (N <= kSmemKeys) ? skeys : P.keys;
    for (uint32_t k = threadIdx.x; k < N; k += blockDim.x)
        keys[k] = (k < n) ? (((unsigned long long)P.hosts[k].ip << 32) | k) : ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= N; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
                const uint32_t lo = 2 * t - (t & (stride - 1));
                const uint32_t hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) { keys[lo] = b; keys[hi] = a; }
            }
            __syncthreads();
        }
    }
    const uint64_t nw = n < cap ? n : cap;
    for (uint32_t k = threadIdx.x; k < nw; k += blockDim.x) out[k] = P.hosts[keys[k] & 0xFFFFFFFFull];
}

// info_copy (may be null): where the settled detect info is also written.
__global__ void __launch_bounds__(kRankThreads) k_sort(const Geo G, WsPtrs P, cbaa_host *__restrict__ out,
                                                       uint64_t cap, cbaa_detect_info *__restrict__ info_copy) {
    __shared__ uint32_t keys[kRankTile];
    __shared__ unsigned long long skeys[kSmemKeys];
    DevState *st = P.state;
    const uint32_t found = st->info.n_hosts;
    const uint32_t n = found < P.m ? found : P.m;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t need = 0, tuples = 0;
        for (uint32_t s = 0; s + 1 < G.n_ra; ++s) {
            const uint32_t c = st->stage_count[s];
            tuples += c;
            if (c > P.m && c > need) need = c;
        }
        if (found > P.m && found > need) need = found;
        st->info.n_tuples = tuples;
        st->info.need_tuples = need;
        st->info.status = need ? CBAA_ERR_WORKSPACE : (found > cap ? CBAA_ERR_CAPACITY : CBAA_OK);
        if (info_copy) *info_copy = st->info;        // every other field was final before this kernel
    }
    if (n > kRankMax) {
        if (blockIdx.x == 0) bitonic_out(P, n, out, cap, skeys);
        return;
    }
    constexpr uint32_t per_block = kRankThreads / kRankLanes;
    if ((uint64_t)blockIdx.x * per_block >= n) return;
    const uint32_t sub = threadIdx.x % kRankLanes;
    const uint32_t i = blockIdx.x * per_block + threadIdx.x / kRankLanes;
    const uint32_t me = i < n ? P.hosts[i].ip : 0u;
    uint32_t rank = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += kRankTile) {
        const uint32_t len = (n - t0) < kRankTile ? (n - t0) : kRankTile;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < len; j += kRankThreads) keys[j] = P.hosts[t0 + j].ip;
        __syncthreads();
        uint32_t r0 = 0, r1 = 0;
        uint32_t j = sub;
        for (; j + kRankLanes < len; j += 2 * kRankLanes) {
            const uint32_t a = keys[j], b = keys[j + kRankLanes];
            r0 += (a < me) || (a == me && t0 + j < i);
            r1 += (b < me) || (b == me && t0 + j + kRankLanes < i);
        }
        if (j < len) {
            const uint32_t a = keys[j];
            r0 += (a < me) || (a == me && t0 + j < i);
        }
        rank += r0 + r1;
    }
    for (uint32_t off = kRankLanes / 2; off > 0; off >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, off);
    if (sub == 0 && i < n && rank < cap) out[rank] = P.hosts[i];
}

template <int WPL>
cudaError_t launch_join(const Geo &G, const uint32_t *cube, const WsPtrs &P, uint32_t s, unsigned blocks, cudaStream_t st) {
    k_join<WPL><<<blocks, 256, 0, st>>>(G, cube, P, s);
    return cudaGetLastError();
}

}  // namespace

int detect_enqueue(const Geo &G, const uint32_t *cube, uint32_t theta, void *ws, size_t ws_bytes,
                   cbaa_host *out, uint64_t cap, cbaa_detect_info *info_copy, int num_sms, cudaStream_t s,
                   uint32_t cs_lo, uint32_t cs_hi) {
    if (cs_hi == 0) cs_hi = G.smask + 1;
    if (cs_lo >= cs_hi || cs_hi > G.smask + 1) return CBAA_ERR_INVALID_ARG;
    WsLayout Ly;
    if (!ws_layout_fit(G, ws_bytes, &Ly)) return CBAA_ERR_WORKSPACE;
    WsPtrs P = ws_pointers(G, Ly, ws);
    const double E = std::exp(-((double)theta / (double)G.g));

    // the state words and the array zero totals (laid out next to each other) in one memset
    const size_t cleared = Ly.za - Ly.state + sizeof(uint64_t) * (size_t)(G.smask + 1) * G.A;
    cudaError_t e = cudaMemsetAsync(P.state, 0, cleared, s);
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_column_stats(G, cube, P.zc, P.za, P.eps, P.zmax, E, s, cs_lo, cs_hi, &P.state->stats_done, true);
    if (e != cudaSuccess) return cuda_status(e);
    k_hot_lists<<<dim3(cs_hi - cs_lo, G.n_ra), 1024, 0, s>>>(G, P, cs_lo);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    const unsigned blocks = (unsigned)num_sms * 4;
    const uint32_t wpl = G.W >= 32 ? G.W / 32 : 1;
    for (uint32_t st = 1; st < G.n_ra; ++st) {
        switch (wpl) {
            case 1: e = launch_join<1>(G, cube, P, st, blocks, s); break;
            case 2: e = launch_join<2>(G, cube, P, st, blocks, s); break;
            case 4: e = launch_join<4>(G, cube, P, st, blocks, s); break;
            case 8: e = launch_join<8>(G, cube, P, st, blocks, s); break;
            case 16: e = launch_join<16>(G, cube, P, st, blocks, s); break;
            default: e = launch_join<32>(G, cube, P, st, blocks, s); break;
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    cbaa_host *dst = out ? out : P.sorted;
    const uint64_t dcap = out ? cap : P.m;
    const uint64_t rank_n = P.m < kRankMax ? P.m : kRankMax;
    const uint64_t per_block = kRankThreads / kRankLanes;
    const uint64_t sort_blocks = (rank_n + per_block - 1) / per_block;
    k_sort<<<(unsigned)(sort_blocks ? sort_blocks : 1), kRankThreads, 0, s>>>(G, P, dst, dcap, info_copy);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    return CBAA_OK;
}

// ---------------------------------------------------------------------------
// Host lists of several owners (ranks that restored disjoint sketch ranges,
// Section III.C's global server split by sketch), each sorted by ip in its
// own block of `cap` records with its count in infos[j].n_hosts, merged into
// one list sorted by ip.  The owners' addresses are disjoint, so a record's
// place is its index in its list plus, for every other list, the number of
// records with a smaller ip (a binary search each).  One thread per record.
__global__ void k_merge_hosts(const cbaa_host *__restrict__ blocks, uint32_t cap, uint32_t k,
                              const cbaa_detect_info *__restrict__ infos, cbaa_host *__restrict__ out,
                              uint64_t out_cap) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (uint64_t)k * cap; t += stride) {
        const uint32_t j = (uint32_t)(t / cap), i = (uint32_t)(t - (uint64_t)j * cap);
        const uint32_t nj = infos[j].n_hosts < cap ? infos[j].n_hosts : cap;
        if (i >= nj) continue;
        const cbaa_host h = blocks[t];
        uint64_t place = i;
        for (uint32_t o = 0; o < k; ++o) {
            if (o == j) continue;
            const cbaa_host *b = blocks + (uint64_t)o * cap;
            uint32_t lo = 0, hi = infos[o].n_hosts < cap ? infos[o].n_hosts : cap;
            while (lo < hi) {                              // first record of list o with ip >= h.ip
                const uint32_t mid = (lo + hi) >> 1;
                if (b[mid].ip < h.ip) lo = mid + 1; else hi = mid;
            }
            place += lo;
        }
        if (place < out_cap) out[place] = h;
    }
}

// The merged list's info: the first status that is not OK (CAPACITY when
// the merged list exceeds out_cap), and the sums of the counts (n_hosts
// counts every host, also past any capacity).
__global__ void k_merge_infos(const cbaa_detect_info *__restrict__ infos, uint32_t k, uint64_t out_cap,
                              cbaa_detect_info *__restrict__ out) {
    if (threadIdx.x != 0) return;
    cbaa_detect_info r = {};
    r.status = CBAA_OK;
    for (uint32_t j = 0; j < k; ++j) {
        const cbaa_detect_info x = infos[j];
        if (r.status == CBAA_OK && x.status != CBAA_OK) r.status = x.status;
        r.n_hosts += x.n_hosts;
        r.n_hot += x.n_hot;
        r.n_tuples += x.n_tuples;
        r.need_tuples = r.need_tuples > x.need_tuples ? r.need_tuples : x.need_tuples;
    }
    if (r.status == CBAA_OK && r.n_hosts > out_cap) r.status = CBAA_ERR_CAPACITY;
    *out = r;
}

cudaError_t launch_merge_hosts(const cbaa_host *blocks, uint32_t cap, uint32_t k, const cbaa_detect_info *infos,
                               cbaa_host *out, uint64_t out_cap, cbaa_detect_info *info_out, cudaStream_t s) {
    const uint64_t total = (uint64_t)k * cap;
    if (total) {
        const uint64_t want = (total + 255) / 256, lim = (uint64_t)num_sms() * 8;
        k_merge_hosts<<<(unsigned)(want < lim ? want : lim), 256, 0, s>>>(blocks, cap, k, infos, out, out_cap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_merge_infos<<<1, 32, 0, s>>>(infos, k, out_cap, info_out);
    return cudaGetLastError();
}

}  // namespace cbaa
