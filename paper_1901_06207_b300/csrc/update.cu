// Alg. 1 (cube update), the OR merge of Section III.C, and the column
// statistics of the end-of-window pass (zero counts, Thm. 1 eps, the
// hot-column bound) for sm_103a.
//
// Update design: the cube is written only by single-bit ORs (Alg. 1 never
// reads it), so every bit set is a fire-and-forget reduction (RED.OR) that
// is executed in L2 without a round trip.  The packet stream (8 B per pair)
// is read with 128-bit loads marked evict-first so that it does not push
// the cube out of L2; the cube itself is left with the default policy and
// stays L2-resident when it fits.
#include <atomic>
#include <mutex>

#include "cbaa_internal.cuh"

namespace cbaa {

namespace {

__device__ __forceinline__ uint4 ld_stream(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.global.or.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// One IP pair through Alg. 1.  NRA/NVA > 0 fix the array counts at compile
// time (the common 3+1 layout); 0 reads them from G.
template <int NRA, int NVA>
__device__ __forceinline__ void apply_pair(const Geo &G, uint32_t *__restrict__ cube, uint32_t iip, uint32_t oip) {
    if (G.n_inner && !orient(G, iip, oip)) return;      // raw {src, dst} against NI (Section III)
    const uint32_t nra = NRA ? NRA : G.n_ra;
    const uint32_t nva = NRA ? NVA : G.n_va;
    const uint32_t row = row_of(G, oip);
    const uint32_t m = mangle(G, iip);
    const uint32_t cs = m & G.smask;            // right r bits select the CS
    const uint32_t lp = m >> G.r;               // left 32 - r bits
    const uint32_t bit = 1u << (row & 31u);
    uint32_t *base = cube + (size_t)cs * G.cs_words + (row >> 5);
#pragma unroll
    for (uint32_t i = 0; i < (NRA ? NRA : CBAA_MAX_RA); ++i) {
        if (NRA == 0 && i >= nra) break;
        red_or(base + G.arr_base[i] + ra_col(G, i, lp) * G.W, bit);
    }
#pragma unroll
    for (uint32_t j = 0; j < (NRA ? NVA : CBAA_MAX_ARRAYS); ++j) {
        if (NRA == 0 && j >= nva) break;
        red_or(base + G.arr_base[nra + j] + va_col(G, j, lp) * G.W, bit);
    }
}

// Grid-stride over 16-byte pairs-of-pairs; each thread keeps U loads in
// flight before issuing their 2*U*A reductions.  Thread 0 of block 0 also
// takes the unaligned head pair and the odd tail pair.
template <int NRA, int NVA, int U>
__global__ void __launch_bounds__(256) k_update(const Geo G, uint32_t *__restrict__ cube,
                                                const uint32_t *__restrict__ pairs, uint64_t n) {
    const uint64_t head = ((reinterpret_cast<uintptr_t>(pairs) & 15u) != 0 && n > 0) ? 1 : 0;
    const uint4 *body = reinterpret_cast<const uint4 *>(pairs + 2 * head);
    const uint64_t n2 = (n - head) / 2;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;

    if (tid == 0) {
        if (head) apply_pair<NRA, NVA>(G, cube, pairs[0], pairs[1]);
        if ((n - head) & 1) {
            const uint64_t t = n - 1;
            apply_pair<NRA, NVA>(G, cube, pairs[2 * t], pairs[2 * t + 1]);
        }
    }
    uint64_t i = tid;
    for (; i + (U - 1) * stride < n2; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_stream(body + i + u * stride);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            apply_pair<NRA, NVA>(G, cube, v[u].x, v[u].y);
            apply_pair<NRA, NVA>(G, cube, v[u].z, v[u].w);
        }
    }
    for (; i < n2; i += stride) {
        const uint4 v = ld_stream(body + i);
        apply_pair<NRA, NVA>(G, cube, v.x, v.y);
        apply_pair<NRA, NVA>(G, cube, v.z, v.w);
    }
}

// ---------------------------------------------------------------------------
// Merge: dst |= OR of up to kMaxSrc sources per launch, 128-bit words
// (assign: dst = OR of the sources, dst not read).

constexpr int kMaxSrc = 16;
struct SrcList {
    const uint4 *p[kMaxSrc];
    int k;
};

// Every source's 16 bytes are loaded before the first OR, so a thread keeps
// L.k + 1 loads in flight.
__global__ void __launch_bounds__(256) k_merge(uint4 *__restrict__ dst, const SrcList L, uint64_t n16, bool assign) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        uint4 b[kMaxSrc];
#pragma unroll
        for (int k = 0; k < kMaxSrc; ++k)
            if (k < L.k) b[k] = ld_stream(L.p[k] + i);
        uint4 a = assign ? make_uint4(0u, 0u, 0u, 0u) : dst[i];
#pragma unroll
        for (int k = 0; k < kMaxSrc; ++k)
            if (k < L.k) { a.x |= b[k].x; a.y |= b[k].y; a.z |= b[k].z; a.w |= b[k].w; }
        dst[i] = a;
    }
}

// ---------------------------------------------------------------------------
// Thm. 1 with measured one-bit fractions, then the hot-column bound, for one
// sketch.  Each operation is a correctly rounded IEEE double operation in a
// fixed order (explicit _rn intrinsics, so nothing is contracted into an
// FMA).  za is read from L2 (__ldcg): other blocks' atomics put it there.
__device__ void eps_zmax_of(const Geo &G, const unsigned long long *za, double E, uint32_t cs,
                            double *__restrict__ eps_out, int64_t *__restrict__ zmax_out) {
    double eps = 1.0;
    for (uint32_t a = 0; a < G.A; ++a) {
        const unsigned long long bits = (unsigned long long)(1u << G.cbn[a]) << G.log2_g;
        const unsigned long long ones = bits - __ldcg(za + (size_t)cs * G.A + a);
        const double p1 = __ddiv_rn(__ull2double_rn(ones), __ull2double_rn(bits));
        eps = __dmul_rn(eps, p1);
    }
    const double g = (double)G.g;
    double t;
    if (G.form == 1) {
        const double b = __dmul_rn(__dmul_rn(g, __dadd_rn(1.0, eps)), E);
        t = __dsub_rn(b, __dmul_rn(g, eps));
    } else {
        t = __dmul_rn(__dmul_rn(g, __dsub_rn(1.0, eps)), E);
    }
    if (eps_out) eps_out[cs] = eps;
    if (zmax_out) zmax_out[cs] = (int64_t)floor(t);
}

// ---------------------------------------------------------------------------
// Zero counts.  Block (cs*A + a, split) walks a slice of array a of sketch
// cs.  TPC threads share one column, each summing the popcounts of its
// PER 16-byte pieces (TPC = W/(4 kZcPieces) clamped to [1, 32], so a
// thread has kZcPieces pieces of a column when the column is long enough),
// then the TPC lanes reduce by shuffles.  kZcU columns per thread group are
// in flight.  One atomic per block adds the slice's zeros to za[cs][a].
constexpr uint32_t kZcPieces = 4;
constexpr uint32_t kZcU = 2;

// With `done` set, the last block to finish also computes eps and Zmax of the
// sketches [cs_lo, cs_hi) (one launch fewer in the detect); done counts the
// finished blocks and must start at zero.
__global__ void __launch_bounds__(256) k_zero_counts(const Geo G, const uint32_t *__restrict__ cube,
                                                     uint16_t *__restrict__ zc,
                                                     unsigned long long *__restrict__ za, uint32_t splits,
                                                     uint32_t arr0, uint32_t *__restrict__ done, double E,
                                                     double *__restrict__ eps_out, int64_t *__restrict__ zmax_out,
                                                     uint32_t cs_lo, uint32_t cs_hi) {
    const uint32_t arr = arr0 + blockIdx.x;          // cs*A + a
    const uint32_t cs = arr / G.A, a = arr % G.A;
    const uint32_t ncol = 1u << G.cbn[a];
    const uint32_t c0 = (uint32_t)(((uint64_t)ncol * blockIdx.y) / splits);
    const uint32_t c1 = (uint32_t)(((uint64_t)ncol * (blockIdx.y + 1)) / splits);
    const uint32_t q = G.W / 4;                      // 16-byte pieces per column
    const uint32_t t0 = q / kZcPieces;
    const uint32_t tpc = t0 < 1 ? 1 : (t0 > 32 ? 32 : t0);
    const uint32_t per = q / tpc;                    // pieces per thread
    const uint32_t sub = threadIdx.x % tpc;
    const uint32_t cols_per_iter = blockDim.x / tpc;
    const uint4 *arr4 = reinterpret_cast<const uint4 *>(cube + (size_t)cs * G.cs_words + G.arr_base[a]);

    unsigned long long acc = 0;
    constexpr uint32_t U = kZcU;
    for (uint32_t base = c0; base < c1; base += U * cols_per_iter) {
        uint32_t ones[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t col = base + u * cols_per_iter + threadIdx.x / tpc;
            ones[u] = 0;
            if (col < c1) {
                const uint4 *c4 = arr4 + (size_t)col * q + sub;
#pragma unroll 4
                for (uint32_t k = 0; k < per; ++k) {
                    const uint4 v = c4[k * tpc];
                    ones[u] += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                }
            }
        }
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t col = base + u * cols_per_iter + threadIdx.x / tpc;
            uint32_t o = ones[u];
            for (uint32_t off = tpc >> 1; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
            if (col < c1 && sub == 0) {
                const uint32_t zeros = G.g - o;
                if (zc) zc[(size_t)arr * G.cmax + col] = (uint16_t)zeros;
                acc += zeros;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ unsigned long long part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += part[w];
        atomicAdd(&za[arr], t);
        s_last = false;
        if (done) {
            __threadfence();
            s_last = atomicAdd(done, 1u) == gridDim.x * gridDim.y - 1;
        }
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (uint32_t cs = cs_lo + threadIdx.x; cs < cs_hi; cs += blockDim.x) eps_zmax_of(G, za, E, cs, eps_out, zmax_out);
    }
}

// eps and Zmax of the sketches [cs_lo, cs_hi) (eps_zmax_of).
__global__ void k_eps_zmax(const Geo G, const unsigned long long *__restrict__ za, double E,
                           double *__restrict__ eps_out, int64_t *__restrict__ zmax_out, uint32_t cs_lo,
                           uint32_t cs_hi) {
    const uint32_t cs = cs_lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (cs < cs_hi) eps_zmax_of(G, za, E, cs, eps_out, zmax_out);
}

}  // namespace

// SM count of the first device asked (only grid sizes depend on it); host
// threads may race to fill it in, with the same value.
static std::atomic<int> g_num_sms{0};

int num_sms() {
    int n = g_num_sms.load(std::memory_order_relaxed);
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 148;
        g_num_sms.store(n, std::memory_order_relaxed);
    }
    return n;
}

static std::mutex g_smem_mu;
struct SmemGrant { const void *fn; int dev; size_t bytes; };
static SmemGrant g_smem[256];
static int g_smem_n = 0;

cudaError_t allow_smem_fn(const void *fn, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mu);
    int i = 0;
    for (; i < g_smem_n; ++i)
        if (g_smem[i].fn == fn && g_smem[i].dev == dev) break;
    if (i < g_smem_n && g_smem[i].bytes >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (i == g_smem_n) {
        if (g_smem_n < 256) g_smem[g_smem_n++] = {fn, dev, bytes};   // else set, just not remembered
    } else {
        g_smem[i].bytes = bytes;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------

cudaError_t launch_update(const Geo &G, uint32_t *cube, const uint32_t *pairs, size_t n, uint32_t blocks_per_sm,
                          cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    constexpr int U = 2;
    const uint64_t n2 = n / 2 + 1;
    uint64_t want = (n2 + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms() * (blocks_per_sm ? blocks_per_sm : 8);   // 256-thread blocks per SM
    const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    if (G.n_ra == 3 && G.n_va == 1)
        k_update<3, 1, U><<<blocks, 256, 0, s>>>(G, cube, pairs, n);
    else
        k_update<0, 0, U><<<blocks, 256, 0, s>>>(G, cube, pairs, n);
    return cudaGetLastError();
}

cudaError_t launch_merge(uint32_t *dst, const uint32_t *const *srcs, int k, uint64_t words, cudaStream_t s,
                         bool assign) {
    const uint64_t n16 = words / 4;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    uint64_t want = (n16 + 255) / 256;
    const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    for (int k0 = 0; k0 < k; k0 += kMaxSrc) {
        SrcList L;
        L.k = (k - k0) < kMaxSrc ? (k - k0) : kMaxSrc;
        for (int j = 0; j < L.k; ++j) L.p[j] = reinterpret_cast<const uint4 *>(srcs[k0 + j]);
        k_merge<<<blocks, 256, 0, s>>>(reinterpret_cast<uint4 *>(dst), L, n16, assign && k0 == 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Zero counts for columns of at most 16 pieces of 16 bytes (g <= 2048):
// TPC = W/4 lanes share a column, one piece each, so a warp's load covers
// 32/TPC whole columns, 512 contiguous bytes (full 128-byte lines: four L1
// wavefronts, where pieces strided over sixteen columns take sixteen).  Each
// lane keeps U = max(8, TPC) loads in flight, then a butterfly over the TPC lanes of a
// column (log2 TPC exchange steps, U/2 + U/4 + ... shuffles) leaves each lane
// the totals of U/TPC columns: value i of lane l is load u = i + (U/TPC)(l mod
// TPC), column group l/TPC of that load.
template <uint32_t TPC>
__global__ void __launch_bounds__(256) k_zero_counts_lines(const Geo G, const uint32_t *__restrict__ cube,
                                                           uint16_t *__restrict__ zc,
                                                           unsigned long long *__restrict__ za, uint32_t splits,
                                                           uint32_t arr0, uint32_t *__restrict__ done, double E,
                                                           double *__restrict__ eps_out,
                                                           int64_t *__restrict__ zmax_out, uint32_t cs_lo,
                                                           uint32_t cs_hi) {
    constexpr uint32_t U = TPC > 8 ? TPC : 8;        // loads in flight (at least the lanes of a column)
    constexpr uint32_t CPL = 32 / TPC;               // columns per warp load
    const uint32_t arr = arr0 + blockIdx.x;          // cs*A + a
    const uint32_t cs = arr / G.A, a = arr % G.A;
    const uint32_t ncol = 1u << G.cbn[a];
    const uint32_t c0 = (uint32_t)(((uint64_t)ncol * blockIdx.y) / splits);
    const uint32_t c1 = (uint32_t)(((uint64_t)ncol * (blockIdx.y + 1)) / splits);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint4 *arr4 = reinterpret_cast<const uint4 *>(cube + (size_t)cs * G.cs_words + G.arr_base[a]);
    unsigned long long acc = 0;
    for (uint32_t base = c0 + warp * U * CPL; base < c1; base += nwarps * U * CPL) {
        uint32_t x[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t col = base + u * CPL + lane / TPC;
            x[u] = 0;
            if (col < c1) {
                const uint4 v = __ldcg(arr4 + (size_t)col * TPC + (lane % TPC));
                x[u] = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
        }
#pragma unroll
        for (uint32_t o = TPC / 2, V = U; o > 0; o >>= 1, V >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (uint32_t i = 0; i < V / 2; ++i) {
                const uint32_t send = up ? x[i] : x[i + V / 2];
                const uint32_t keep = up ? x[i + V / 2] : x[i];
                x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
#pragma unroll
        for (uint32_t i = 0; i < U / TPC; ++i) {
            const uint32_t u = i + (U / TPC) * (lane % TPC);
            const uint32_t col = base + u * CPL + lane / TPC;
            if (col < c1) {
                const uint32_t zeros = G.g - x[i];
                if (zc) zc[(size_t)arr * G.cmax + col] = (uint16_t)zeros;
                acc += zeros;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ unsigned long long part[8];
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (uint32_t w = 0; w < nwarps; ++w) t += part[w];
        atomicAdd(&za[arr], t);
        s_last = false;
        if (done) {
            __threadfence();
            s_last = atomicAdd(done, 1u) == gridDim.x * gridDim.y - 1;
        }
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (uint32_t c = cs_lo + threadIdx.x; c < cs_hi; c += blockDim.x) eps_zmax_of(G, za, E, c, eps_out, zmax_out);
    }
}

cudaError_t launch_column_stats(const Geo &G, const uint32_t *cube, uint16_t *zc, uint64_t *za,
                                double *eps, int64_t *zmax, double E, cudaStream_t s, uint32_t cs_lo,
                                uint32_t cs_hi, uint32_t *done, bool za_zeroed) {
    if (cs_hi == 0) cs_hi = G.smask + 1;
    cudaError_t e = cudaSuccess;
    if (!za_zeroed && (e = cudaMemsetAsync(za, 0, sizeof(uint64_t) * (size_t)(G.smask + 1) * G.A, s)) != cudaSuccess)
        return e;
    if (cs_lo >= cs_hi) return cudaSuccess;
    const uint32_t arrays = (cs_hi - cs_lo) * G.A;
    // Enough blocks to cover every SM several times; each slice is whole columns.
    uint32_t splits = 1;
    while ((uint64_t)arrays * splits < (uint64_t)num_sms() * 8 && splits < 64) splits <<= 1;
    const uint32_t min_cols = 1u << 5;   // cbn >= 5 for every array
    if (splits > min_cols) splits = min_cols;
    const bool fused = done && (eps || zmax);
    auto *zap = reinterpret_cast<unsigned long long *>(za);
    uint32_t *dn = fused ? done : nullptr;
    const uint32_t pieces = G.W / 4;                 // 16-byte pieces per column
    if (pieces <= 16) {
        // whole lines per warp load; a slice per block of at least one pass of its 8 warps x U loads
        const uint32_t per_pass = 8 * (pieces > 8 ? pieces : 8) * (32 / pieces);
        // about two blocks per SM, each looping over its slice: fewer block ends (a fence and a shared
        // counter atomic each) and the next pass's loads issued while others reduce
        uint32_t sl = 1;
        while ((uint64_t)arrays * sl < (uint64_t)num_sms() * 2 && sl < splits && G.cmax / (2 * sl) >= per_pass)
            sl <<= 1;
        switch (pieces) {
            case 1: k_zero_counts_lines<1><<<dim3(arrays, sl), 256, 0, s>>>(G, cube, zc, zap, sl, cs_lo * G.A, dn, E,
                                                                            eps, zmax, cs_lo, cs_hi); break;
            case 2: k_zero_counts_lines<2><<<dim3(arrays, sl), 256, 0, s>>>(G, cube, zc, zap, sl, cs_lo * G.A, dn, E,
                                                                            eps, zmax, cs_lo, cs_hi); break;
            case 4: k_zero_counts_lines<4><<<dim3(arrays, sl), 256, 0, s>>>(G, cube, zc, zap, sl, cs_lo * G.A, dn, E,
                                                                            eps, zmax, cs_lo, cs_hi); break;
            case 8: k_zero_counts_lines<8><<<dim3(arrays, sl), 256, 0, s>>>(G, cube, zc, zap, sl, cs_lo * G.A, dn, E,
                                                                            eps, zmax, cs_lo, cs_hi); break;
            default: k_zero_counts_lines<16><<<dim3(arrays, sl), 256, 0, s>>>(G, cube, zc, zap, sl, cs_lo * G.A, dn,
                                                                              E, eps, zmax, cs_lo, cs_hi); break;
        }
    } else {
        k_zero_counts<<<dim3(arrays, splits), 256, 0, s>>>(G, cube, zc, zap, splits, cs_lo * G.A, dn, E, eps, zmax,
                                                           cs_lo, cs_hi);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((eps || zmax) && !fused) {
        const uint32_t S = cs_hi - cs_lo;
        k_eps_zmax<<<(S + 127) / 128, 128, 0, s>>>(G, reinterpret_cast<const unsigned long long *>(za), E, eps, zmax,
                                                   cs_lo, cs_hi);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace cbaa
