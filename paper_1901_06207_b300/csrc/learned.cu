// Learned cardinality correction: per-address features read from the cube,
// and a 16-64-64-1 MLP (BF16 weights, FP32 activations and accumulation)
// with forward, gradient and Adam kernels.
//
// The paper estimates with Thm. 2 only.  When a cube is undersized its
// arrays saturate and the union column of a host shares many bits with
// others; the network maps what the cube shows about an address (zero bits
// of each of its columns and of their AND, the zero fraction of each array
// of its sketch, eps, the Thm. 2 estimate) to a correction of ln(1 + Thm. 2
// estimate) towards ln(1 + cardinality).  The plain estimate stays the
// fallback wherever the network's output is not a finite number.
#include <cuda_bf16.h>

#include "cbaa_internal.cuh"
#include "learned.h"

namespace cbaa {

namespace {

constexpr int IN = CBAA_MLP_IN, HID = CBAA_MLP_HIDDEN;
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + HID, NPAR = OB3 + 1;
static_assert(NPAR == CBAA_MLP_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// Features: one warp per address.  Lane l holds words l, l+32, ... of each
// of the address's |RA|+|VA| columns (Alg. 1's column indices).
__global__ void __launch_bounds__(256) k_features(const Geo G, const uint32_t *__restrict__ cube,
                                                  const unsigned long long *__restrict__ za,
                                                  const double *__restrict__ eps_cs,
                                                  const uint32_t *__restrict__ ips, uint64_t n,
                                                  float *__restrict__ feats) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t k = warp; k < n; k += nw) {
        const uint32_t m = mangle(G, ips[k]);
        const uint32_t cs = m & G.smask, lp = m >> G.r;
        uint32_t cols[CBAA_MAX_ARRAYS];
        for (uint32_t i = 0; i < G.n_ra; ++i) cols[i] = ra_col(G, i, lp);
        for (uint32_t j = 0; j < G.n_va; ++j) cols[G.n_ra + j] = va_col(G, j, lp);
        uint32_t ones[CBAA_MAX_ARRAYS] = {0};
        uint32_t uones = 0;
        for (uint32_t w = lane; w < G.W; w += 32) {
            uint32_t acc = 0xFFFFFFFFu;
            for (uint32_t a = 0; a < G.A; ++a) {
                const uint32_t v = cube[col_word0(G, cs, a, cols[a]) + w];
                ones[a] += __popc(v);
                acc &= v;
            }
            uones += __popc(acc);
        }
        for (uint32_t a = 0; a < G.A; ++a) ones[a] = __reduce_add_sync(0xffffffffu, ones[a]);
        uones = __reduce_add_sync(0xffffffffu, uones);
        if (lane == 0) {
            const float g = (float)G.g;
            float f[IN];
            for (int i = 0; i < IN; ++i) f[i] = 0.f;
            const uint32_t A4 = G.A < 4 ? G.A : 4;
            float zmin = 1.f;
            for (uint32_t a = 0; a < A4; ++a) {
                const float z = (float)(G.g - ones[a]) / g;
                f[a] = z;
                zmin = fminf(zmin, z);
                const double bits = (double)((unsigned long long)(1u << G.cbn[a]) << G.log2_g);
                f[5 + a] = (float)((double)za[(size_t)cs * G.A + a] / bits);
            }
            const uint32_t zu = G.g - uones;
            const double e = eps_cs[cs];
            f[4] = (float)zu / g;
            f[9] = (float)e;
            const double den = (double)G.g - (double)G.g * e;
            double est = -(double)G.g * log((double)(zu ? zu : 1u) / den);
            if (est < 0.0) est = 0.0;
            f[10] = (float)(est / (double)G.g);
            f[11] = (float)log1p(est) / 10.f;
            f[12] = zu ? 0.f : 1.f;
            f[13] = zmin;
            // Columns of a real host share its own bits, so their AND keeps far more ones than
            // independent columns would; a phantom's columns are unrelated.  f14 is that gap,
            // ln(ones fraction of the union) - sum_a ln(ones fraction of column a).
            const float floor1 = 1.f / g;
            const float lu = logf(fmaxf(1.f - f[4], floor1));
            float lsum = 0.f;
            for (uint32_t a = 0; a < G.A; ++a) lsum += logf(fmaxf((float)ones[a] / g, floor1));
            f[14] = lu - lsum;
            f[15] = lu;
            float4 *o = reinterpret_cast<float4 *>(feats + k * IN);
            for (int q = 0; q < IN / 4; ++q) o[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        }
    }
}

__device__ __forceinline__ void load_weights(const __nv_bfloat16 *__restrict__ Wb, float *w) {
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) w[i] = __bfloat162float(Wb[i]);
}

__device__ __forceinline__ void load_x(const float *__restrict__ X, uint64_t s, float (&x)[IN]) {
    const float4 *p = reinterpret_cast<const float4 *>(X + s * IN);
#pragma unroll
    for (int q = 0; q < IN / 4; ++q) {
        const float4 v = p[q];
        x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
    }
}

// y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, one thread per sample (no
// loop over samples, so the weights stay in shared memory instead of being
// hoisted into registers).
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16 *__restrict__ Wb,
                                                     const float *__restrict__ X, uint64_t n,
                                                     float *__restrict__ Y) {
    __shared__ float w[NPAR];
    load_weights(Wb, w);
    __syncthreads();
    const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[IN];
    load_x(X, s, x);
    float h1[HID];
#pragma unroll
    for (int i = 0; i < HID; ++i) {
        float a = w[OB1 + i];
#pragma unroll
        for (int j = 0; j < IN; ++j) a = fmaf(w[OW1 + i * IN + j], x[j], a);
        h1[i] = fmaxf(a, 0.f);
    }
    float y = w[OB3];
#pragma unroll 1
    for (int i = 0; i < HID; ++i) {
        float a = w[OB2 + i];
#pragma unroll
        for (int j = 0; j < HID; ++j) a = fmaf(w[OW2 + i * HID + j], h1[j], a);
        y = fmaf(w[OW3 + i], fmaxf(a, 0.f), y);
    }
    Y[s] = y;
}

// Gradient of sum_s (y_s - t_s)^2 * scale over all n samples, accumulated into
// grad (FP32, parameter layout) and loss_sum.  Blocks of TB threads walk
// tiles of TILE samples: the PARTS threads of a sample each take HID/PARTS
// hidden units through the forward and backward passes, with activations
// and deltas in shared memory as [feature][sample] rows padded to TILE+1
// floats (conflict-free in both the per-sample passes and the per-weight
// reductions); then every thread accumulates its share of the weight
// gradients over the tile's samples in registers, and adds them to `grad`
// once at the end.  Small tiles spread a batch over many SMs (a 4096-sample
// batch fills 128 blocks of eight warps).
constexpr int TB = 256;
constexpr int TILE = 32;
constexpr int PARTS = TB / TILE;
constexpr int HP = HID / PARTS;
constexpr int LD = TILE + 1;
constexpr int R2 = HID * HID / TB;     // W2 rows of one column a thread accumulates
constexpr int R1 = HID * IN / TB;      // W1 rows of one column a thread accumulates
static_assert(TB % TILE == 0 && HID % PARTS == 0 && TB % HID == 0 && TB % IN == 0 && TB > HID, "tile split");

__global__ void __launch_bounds__(TB) k_mlp_grad(const __nv_bfloat16 *__restrict__ Wb, const float *__restrict__ X,
                                                 const float *__restrict__ Tgt, uint64_t n, float scale,
                                                 float *__restrict__ grad, float *__restrict__ loss_sum) {
    extern __shared__ float sm[];
    float *w = sm;                         // NPAR
    float *H1 = w + ((NPAR + 3) & ~3);     // HID x LD
    float *H2 = H1 + HID * LD;
    float *D1 = H2 + HID * LD;
    float *D2 = D1 + HID * LD;
    float *Xs = D2 + HID * LD;             // IN x LD
    float *Yp = Xs + IN * LD;              // PARTS x LD: each part's share of the output
    float *D3 = Yp + PARTS * LD;           // LD
    load_weights(Wb, w);
    const int k = threadIdx.x;
    const int sl = k % TILE, i0 = (k / TILE) * HP;   // this thread's sample in the tile, first hidden unit
    // register accumulators: W2 rows ib2*R2.. of column j2, W1 rows ib1*R1.. of column j1
    const int j2 = k % HID, ib2 = k / HID, j1 = k % IN, ib1 = k / IN;
    float g2[R2], g1[R1];
#pragma unroll
    for (int q = 0; q < R2; ++q) g2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < R1; ++q) g1[q] = 0.f;
    float gw3 = 0.f, gb2 = 0.f, gb1 = 0.f, gb3 = 0.f, lsum = 0.f;
    __syncthreads();
    const uint64_t tiles = (n + TILE - 1) / TILE;
    for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint64_t s = tile * TILE + sl;
        const bool valid = s < n;
        float x[IN];
        if (valid) {
            load_x(X, s, x);
        } else {
#pragma unroll
            for (int j = 0; j < IN; ++j) x[j] = 0.f;
        }
        if (i0 == 0) {
#pragma unroll
            for (int j = 0; j < IN; ++j) Xs[j * LD + sl] = x[j];
        }
        for (int i = i0; i < i0 + HP; ++i) {
            float a = w[OB1 + i];
#pragma unroll
            for (int j = 0; j < IN; ++j) a = fmaf(w[OW1 + i * IN + j], x[j], a);
            H1[i * LD + sl] = fmaxf(a, 0.f);
        }
        __syncthreads();                                   // H1 of the tile complete
        float yp = 0.f;
        for (int i = i0; i < i0 + HP; ++i) {
            float a = w[OB2 + i];
            for (int j = 0; j < HID; ++j) a = fmaf(w[OW2 + i * HID + j], H1[j * LD + sl], a);
            const float h = fmaxf(a, 0.f);
            H2[i * LD + sl] = h;
            yp = fmaf(w[OW3 + i], h, yp);
        }
        Yp[(i0 / HP) * LD + sl] = yp;
        __syncthreads();                                   // every part's share of y complete
        float y = w[OB3];
#pragma unroll
        for (int p = 0; p < PARTS; ++p) y += Yp[p * LD + sl];
        const float r = valid ? (y - Tgt[s]) : 0.f;
        const float d3 = 2.f * r * scale;
        if (i0 == 0) {
            lsum = fmaf(r, r, lsum);
            D3[sl] = d3;
        }
        for (int i = i0; i < i0 + HP; ++i) D2[i * LD + sl] = (H2[i * LD + sl] > 0.f) ? d3 * w[OW3 + i] : 0.f;
        __syncthreads();                                   // D2 complete
        for (int j = i0; j < i0 + HP; ++j) {
            float a = 0.f;
            for (int i = 0; i < HID; ++i) a = fmaf(D2[i * LD + sl], w[OW2 + i * HID + j], a);
            D1[j * LD + sl] = (H1[j * LD + sl] > 0.f) ? a : 0.f;
        }
        __syncthreads();                                   // D1, D3 and Xs complete
        for (int t = 0; t < TILE; ++t) {
            const float h1 = H1[j2 * LD + t];
#pragma unroll
            for (int q = 0; q < R2; ++q) g2[q] = fmaf(D2[(ib2 * R2 + q) * LD + t], h1, g2[q]);
            const float xv = Xs[j1 * LD + t];
#pragma unroll
            for (int q = 0; q < R1; ++q) g1[q] = fmaf(D1[(ib1 * R1 + q) * LD + t], xv, g1[q]);
            if (k < HID) {
                gw3 = fmaf(D3[t], H2[k * LD + t], gw3);
                gb2 += D2[k * LD + t];
                gb1 += D1[k * LD + t];
            } else if (k == HID) {
                gb3 += D3[t];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < R2; ++q) atomicAdd(&grad[OW2 + (ib2 * R2 + q) * HID + j2], g2[q]);
#pragma unroll
    for (int q = 0; q < R1; ++q) atomicAdd(&grad[OW1 + (ib1 * R1 + q) * IN + j1], g1[q]);
    if (k < HID) {
        atomicAdd(&grad[OW3 + k], gw3);
        atomicAdd(&grad[OB2 + k], gb2);
        atomicAdd(&grad[OB1 + k], gb1);
    } else if (k == HID) {
        atomicAdd(&grad[OB3], gb3);
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((k & 31) == 0 && lsum != 0.f) atomicAdd(loss_sum, lsum);
}

// Adam on FP32 master weights; the BF16 copy the kernels read is rounded
// to nearest even from the updated master.
__global__ void k_adam(float *__restrict__ master, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ Wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = p;
    Wb[i] = __float2bfloat16_rn(p);
}

__global__ void k_to_bf16(const float *__restrict__ master, __nv_bfloat16 *__restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPAR) Wb[i] = __float2bfloat16_rn(master[i]);
}

// Learned decision with the plain estimate as fallback.  The network
// predicts a correction in log space: card = exp(ln(1 + est) + y) - 1 with
// est the Thm. 2 estimate (ln(1 + est) is feature 11 times 10); where y is
// not finite the Thm. 2 estimate itself is used.
__global__ void k_decide(const float *__restrict__ y, const float *__restrict__ feats, uint64_t n, float g,
                         float theta, float *__restrict__ card, uint8_t *__restrict__ decision) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const float yv = y[s];
        const float plain = feats[s * IN + 10] * g;
        const float c = isfinite(yv) ? expm1f(fminf(10.f * feats[s * IN + 11] + yv, 30.f)) : plain;
        card[s] = c;
        decision[s] = c >= theta ? 1 : 0;
    }
}

// Training target of one sample: ln(1 + exact cardinality) - ln(1 + Thm. 2
// estimate), the latter as the features carry it (feature 11 = ln(1 + est)/10).
__global__ void k_target(const float *__restrict__ feats, const float *__restrict__ count, uint64_t n,
                         float *__restrict__ t) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride)
        t[s] = log1pf(count[s]) - 10.f * feats[s * IN + 11];
}

}  // namespace

cudaError_t launch_target(const float *feats, const float *count, uint64_t n, float *t, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    k_target<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(feats, count, n, t);
    return cudaGetLastError();
}

cudaError_t launch_features(const Geo &G, const uint32_t *cube, const uint64_t *za, const double *eps,
                            const uint32_t *ips, uint64_t n, float *feats, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n * 32 + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms() * 16;
    k_features<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(
        G, cube, reinterpret_cast<const unsigned long long *>(za), eps, ips, n, feats);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const uint16_t *Wb, const float *X, uint64_t n, float *Y, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    k_mlp_forward<<<(unsigned)blocks, 256, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(Wb), X, n, Y);
    return cudaGetLastError();
}

size_t mlp_grad_smem() {
    return sizeof(float) * ((size_t)((NPAR + 3) & ~3) + (size_t)(4 * HID + IN + PARTS + 1) * LD);
}

cudaError_t launch_mlp_grad(const uint16_t *Wb, const float *X, const float *T, uint64_t n, float scale,
                            float *grad, float *loss, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const size_t smem = mlp_grad_smem();
    cudaError_t e = allow_smem(k_mlp_grad, smem);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = (n + TILE - 1) / TILE;
    const uint64_t cap = (uint64_t)num_sms();
    k_mlp_grad<<<(unsigned)(tiles < cap ? tiles : cap), TB, smem, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(Wb), X, T, n, scale, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *master, const float *grad, float *m, float *v, uint16_t *Wb, float lr, float b1,
                        float b2, float eps, uint32_t step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NPAR + 255) / 256, 256, 0, s>>>(master, grad, m, v, reinterpret_cast<__nv_bfloat16 *>(Wb), lr, b1, b2,
                                              eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *master, uint16_t *Wb, cudaStream_t s) {
    k_to_bf16<<<(NPAR + 255) / 256, 256, 0, s>>>(master, reinterpret_cast<__nv_bfloat16 *>(Wb));
    return cudaGetLastError();
}

cudaError_t launch_decide(const float *y, const float *feats, uint64_t n, float g, float theta, float *card,
                          uint8_t *decision, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n + 255) / 256;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    k_decide<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(y, feats, n, g, theta, card, decision);
    return cudaGetLastError();
}

}  // namespace cbaa
