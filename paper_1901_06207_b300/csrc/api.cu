// C ABI of libcbaa.so: argument checks, geometry derivation, launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "cbaa_internal.cuh"
#include "detect_layout.h"
#include "update_binned.h"
#include "learned.h"

struct cbaa_cube {
    cbaa_params p;
    cbaa::Geo G;
    uint32_t *data;
    size_t bytes;
};

namespace cbaa {

Geo make_geo(const cbaa_params &p) {
    Geo G;
    std::memset(&G, 0, sizeof G);
    G.r = p.r;
    G.L = 32u - p.r;
    G.smask = (1u << p.r) - 1u;
    G.n_ra = p.n_ra;
    G.n_va = p.n_va;
    G.A = p.n_ra + p.n_va;
    G.log2_g = p.log2_g;
    G.g = 1u << p.log2_g;
    G.W = G.g / 32u;
    G.form = p.threshold_form;
    G.seed_m = p.seed_mangle;
    G.seed_bv = p.seed_bv;
    uint32_t base = 0;
    for (uint32_t a = 0; a < G.A; ++a) {
        G.cbn[a] = p.cbn[a];
        G.arr_base[a] = base;
        base += (1u << p.cbn[a]) * G.W;
        if ((1u << p.cbn[a]) > G.cmax) G.cmax = 1u << p.cbn[a];
    }
    G.arr_base[G.A] = base;
    for (uint32_t a = 0; a <= G.A; ++a) G.col_base[a] = G.arr_base[a] / G.W;
    G.cs_words = base;
    G.cube_words = (uint64_t)base << p.r;
    for (uint32_t i = 0; i < G.n_ra; ++i) {
        G.ring_off[i] = p.ring_off[i];
        G.ep[i] = (p.ring_off[(i + 1) % G.n_ra] + G.L - p.ring_off[i]) % G.L;
        G.cp[i] = p.cbn[i] - G.ep[i];
    }
    for (uint32_t j = 0; j < G.n_va; ++j) G.seed_va[j] = p.seed_va[j];
    return G;
}

}  // namespace cbaa

using cbaa::Geo;
using cbaa::cuda_status;

namespace {

int validate(const cbaa_params *p) {
    if (!p) return CBAA_ERR_INVALID_ARG;
    if (p->r < 1 || p->r > 16) return CBAA_ERR_INVALID_ARG;
    if (p->n_ra < 2 || p->n_ra > CBAA_MAX_RA) return CBAA_ERR_INVALID_ARG;
    if (p->n_ra + p->n_va > CBAA_MAX_ARRAYS) return CBAA_ERR_INVALID_ARG;
    if (p->log2_g < 7 || p->log2_g > 15) return CBAA_ERR_INVALID_ARG;
    if (p->threshold_form > 1) return CBAA_ERR_INVALID_ARG;
    const uint32_t L = 32u - p->r, A = p->n_ra + p->n_va;
    for (uint32_t a = 0; a < A; ++a) {
        if (p->cbn[a] < 5 || p->cbn[a] > 16) return CBAA_ERR_INVALID_ARG;
        if (a < p->n_ra && p->cbn[a] > L) return CBAA_ERR_INVALID_ARG;
    }
    if (p->ring_off[0] != 0) return CBAA_ERR_INVALID_ARG;
    for (uint32_t i = 1; i < p->n_ra; ++i)
        if (p->ring_off[i] <= p->ring_off[i - 1]) return CBAA_ERR_INVALID_ARG;
    if (p->ring_off[p->n_ra - 1] >= L) return CBAA_ERR_INVALID_ARG;
    uint32_t ep[CBAA_MAX_RA];
    for (uint32_t i = 0; i < p->n_ra; ++i) ep[i] = (p->ring_off[(i + 1) % p->n_ra] + L - p->ring_off[i]) % L;
    for (uint32_t i = 0; i < p->n_ra; ++i) {
        if (p->cbn[i] < ep[i]) return CBAA_ERR_INVALID_ARG;                          // |CP(i)| >= 0
        if (p->cbn[i] - ep[i] > ep[(i + 1) % p->n_ra]) return CBAA_ERR_INVALID_ARG;  // CP(i) inside EP(i+1)
    }
    uint64_t cs_words = 0;
    for (uint32_t a = 0; a < A; ++a) cs_words += (uint64_t)(1u << p->cbn[a]) << (p->log2_g - 5);
    if ((cs_words << p->r) >= (1ull << 32)) return CBAA_ERR_INVALID_ARG;   // 32-bit word offsets
    return CBAA_OK;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

thread_local cudaError_t t_last_cuda = cudaSuccess;

cbaa_tuning g_tuning = {};
std::mutex g_tuning_mu;

cbaa_tuning current_tuning() {
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning;
}

}  // namespace

int cbaa::cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CBAA_OK;
    t_last_cuda = e;
    return CBAA_ERR_CUDA;
}

extern "C" {

const char *cbaa_status_str(int status) {
    switch (status) {
        case CBAA_OK: return "ok";
        case CBAA_ERR_INVALID_ARG: return "invalid argument";
        case CBAA_ERR_GEOMETRY: return "geometry mismatch";
        case CBAA_ERR_CAPACITY: return "output capacity exceeded";
        case CBAA_ERR_WORKSPACE: return "workspace too small";
        case CBAA_ERR_CUDA: return "CUDA error";
        case CBAA_ERR_TIMEOUT: return "device wait timed out";
        case CBAA_ERR_NO_DEVICE: return "no CUDA device";
        default: return "unknown status";
    }
}

int cbaa_params_validate(const cbaa_params *p) { return validate(p); }

const char *cbaa_last_cuda_error(void) { return cudaGetErrorName(t_last_cuda); }

size_t cbaa_cube_bytes(const cbaa_params *p) {
    if (validate(p) != CBAA_OK) return 0;
    return (size_t)cbaa::make_geo(*p).cube_words * 4u;
}

size_t cbaa_detect_workspace_bytes(const cbaa_params *p, size_t max_candidates) {
    if (validate(p) != CBAA_OK || max_candidates == 0 || max_candidates > (1ull << 31)) return 0;
    return cbaa::ws_layout(cbaa::make_geo(*p), max_candidates).total;
}

int cbaa_cube_init(const cbaa_params *p, void *dev_mem, size_t bytes, cbaa_cube **out, void *stream) {
    if (!out) return CBAA_ERR_INVALID_ARG;
    *out = nullptr;
    int st = validate(p);
    if (st != CBAA_OK) return st;
    const Geo G = cbaa::make_geo(*p);
    if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 15u) || bytes < G.cube_words * 4u)
        return CBAA_ERR_INVALID_ARG;
    cbaa_cube *c = new (std::nothrow) cbaa_cube;
    if (!c) return CBAA_ERR_INVALID_ARG;
    c->p = *p;
    c->G = G;
    c->data = static_cast<uint32_t *>(dev_mem);
    c->bytes = G.cube_words * 4u;
    const int st_mem = cuda_status(cudaMemsetAsync(c->data, 0, c->bytes, as_stream(stream)));
    if (st_mem != CBAA_OK) {
        delete c;
        return st_mem;
    }
    *out = c;
    return CBAA_OK;
}

int cbaa_cube_destroy(cbaa_cube *cube) {
    delete cube;
    return CBAA_OK;
}

void *cbaa_cube_data(const cbaa_cube *cube) { return cube ? cube->data : nullptr; }

int cbaa_cube_params(const cbaa_cube *cube, cbaa_params *out) {
    if (!cube || !out) return CBAA_ERR_INVALID_ARG;
    *out = cube->p;
    return CBAA_OK;
}

int cbaa_cube_reset(cbaa_cube *cube, void *stream) {
    if (!cube) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cudaMemsetAsync(cube->data, 0, cube->bytes, as_stream(stream)));
}

int cbaa_cube_set_inner_net(cbaa_cube *cube, const cbaa_inner_net *net) {
    if (!cube) return CBAA_ERR_INVALID_ARG;
    const uint32_t k = net ? net->n : 0u;
    if (k > CBAA_MAX_INNER) return CBAA_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < k; ++i)
        if (net->len[i] > 32) return CBAA_ERR_INVALID_ARG;
    cbaa::Geo &G = cube->G;
    G.n_inner = k;
    for (uint32_t i = 0; i < CBAA_MAX_INNER; ++i) {
        const uint32_t mask = (i < k && net->len[i]) ? ~0u << (32 - net->len[i]) : 0u;
        G.inner_mask[i] = mask;
        G.inner_net[i] = i < k ? (net->addr[i] & mask) : 0u;
    }
    return CBAA_OK;
}

int cbaa_cube_update(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *stream) {
    if (!cube) return CBAA_ERR_INVALID_ARG;
    if (n == 0) return CBAA_OK;
    if (!dev_pairs || (reinterpret_cast<uintptr_t>(dev_pairs) & 7u)) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_update(cube->G, cube->data, dev_pairs, n, current_tuning().direct_blocks_per_sm,
                               as_stream(stream)));
}

size_t cbaa_update_workspace_bytes(const cbaa_params *p, size_t max_pairs) {
    return cbaa_update_multi_workspace_bytes(p, 1, max_pairs);
}

size_t cbaa_update_multi_workspace_bytes(const cbaa_params *p, int n_cubes, size_t max_pairs) {
    if (validate(p) != CBAA_OK || max_pairs == 0 || n_cubes < 1 || n_cubes > (int)cbaa::kMaxRouters) return 0;
    const Geo G = cbaa::make_geo(*p);
    if ((uint64_t)n_cubes * cbaa::tiles_per_cube(G) > cbaa::kMaxBins) return 0;
    return cbaa::bin_ws_bytes(G, (uint32_t)n_cubes, max_pairs);
}

}  // extern "C"

namespace {

// cbaa_cube_update_multi, and with `global` set cbaa_cube_update_multi_merge.
// assign (one cube only): the cube's words become the pass's bits alone.
int update_multi(cbaa_cube *const *cubes, int n_cubes, const uint32_t *const *dev_pairs, const size_t *n,
                 cbaa_cube *global, void *dev_ws, size_t ws_bytes, void *stream, bool assign = false) {
    if (!cubes || !dev_pairs || !n || n_cubes < 1 || n_cubes > (int)cbaa::kMaxRouters) return CBAA_ERR_INVALID_ARG;
    if (!dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 15u)) return CBAA_ERR_INVALID_ARG;
    const cbaa_cube *c0 = cubes[0];
    if (!c0) return CBAA_ERR_INVALID_ARG;
    const Geo &G = c0->G;
    const uint32_t tpc = cbaa::tiles_per_cube(G);
    if ((uint64_t)n_cubes * tpc > cbaa::kMaxBins) return CBAA_ERR_INVALID_ARG;
    cbaa::BinSegs S;
    std::memset(&S, 0, sizeof S);
    S.n_routers = (uint32_t)n_cubes;
    S.tiles_per_seg = tpc;
    S.seg_words = tpc << cbaa::kBinTileBits;
    uint64_t total = 0;
    for (int j = 0; j < n_cubes; ++j) {
        const cbaa_cube *c = cubes[j];
        if (!c) return CBAA_ERR_INVALID_ARG;
        if (std::memcmp(&c->p, &c0->p, sizeof(cbaa_params)) != 0) return CBAA_ERR_GEOMETRY;
        if (c->G.n_inner != G.n_inner ||
            std::memcmp(c->G.inner_net, G.inner_net, sizeof G.inner_net) != 0 ||
            std::memcmp(c->G.inner_mask, G.inner_mask, sizeof G.inner_mask) != 0)
            return CBAA_ERR_INVALID_ARG;                 // one NI for all cubes of a pass
        for (int i = 0; i < j; ++i)
            if (cubes[i] == c) return CBAA_ERR_INVALID_ARG;
        S.cube[j] = c->data;
        if (n[j] == 0) continue;
        if (!dev_pairs[j] || (reinterpret_cast<uintptr_t>(dev_pairs[j]) & 7u)) return CBAA_ERR_INVALID_ARG;
        S.pairs[S.k] = dev_pairs[j];
        S.start[S.k] = total;
        S.router[S.k] = (uint32_t)j;
        ++S.k;
        total += n[j];
    }
    S.start[S.k] = total;
    if (global) {                                    // the global cube: same structure, not a router cube
        if (std::memcmp(&global->p, &c0->p, sizeof(cbaa_params)) != 0) return CBAA_ERR_GEOMETRY;
        for (int j = 0; j < n_cubes; ++j)
            if (cubes[j] == global) return CBAA_ERR_INVALID_ARG;
        S.merge = global->data;
    }
    if (total == 0) return CBAA_OK;
    cbaa::BinWs W;
    if (!cbaa::bin_ws_make(G, (uint32_t)n_cubes, dev_ws, ws_bytes, &W)) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_update_segments(G, S, total, W, current_tuning(), as_stream(stream),
                                                    assign && n_cubes == 1));
}

}  // namespace

extern "C" {

int cbaa_cube_update_multi(cbaa_cube *const *cubes, int n_cubes, const uint32_t *const *dev_pairs, const size_t *n,
                           void *dev_ws, size_t ws_bytes, void *stream) {
    return update_multi(cubes, n_cubes, dev_pairs, n, nullptr, dev_ws, ws_bytes, stream);
}

int cbaa_cube_update_multi_merge(cbaa_cube *const *cubes, int n_cubes, const uint32_t *const *dev_pairs,
                                 const size_t *n, cbaa_cube *global, void *dev_ws, size_t ws_bytes, void *stream) {
    if (!global) return CBAA_ERR_INVALID_ARG;
    return update_multi(cubes, n_cubes, dev_pairs, n, global, dev_ws, ws_bytes, stream);
}

int cbaa_cube_update_binned(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *dev_ws, size_t ws_bytes,
                            void *stream) {
    if (!cube) return CBAA_ERR_INVALID_ARG;
    if (n == 0) return CBAA_OK;
    cbaa_cube *cubes[1] = {cube};
    const uint32_t *pp[1] = {dev_pairs};
    const size_t nn[1] = {n};
    return cbaa_cube_update_multi(cubes, 1, pp, nn, dev_ws, ws_bytes, stream);
}

int cbaa_cube_update_binned_assign(cbaa_cube *cube, const uint32_t *dev_pairs, size_t n, void *dev_ws,
                                   size_t ws_bytes, void *stream) {
    if (!cube) return CBAA_ERR_INVALID_ARG;
    if (n == 0) return cuda_status(cudaMemsetAsync(cube->data, 0, cube->bytes, as_stream(stream)));
    cbaa_cube *cubes[1] = {cube};
    const uint32_t *pp[1] = {dev_pairs};
    const size_t nn[1] = {n};
    return update_multi(cubes, 1, pp, nn, nullptr, dev_ws, ws_bytes, stream, true);
}

int cbaa_set_tuning(const cbaa_tuning *t) {
    if (!t || t->scatter_shape > 8 || t->count_blocks_per_sm > 64 || t->apply_items_per_sm > 1024 ||
        t->direct_blocks_per_sm > 64 || t->tile_kind > 3 || t->heavy > 3 || t->split_blocks > 4096)
        return CBAA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    g_tuning = *t;
    return CBAA_OK;
}

int cbaa_get_tuning(cbaa_tuning *t) {
    if (!t) return CBAA_ERR_INVALID_ARG;
    *t = current_tuning();
    return CBAA_OK;
}

}  // extern "C"

namespace {

// cbaa_cube_merge (assign false) and cbaa_cube_merge_assign.
int merge(cbaa_cube *dst, const cbaa_cube *const *srcs, int k, void *stream, bool assign) {
    if (!dst || k < 0 || (k > 0 && !srcs)) return CBAA_ERR_INVALID_ARG;
    if (k == 0) return assign ? cuda_status(cudaMemsetAsync(dst->data, 0, dst->bytes, as_stream(stream))) : CBAA_OK;
    for (int j = 0; j < k; ++j) {                 // every source checked before anything is enqueued
        const cbaa_cube *s = srcs[j];
        if (!s || s == dst) return CBAA_ERR_INVALID_ARG;
        if (std::memcmp(&s->p, &dst->p, sizeof(cbaa_params)) != 0) return CBAA_ERR_GEOMETRY;
    }
    const uint32_t *ptrs[64];
    for (int k0 = 0; k0 < k; k0 += 64) {
        const int kk = (k - k0) < 64 ? (k - k0) : 64;
        for (int j = 0; j < kk; ++j) ptrs[j] = srcs[k0 + j]->data;
        const int st = cuda_status(cbaa::launch_merge(dst->data, ptrs, kk, dst->G.cube_words, as_stream(stream),
                                                      assign && k0 == 0));
        if (st != CBAA_OK) return st;
    }
    return CBAA_OK;
}

}  // namespace

extern "C" {

int cbaa_cube_merge(cbaa_cube *dst, const cbaa_cube *const *srcs, int k, void *stream) {
    return merge(dst, srcs, k, stream, false);
}

int cbaa_cube_merge_assign(cbaa_cube *dst, const cbaa_cube *const *srcs, int k, void *stream) {
    return merge(dst, srcs, k, stream, true);
}

int cbaa_column_stats(const cbaa_cube *cube, uint32_t theta, uint16_t *dev_zc, uint64_t *dev_za, double *dev_eps,
                      int64_t *dev_zmax, void *stream) {
    if (!cube || !dev_za) return CBAA_ERR_INVALID_ARG;
    const double E = std::exp(-((double)theta / (double)cube->G.g));
    return cuda_status(cbaa::launch_column_stats(cube->G, cube->data, dev_zc, dev_za, dev_eps, dev_zmax, E, as_stream(stream)));
}

int cbaa_detect_async(const cbaa_cube *cube, uint32_t theta, void *dev_ws, size_t ws_bytes, cbaa_host *dev_out,
                      size_t cap, cbaa_detect_info *dev_info, void *stream) {
    if (!cube || !dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 15u) || !dev_info || (cap > 0 && !dev_out))
        return CBAA_ERR_INVALID_ARG;
    return cbaa::detect_enqueue(cube->G, cube->data, theta, dev_ws, ws_bytes, dev_out, cap, dev_info,
                                cbaa::num_sms(), as_stream(stream));
}

int cbaa_detect_range_async(const cbaa_cube *cube, uint32_t cs_lo, uint32_t cs_hi, uint32_t theta, void *dev_ws,
                            size_t ws_bytes, cbaa_host *dev_out, size_t cap, cbaa_detect_info *dev_info,
                            void *stream) {
    if (!cube || !dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 15u) || !dev_info || (cap > 0 && !dev_out))
        return CBAA_ERR_INVALID_ARG;
    if (cs_lo >= cs_hi || cs_hi > cube->G.smask + 1) return CBAA_ERR_INVALID_ARG;
    return cbaa::detect_enqueue(cube->G, cube->data, theta, dev_ws, ws_bytes, dev_out, cap, dev_info,
                                cbaa::num_sms(), as_stream(stream), cs_lo, cs_hi);
}

int cbaa_merge_hosts(const cbaa_host *dev_blocks, size_t block_cap, int k, const cbaa_detect_info *dev_infos,
                     cbaa_host *dev_out, size_t out_cap, cbaa_detect_info *dev_info_out, void *stream) {
    if (k < 1 || block_cap > 0xFFFFFFFFull || !dev_infos || !dev_info_out || (block_cap && !dev_blocks) ||
        (out_cap && !dev_out))
        return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_merge_hosts(dev_blocks, (uint32_t)block_cap, (uint32_t)k, dev_infos, dev_out,
                                                out_cap, dev_info_out, as_stream(stream)));
}

int cbaa_or_words(uint32_t *dst, const uint32_t *const *srcs, int k, size_t words, void *stream) {
    if (k < 0 || (k > 0 && words > 0 && (!dst || !srcs))) return CBAA_ERR_INVALID_ARG;
    if (k == 0 || words == 0) return CBAA_OK;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) || (words & 3u)) return CBAA_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
        if (!srcs[j] || srcs[j] == dst || (reinterpret_cast<uintptr_t>(srcs[j]) & 15u)) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_merge(dst, srcs, k, words, as_stream(stream)));
}

int cbaa_detect(const cbaa_cube *cube, uint32_t theta, void *dev_ws, size_t ws_bytes, cbaa_host *host_out, size_t cap,
                size_t *n_out, void *stream) {
    if (!cube || !dev_ws || (reinterpret_cast<uintptr_t>(dev_ws) & 15u) || !n_out || (cap > 0 && !host_out))
        return CBAA_ERR_INVALID_ARG;
    *n_out = 0;
    cudaStream_t s = as_stream(stream);
    cbaa::WsLayout Ly;
    if (!cbaa::ws_layout_fit(cube->G, ws_bytes, &Ly)) return CBAA_ERR_WORKSPACE;
    const cbaa::WsPtrs P = cbaa::ws_pointers(cube->G, Ly, dev_ws);
    int st = cbaa::detect_enqueue(cube->G, cube->data, theta, dev_ws, ws_bytes, nullptr, 0, nullptr,
                                  cbaa::num_sms(), s);
    if (st != CBAA_OK) return st;
    cbaa_detect_info info;
    if ((st = cuda_status(cudaMemcpyAsync(&info, &P.state->info, sizeof info, cudaMemcpyDeviceToHost, s))) != CBAA_OK)
        return st;
    if ((st = cuda_status(cudaStreamSynchronize(s))) != CBAA_OK) return st;
    if (info.status == CBAA_ERR_WORKSPACE) {
        *n_out = info.need_tuples;
        return CBAA_ERR_WORKSPACE;
    }
    *n_out = info.n_hosts;
    const size_t nw = info.n_hosts < cap ? info.n_hosts : cap;
    if (nw > 0) {
        if ((st = cuda_status(cudaMemcpyAsync(host_out, P.sorted, nw * sizeof(cbaa_host), cudaMemcpyDeviceToHost,
                                              s))) != CBAA_OK)
            return st;
        if ((st = cuda_status(cudaStreamSynchronize(s))) != CBAA_OK) return st;
    }
    return info.n_hosts > cap ? CBAA_ERR_CAPACITY : CBAA_OK;
}

int cbaa_host_features(const cbaa_cube *cube, const uint64_t *dev_za, const double *dev_eps,
                       const uint32_t *dev_ips, size_t n, float *dev_feats, void *stream) {
    if (!cube || !dev_za || !dev_eps || (n && (!dev_ips || !dev_feats)) ||
        (reinterpret_cast<uintptr_t>(dev_feats) & 15u))
        return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_features(cube->G, cube->data, dev_za, dev_eps, dev_ips, n, dev_feats,
                                             as_stream(stream)));
}

int cbaa_mlp_forward(const uint16_t *dev_w_bf16, const float *dev_x, size_t n, float *dev_y, void *stream) {
    if (!dev_w_bf16 || (n && (!dev_x || !dev_y)) || (reinterpret_cast<uintptr_t>(dev_x) & 15u))
        return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_mlp_forward(dev_w_bf16, dev_x, n, dev_y, as_stream(stream)));
}

int cbaa_mlp_grad(const uint16_t *dev_w_bf16, const float *dev_x, const float *dev_t, size_t n, float scale,
                  float *dev_grad, float *dev_loss, void *stream) {
    if (!dev_w_bf16 || !dev_grad || !dev_loss || (n && (!dev_x || !dev_t)) ||
        (reinterpret_cast<uintptr_t>(dev_x) & 15u))
        return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_mlp_grad(dev_w_bf16, dev_x, dev_t, n, scale, dev_grad, dev_loss,
                                             as_stream(stream)));
}

int cbaa_mlp_adam(float *dev_master, const float *dev_grad, float *dev_m, float *dev_v, uint16_t *dev_w_bf16,
                  float lr, float beta1, float beta2, float eps, uint32_t step, void *stream) {
    if (!dev_master || !dev_grad || !dev_m || !dev_v || !dev_w_bf16 || step == 0) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_adam(dev_master, dev_grad, dev_m, dev_v, dev_w_bf16, lr, beta1, beta2, eps, step,
                                         as_stream(stream)));
}

int cbaa_mlp_to_bf16(const float *dev_master, uint16_t *dev_w_bf16, void *stream) {
    if (!dev_master || !dev_w_bf16) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_to_bf16(dev_master, dev_w_bf16, as_stream(stream)));
}

int cbaa_learned_target(const float *dev_feats, const float *dev_count, size_t n, float *dev_t, void *stream) {
    if (n && (!dev_feats || !dev_count || !dev_t)) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_target(dev_feats, dev_count, n, dev_t, as_stream(stream)));
}

int cbaa_learned_decide(const float *dev_y, const float *dev_feats, size_t n, uint32_t log2_g, float theta,
                        float *dev_card, uint8_t *dev_decision, void *stream) {
    if ((n && (!dev_y || !dev_feats || !dev_card || !dev_decision)) || log2_g > 31) return CBAA_ERR_INVALID_ARG;
    return cuda_status(cbaa::launch_decide(dev_y, dev_feats, n, (float)(1u << log2_g), theta, dev_card,
                                           dev_decision, as_stream(stream)));
}

}  // extern "C"
