// Detect workspace layout (host arithmetic + the pointer bundle kernels get).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "cbaa_internal.cuh"

namespace cbaa {

// A partial or complete hot-column tuple <hc_0, ..., hc_{|RA|-1}> of one CS.
struct __align__(16) Tuple {
    uint16_t cs;
    uint16_t hc[7];
};
static_assert(sizeof(Tuple) == 16, "tuple is one 16-byte record");

struct DevState {
    cbaa_detect_info info;
    uint32_t stage_count[CBAA_MAX_RA];   // [0] = seed tuples (hot columns of RA 0), [s] = output of join stage s
    uint32_t stats_done;                 // zero-count blocks finished (the last computes eps and Zmax)
    uint32_t pad;
};

struct WsLayout {
    uint64_t m;                       // tuples / hosts per stage
    uint64_t keys_n;                  // sort keys (power of two >= m)
    size_t state, zc, za, eps, zmax, hc, nhc, boff, tup0, tup1, hosts, sorted, keys, total;
    uint32_t hc_stride, boff_stride;
};

struct WsPtrs {
    DevState *state;
    uint16_t *zc;
    uint64_t *za;
    double *eps;
    int64_t *zmax;
    uint16_t *hc;
    uint32_t *nhc;
    uint32_t *boff;
    Tuple *tup[2];
    cbaa_host *hosts;
    cbaa_host *sorted;
    unsigned long long *keys;
    uint32_t m, hc_stride, boff_stride;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline WsLayout ws_layout(const Geo &G, uint64_t m) {
    WsLayout L{};
    const size_t S = (size_t)G.smask + 1;
    uint32_t cmax_ra = 0, kb_max = 0;
    for (uint32_t i = 0; i < G.n_ra; ++i) {
        if ((1u << G.cbn[i]) > cmax_ra) cmax_ra = 1u << G.cbn[i];
        if (G.cp[i] > kb_max) kb_max = G.cp[i];
    }
    L.m = m;
    L.keys_n = 1;
    while (L.keys_n < m) L.keys_n <<= 1;
    L.hc_stride = cmax_ra;
    L.boff_stride = (1u << kb_max) + 1u;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.state = take(sizeof(DevState));
    L.za = take(sizeof(uint64_t) * S * G.A);          // right after the state: one memset clears both
    L.zc = take(sizeof(uint16_t) * S * G.A * G.cmax);
    L.eps = take(sizeof(double) * S);
    L.zmax = take(sizeof(int64_t) * S);
    L.hc = take(sizeof(uint16_t) * S * G.n_ra * L.hc_stride);
    L.nhc = take(sizeof(uint32_t) * S * G.n_ra);
    L.boff = take(sizeof(uint32_t) * S * G.n_ra * L.boff_stride);
    L.tup0 = take(sizeof(Tuple) * m);
    L.tup1 = take(sizeof(Tuple) * m);
    L.hosts = take(sizeof(cbaa_host) * m);
    L.sorted = take(sizeof(cbaa_host) * m);
    L.keys = take(sizeof(unsigned long long) * L.keys_n);
    L.total = o;
    return L;
}

// Largest m (capped at 2^31) whose layout fits in `bytes`; false if even m = 1 does not.
inline bool ws_layout_fit(const Geo &G, size_t bytes, WsLayout *out) {
    if (ws_layout(G, 1).total > bytes) return false;
    uint64_t lo = 1, hi = 1;
    while (hi < (1ull << 31) && ws_layout(G, hi * 2).total <= bytes) hi *= 2;
    lo = hi;
    hi = hi * 2;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) / 2;
        if (ws_layout(G, mid).total <= bytes) lo = mid; else hi = mid;
    }
    *out = ws_layout(G, lo);
    return true;
}

inline WsPtrs ws_pointers(const Geo &G, const WsLayout &L, void *base) {
    (void)G;
    char *b = static_cast<char *>(base);
    WsPtrs P;
    P.state = reinterpret_cast<DevState *>(b + L.state);
    P.zc = reinterpret_cast<uint16_t *>(b + L.zc);
    P.za = reinterpret_cast<uint64_t *>(b + L.za);
    P.eps = reinterpret_cast<double *>(b + L.eps);
    P.zmax = reinterpret_cast<int64_t *>(b + L.zmax);
    P.hc = reinterpret_cast<uint16_t *>(b + L.hc);
    P.nhc = reinterpret_cast<uint32_t *>(b + L.nhc);
    P.boff = reinterpret_cast<uint32_t *>(b + L.boff);
    P.tup[0] = reinterpret_cast<Tuple *>(b + L.tup0);
    P.tup[1] = reinterpret_cast<Tuple *>(b + L.tup1);
    P.hosts = reinterpret_cast<cbaa_host *>(b + L.hosts);
    P.sorted = reinterpret_cast<cbaa_host *>(b + L.sorted);
    P.keys = reinterpret_cast<unsigned long long *>(b + L.keys);
    P.m = (uint32_t)L.m;
    P.hc_stride = L.hc_stride;
    P.boff_stride = L.boff_stride;
    return P;
}

// Restoration of the sketches [cs_lo, cs_hi) (cs_hi = 0: all of them).
// Merge k owners' sorted host lists (blocks of cap records, counts in infos)
// into out (room for out_cap) sorted by ip, and their infos into info_out.
cudaError_t launch_merge_hosts(const cbaa_host *blocks, uint32_t cap, uint32_t k, const cbaa_detect_info *infos,
                               cbaa_host *out, uint64_t out_cap, cbaa_detect_info *info_out, cudaStream_t s);
int detect_enqueue(const Geo &G, const uint32_t *cube, uint32_t theta, void *ws, size_t ws_bytes,
                   cbaa_host *out, uint64_t cap, cbaa_detect_info *info_copy, int num_sms, cudaStream_t s,
                   uint32_t cs_lo = 0, uint32_t cs_hi = 0);

}  // namespace cbaa
