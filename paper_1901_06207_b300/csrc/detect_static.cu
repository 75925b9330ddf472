// Detect with library-owned scratch: for callers that cannot allocate
// device memory at run time.  The work is the same enqueue as
// cbaa_detect_async; only where the scratch lives differs.
#include <mutex>

#include "cbaa_internal.cuh"
#include "detect_layout.h"

namespace {

// One array per device that loads the library, held until process exit.
static __device__ __align__(256) unsigned char g_detect_scratch[CBAA_STATIC_SCRATCH_BYTES];

// The name above is only a host-side stand-in; its device address is looked
// up once per device and cached here.
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CBAA_ERR_NO_DEVICE;
    if (dev < 0 || dev >= kMaxDevices) return CBAA_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_detect_scratch);
        if (e != cudaSuccess) return cbaa::cuda_status(e);
        if (!p) return CBAA_ERR_NO_DEVICE;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CBAA_OK;
}

}  // namespace

extern "C" int cbaa_detect_static(const cbaa_cube *cube, uint32_t theta, cbaa_host *dev_out, size_t cap,
                                  cbaa_detect_info *dev_info, void *stream) {
    if (!cube || !dev_info || (cap > 0 && !dev_out)) return CBAA_ERR_INVALID_ARG;
    cbaa_params p;
    if (cbaa_cube_params(cube, &p) != CBAA_OK) return CBAA_ERR_INVALID_ARG;
    const uint32_t *data = static_cast<const uint32_t *>(cbaa_cube_data(cube));
    const cbaa::Geo G = cbaa::make_geo(p);
    // The geometry's fixed tables (zero counts, hot lists, bucket offsets)
    // plus room for at least one tuple must fit in the static array.
    if (cbaa::ws_layout(G, 1).total > CBAA_STATIC_SCRATCH_BYTES) return CBAA_ERR_WORKSPACE;
    void *ws = nullptr;
    const int st = scratch_for_current_device(&ws);
    if (st != CBAA_OK) return st;
    // detect_enqueue zeroes the state words and array totals it accumulates
    // into, so nothing left by an earlier call is read.
    return cbaa::detect_enqueue(G, data, theta, ws, CBAA_STATIC_SCRATCH_BYTES, dev_out, cap, dev_info,
                                cbaa::num_sms(), reinterpret_cast<cudaStream_t>(stream));
}
