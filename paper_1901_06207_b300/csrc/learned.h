// Learned-estimator kernels (features, MLP forward / gradient / Adam, decision).
#pragma once

#include "cbaa_internal.cuh"

namespace cbaa {
cudaError_t launch_features(const Geo &G, const uint32_t *cube, const uint64_t *za, const double *eps,
                            const uint32_t *ips, uint64_t n, float *feats, cudaStream_t s);
cudaError_t launch_mlp_forward(const uint16_t *Wb, const float *X, uint64_t n, float *Y, cudaStream_t s);
cudaError_t launch_mlp_grad(const uint16_t *Wb, const float *X, const float *T, uint64_t n, float scale,
                            float *grad, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *master, const float *grad, float *m, float *v, uint16_t *Wb, float lr, float b1,
                        float b2, float eps, uint32_t step, cudaStream_t s);
cudaError_t launch_to_bf16(const float *master, uint16_t *Wb, cudaStream_t s);
cudaError_t launch_target(const float *feats, const float *count, uint64_t n, float *t, cudaStream_t s);
cudaError_t launch_decide(const float *y, const float *feats, uint64_t n, float g, float theta, float *card,
                          uint8_t *decision, cudaStream_t s);
}  // namespace cbaa
