// 3D launchers (lbm3d.cu): D3Q19 for f and s, D3Q7 for g.
#pragma once

#include <cuda_runtime.h>
#include "lbm_common.cuh"

namespace lbm {

template <typename S>
cudaError_t launch_step3d(const void *pin, void *pout, float *phi_prev, const float *q_in,
                          float *q_out, const DevParams &P, cudaStream_t st);
template <typename S>
cudaError_t launch_macro3d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *const o_u[3],
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st);
template <typename S>
cudaError_t launch_init3d(const float *phi0, const float *T0, const float *const u0[3],
                          const float *p0, void *pout, float *phi_prev, float *q_out,
                          const DevParams &P, cudaStream_t st);
cudaError_t launch_streammap3d(int set, int32_t *src, int8_t *kind, const DevParams &P,
                               cudaStream_t st);

}  // namespace lbm
