// Periodic state check (optional, lbm_set_health_check): every `every` steps
// one launch reads the current state, forms phi = sum_i gbar_i + q/2 (Eq.
// Moment_Phi) and sets bit 4 of the handle's status word when a cell's phi
// leaves [1/2 - excess, 1/2 + excess] or is not a number, or when one of its
// stored populations or its lagged source is not finite.  A blow-up is thus
// reported by the next lbm_sync as LBM_ENONFINITE without a host round trip
// per step.  Algorithmic bytes per cell: the (2 Qf + Qg) stored populations
// and one float, read only.
#include "lbm_common.cuh"
#include "lbm_kernels.h"

namespace lbm {

template <typename S, int QF, int QG>
__global__ void __launch_bounds__(256)
health_kernel(const S *__restrict__ pops, const float *__restrict__ q, float excess, int *err,
              const DevParams P) {
    const size_t N = (size_t)P.N;
    bool bad = false;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
        const float qc = q[c];
        float phi = 0.5f * qc;
#pragma unroll
        for (int i = 0; i < QG; ++i) phi += Codec<S>::load(pops + off_g(QF, i, c, N), QF + i, P);
        // a NaN or an infinity in any stored f or s value makes this sum non-finite
        float fs = 0.0f;
#pragma unroll
        for (int i = 0; i < QF; ++i) {
            float a, b;
            load_pair<S>(pops + off_f(i, 0, N), (long long)c, a, b);
            fs += fabsf(a) + fabsf(b);
        }
        // written so that a NaN fails every test
        bad |= !(fabsf(phi - 0.5f) <= excess) || !(fabsf(qc) <= 3.0e38f) || !(fs <= 3.0e38f);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 4);
}

template <typename S>
cudaError_t launch_health(const void *pops, const float *q, float excess, int *err, const DevParams &P,
                          int dim, cudaStream_t st) {
    const size_t N = (size_t)P.N;
    size_t blocks = (N + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (dim == 2)
        health_kernel<S, 9, 9><<<(unsigned)blocks, 256, 0, st>>>((const S *)pops, q, excess, err, P);
    else
        health_kernel<S, 19, 7><<<(unsigned)blocks, 256, 0, st>>>((const S *)pops, q, excess, err, P);
    return cudaGetLastError();
}

template cudaError_t launch_health<float>(const void *, const float *, float, int *, const DevParams &, int,
                                          cudaStream_t);
template cudaError_t launch_health<__half>(const void *, const float *, float, int *, const DevParams &, int,
                                           cudaStream_t);
template cudaError_t launch_health<__nv_bfloat16>(const void *, const float *, float, int *, const DevParams &,
                                                  int, cudaStream_t);

}  // namespace lbm
