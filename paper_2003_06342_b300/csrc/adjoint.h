// Adjoint launchers (adjoint2d.cu) and the FP64 block-sum-and-add helper.
#pragma once

#include <cuda_runtime.h>
#include "lbm_common.cuh"

namespace lbm {

// Sum three doubles over the block (warp shuffles, then one warp) and add the
// block's sums to out[0..2] with one atomic each.  Every thread must call it.
__device__ __forceinline__ void block_sum3_atomic(double a, double b, double c, double *out) {
    __shared__ double sa[32], sb[32], sc[32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(full, a, o);
        b += __shfl_down_sync(full, b, o);
        c += __shfl_down_sync(full, c, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (lane == 0) { sa[warp] = a; sb[warp] = b; sc[warp] = c; }
    __syncthreads();
    if (warp == 0) {
        a = lane < nwarps ? sa[lane] : 0.0;
        b = lane < nwarps ? sb[lane] : 0.0;
        c = lane < nwarps ? sc[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(full, a, o);
            b += __shfl_down_sync(full, b, o);
            c += __shfl_down_sync(full, c, o);
        }
        if (lane == 0) {
            atomicAdd(out, a);
            atomicAdd(out + 1, b);
            atomicAdd(out + 2, c);
        }
    }
}

// The same for per-thread FP32 terms: the warp sums are taken in FP32 (32
// terms), everything above a warp in FP64.  Keeps FP64 arithmetic, which is
// slow on B300, out of the per-cell path.  Every thread must call it.
__device__ __forceinline__ void block_sum3f_atomic(float a, float b, float c, double *out) {
    __shared__ double sa[32], sb[32], sc[32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(full, a, o);
        b += __shfl_down_sync(full, b, o);
        c += __shfl_down_sync(full, c, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (lane == 0) { sa[warp] = (double)a; sb[warp] = (double)b; sc[warp] = (double)c; }
    __syncthreads();
    if (warp == 0) {
        double da = lane < nwarps ? sa[lane] : 0.0;
        double db = lane < nwarps ? sb[lane] : 0.0;
        double dc = lane < nwarps ? sc[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            da += __shfl_down_sync(full, da, o);
            db += __shfl_down_sync(full, db, o);
            dc += __shfl_down_sync(full, dc, o);
        }
        if (lane == 0) {
            atomicAdd(out, da);
            atomicAdd(out + 1, db);
            atomicAdd(out + 2, dc);
        }
    }
}

cudaError_t launch_adj_terminal2d(const float *st, const float *target, float *adj, double *J,
                                  const DevParams &P, cudaStream_t stream);
cudaError_t launch_adj_step2d(const float *st, const float *lam_next, float *lam, float *cst,
                              double *dparams, const DevParams &P, cudaStream_t stream);
cudaError_t launch_adj_init2d(const float *phi0, const float *T0, const float *ux0,
                              const float *uy0, const float *lam, float *dT0, double *dparams,
                              const DevParams &P, cudaStream_t stream);

}  // namespace lbm
