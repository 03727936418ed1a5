// Second pass of the FP64 global reductions and dtype conversions.
#include "lbm_kernels.h"

namespace lbm {

// One block of 256 threads sums the per-block pairs in a fixed order.
__global__ void __launch_bounds__(256) final_sum2_kernel(const double *__restrict__ partial,
                                                         int nblocks, double *out) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    block_sum2(a, b, out);   // single block: writes out[0], out[1]
}

cudaError_t launch_final_sum2(const double *partial, int nblocks, double *out, cudaStream_t st) {
    final_sum2_kernel<<<1, 256, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(const double *__restrict__ s, float *__restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

__global__ void f32_to_f64_kernel(const float *__restrict__ s, double *__restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 148 * 32 ? 148 * 32 : (b == 0 ? 1 : b));
}

cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t st) {
    f64_to_f32_kernel<<<grid_for(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, size_t n, cudaStream_t st) {
    f32_to_f64_kernel<<<grid_for(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace lbm
