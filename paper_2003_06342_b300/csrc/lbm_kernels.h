// Kernel launchers shared between the kernel files and the C ABI layer, and
// the FP64 block reduction used by the moment kernels.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include "lbm_common.cuh"

namespace lbm {

// Sum two doubles over the block (warp shuffles, then one warp over the
// per-warp sums) and store the pair at partial[2*blockIdx.x].  Every thread
// of the block must call it.  The summation order is fixed, so results are
// reproducible run to run.
// Programmatic dependent launch.  A kernel launched by pdl_launch may have
// its blocks scheduled while the kernel before it on the stream drains; it
// calls pdl_wait first, which returns once that kernel has completed and its
// writes are visible, and then lets the kernel after it be scheduled the same
// way.  Nothing before pdl_wait touches global memory.  Launched without the
// attribute (or after a copy), the wait returns at once.
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Blocks of 256 threads of the moment kernels, which also form the FP64
// mass and energy partial sums: one thread per cell up to two waves of 148 x
// 4 blocks, then a grid-stride loop, so each thread adds several cells into
// its FP64 accumulators before the (FP64) warp-shuffle block reduction.  B300
// runs FP64 at a small fraction of its FP32 rate, and the block reduction's
// shuffles and adds dominated a one-cell-per-thread sum.
inline int moment_blocks(long long n_cells) {
    const long long b = (n_cells + 255) / 256;
    return (int)(b < 148 * 8 ? (b < 1 ? 1 : b) : 148 * 8);
}

__device__ __forceinline__ void block_sum2(double a, double b, double *partial) {
    __shared__ double sa[32], sb[32];
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(full, a, o);
        b += __shfl_down_sync(full, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (lane == 0) { sa[warp] = a; sb[warp] = b; }
    __syncthreads();
    if (warp == 0) {
        a = lane < nwarps ? sa[lane] : 0.0;
        b = lane < nwarps ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(full, a, o);
            b += __shfl_down_sync(full, b, o);
        }
        if (lane == 0) {
            partial[2 * blockIdx.x] = a;
            partial[2 * blockIdx.x + 1] = b;
        }
    }
}

// 2D phase field alone in an imposed velocity u(x) * factor (cac2d.cu);
// vel holds ux then uy, N floats each
template <typename S>
cudaError_t launch_cac2d(const void *pin, void *pout, const float *vel, float factor,
                         const DevParams &P, cudaStream_t st);

// 3D phase field alone (cac3d.cu): vel holds ux, uy, uz (N floats each);
// q_zero is a lagged-source buffer of zeros (no phase change)
template <typename S>
cudaError_t launch_cac3d(const void *pin, void *pout, const float *q_zero, const float *vel, float factor,
                         const DevParams &P, cudaStream_t st);

// periodic state check (health.cu): bit 4 of *err when phi leaves
// [1/2 - excess, 1/2 + excess] or phi / the lagged source is not finite
template <typename S>
cudaError_t launch_health(const void *pops, const float *q, float excess, int *err, const DevParams &P,
                          int dim, cudaStream_t st);

// 2D (lbm2d.cu); S = float, __half or __nv_bfloat16 storage
template <typename S>
cudaError_t launch_step2d(const void *pin, void *pout, float *phi_prev, const float *q_in,
                          float *q_out, const DevParams &P, cudaStream_t st);
template <typename S>
cudaError_t launch_macro2d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *o_ux, float *o_uy,
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st);
template <typename S>
cudaError_t launch_init2d(const float *phi0, const float *T0, const float *ux0, const float *uy0,
                          const float *p0, void *pout, float *phi_prev, float *q_out,
                          const DevParams &P, cudaStream_t st);
cudaError_t launch_streammap2d(int32_t *src, int8_t *kind, const DevParams &P, cudaStream_t st);

// column blocks of the state (columns.cu): copy the populations, phi^{n-1}
// and the lagged source of columns [x0, x0 + ncols) (every y and z; rows =
// ny nz) to (pack) or from (unpack) buf: Qtot planes of rows x ncols stored
// values, padded to 16 bytes, then two planes of rows x ncols floats
size_t columns_pop_bytes(long long cells, int Qtot, size_t elem);
template <typename S>
cudaError_t launch_columns(void *pops, float *phi_prev, float *q, void *buf, int x0, int ncols, int nx,
                           long long rows, long long N, int Qf, int Qtot, bool pack, cudaStream_t st);

// reductions (reduce.cu): sum nblocks (a, b) pairs into out[0..1]
cudaError_t launch_final_sum2(const double *partial, int nblocks, double *out, cudaStream_t st);
// float -> float copy with optional double conversion helpers
cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, size_t n, cudaStream_t st);
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, size_t n, cudaStream_t st);

}  // namespace lbm
