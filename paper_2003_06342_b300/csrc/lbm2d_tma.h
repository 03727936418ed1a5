// TMA-staged persistent 2D step (lbm2d_tma.cu): tensor maps and launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include "lbm_common.cuh"

namespace lbm {

// Tensor maps of the two population buffers (g centre and side boxes, f/s
// box), the two lagged-source buffers (centre and side boxes) and phi^{n-1};
// index = which buffer is read.
struct TmaMaps2d {
    CUtensorMap gc[2], gs[2], fs[2], qc[2], qs[2], pp;
};

// Grid and storage allow 16-byte-aligned boxes (row and plane strides).
bool tma2d_eligible(const DevParams &P, int elem_bytes);
// Encode the maps; 0 on success.
int make_tma_maps2d(TmaMaps2d *M, const DevParams &P, int elem_bytes, void *const pops[2],
                    float *const q[2], float *phi_prev);
// Set the kernel's dynamic shared-memory limit; resident blocks per SM (0 on failure).
int tma2d_blocks_per_sm(int elem_bytes);

template <typename S>
cudaError_t launch_step2d_tma(const TmaMaps2d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, int nblocks, cudaStream_t st);

}  // namespace lbm
