// TMA-staged 3D step (lbm3d_tma.cu): tensor maps and launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include "lbm_common.cuh"

namespace lbm {

// Tensor maps of the two population buffers as (x, y, z, plane): `fs` over
// the (f_i, s_i) pair planes (one element = one pair) with a 32 x 4 x 1 x 19
// box (the f and s sets of one tile layer), `g` over the g planes with a
// 32 x 4 x 1 x 7 box; of the two lagged-source buffers and of phi^{n-1}
// (32 x 4 x 1 boxes); index = which buffer is read.
struct TmaMaps3d {
    CUtensorMap fs[2], g[2], q[2], pp;
};

// Row, plane and population-plane strides are multiples of 16 bytes and the
// grid holds at least one whole 32 x 4 tile.
bool tma3d_eligible(const DevParams &P, int elem_bytes);
// Encode the maps; 0 on success.
int make_tma_maps3d(TmaMaps3d *M, const DevParams &P, int elem_bytes, void *const pops[2],
                    float *const q[2], float *phi_prev);
// Set the kernel's dynamic shared-memory limit; resident blocks per SM (0 on failure).
int tma3d_blocks_per_sm(int elem_bytes);

// Polls of the first mbarrier wait of every block (negative: the default
// WAIT_LIMIT), on the current device; the timeout test's hook.
cudaError_t set_first_wait_limit3d(int polls);

template <typename S>
cudaError_t launch_step3d_tma(const TmaMaps3d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, cudaStream_t st);

}  // namespace lbm
