// 2D step, persistent and TMA-staged.
//
// Same update as step2d_kernel (lbm2d.cu), organised so that the loads of the
// next tile overlap the arithmetic of the current one.  Each block walks the
// 32x8 tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...  For a tile whose
// one-cell halo lies inside the grid, one thread issues five bulk tensor
// copies (cp.async.bulk.tensor) into a shared-memory stage:
//   g planes  9 x 10 x 32 from (x0, y0 - 1)  (tile columns, both halo rows)
//             9 x 10 x SW from (x0 - SW, y0 - 1) and (x0 + 32, y0 - 1)
//             (the halo columns, in 16-byte boxes: SW = 4 floats or 8 halves)
//   q         10 x 32 and two 10 x 4 side boxes, placed the same way
//   f planes  9 x 8 x 32  from (x0, y0)
//   s planes  9 x 8 x 32  from (x0, y0)
//   phi^{n-1} 8 x 32      from (x0, y0)
// (each row of a centre box is one whole 128-byte line of a 32-float row)
// completing on that stage's mbarrier; two stages alternate, so the copies of
// tile k+1 are in flight while tile k is computed.  The block then forms
// phi^n - phi_ref on the tile and its halo from the staged g and q (no global
// loads), and each thread runs the shared per-cell update and pushes its 27
// post-collision values to global memory.  Tiles that touch the grid's edge
// (periodic wrap or walls) take the generic path of the tiled kernel.
//
// Every wait on an mbarrier is bounded: on expiry the block records an error
// code in a device word, waits (again bounded) for a copy it may still have in
// flight, and returns; the host reports it as LBM_ETIMEOUT at the next sync.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm2d_cell.cuh"
#include "lbm2d_tma.h"
#include "tma_util.cuh"

namespace lbm {

template <typename S> struct TmaGeom {
    static constexpr int ES = (int)sizeof(S);
    static constexpr int SW = 16 / ES;                    // side boxes: 16 bytes wide
    static constexpr int GH = TY + 2;                     // tile rows + the two halo rows
    static constexpr int QSW = 4;                         // q is float32
    static constexpr int al(int b) { return (b + 127) / 128 * 128; }
    static constexpr int GC_BYTES = 9 * GH * TX * ES;     // g, columns x0..x0+31
    static constexpr int GS_BYTES = 9 * GH * SW * ES;     // g, SW columns left or right
    static constexpr int QC_BYTES = GH * TX * 4;
    static constexpr int QS_BYTES = GH * QSW * 4;
    static constexpr int F_BYTES = 9 * TY * TX * ES;
    static constexpr int PP_BYTES = TY * TX * 4;
    static constexpr int OFF_GC = 0;
    static constexpr int OFF_GL = OFF_GC + al(GC_BYTES);
    static constexpr int OFF_GR = OFF_GL + al(GS_BYTES);
    static constexpr int OFF_QC = OFF_GR + al(GS_BYTES);
    static constexpr int OFF_QL = OFF_QC + al(QC_BYTES);
    static constexpr int OFF_QR = OFF_QL + al(QS_BYTES);
    static constexpr int OFF_F = OFF_QR + al(QS_BYTES);
    static constexpr int OFF_S = OFF_F + al(F_BYTES);
    static constexpr int OFF_PP = OFF_S + al(F_BYTES);
    static constexpr int STAGE = OFF_PP + al(PP_BYTES);
    static constexpr unsigned TX_BYTES = GC_BYTES + 2 * GS_BYTES + QC_BYTES + 2 * QS_BYTES +
                                         2 * F_BYTES + PP_BYTES;
};

__device__ __forceinline__ bool tile_is_fast(int x0, int y0, const DevParams &P) {
    return x0 >= 1 && x0 + TX + 1 <= P.n[0] && y0 >= 1 && y0 + TY + 1 <= P.n[1];
}

template <typename S>
__device__ __forceinline__ void issue_tile(unsigned char *stage, uint64_t *bar, const TmaMaps2d &M,
                                           int par, int x0, int y0) {
    using Gm = TmaGeom<S>;
    // order earlier generic-proxy accesses of this stage before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::TX_BYTES);
    // every box starts on a 16-byte boundary; the centre boxes cover whole
    // 128-byte lines of the tile's own columns
    tma_load_3d(stage + Gm::OFF_GC, &M.gc[par], x0, y0 - 1, 9, bar);
    tma_load_3d(stage + Gm::OFF_GL, &M.gs[par], x0 - Gm::SW, y0 - 1, 9, bar);
    tma_load_3d(stage + Gm::OFF_GR, &M.gs[par], x0 + TX, y0 - 1, 9, bar);
    tma_load_2d(stage + Gm::OFF_QC, &M.qc[par], x0, y0 - 1, bar);
    tma_load_2d(stage + Gm::OFF_QL, &M.qs[par], x0 - Gm::QSW, y0 - 1, bar);
    tma_load_2d(stage + Gm::OFF_QR, &M.qs[par], x0 + TX, y0 - 1, bar);
    tma_load_3d(stage + Gm::OFF_F, &M.fs[par], x0, y0, 0, bar);
    tma_load_3d(stage + Gm::OFF_S, &M.fs[par], x0, y0, 18, bar);
    tma_load_2d(stage + Gm::OFF_PP, &M.pp, x0, y0, bar);
}

template <typename S>
__global__ void __launch_bounds__(TX * TY, 2)
step2d_tma_kernel(const __grid_constant__ TmaMaps2d maps, const S *__restrict__ pin,
                  S *__restrict__ pout, float *__restrict__ phi_prev,
                  const float *__restrict__ q_in, float *__restrict__ q_out, int par, int *err,
                  const DevParams P) {
    using Gm = TmaGeom<S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies want 128-byte aligned destinations
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float sphi[SY * SX];
    const int nx = P.n[0];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int tiles_x = (nx + TX - 1) / TX;
    const int ntiles = tiles_x * ((P.n[1] + TY - 1) / TY);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t phase0 = 0, phase1 = 0;
    int stage = 0;
    int t = blockIdx.x;
    if (t < ntiles && tid == 0) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        if (tile_is_fast(x0, y0, P)) issue_tile<S>(smem, &bars[0], maps, par, x0, y0);
    }
    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        const int tn = t + gridDim.x;
        bool next_issued = false;
        if (tn < ntiles) {
            const int xn = (tn % tiles_x) * TX, yn = (tn / tiles_x) * TY;
            next_issued = tile_is_fast(xn, yn, P);
            if (next_issued && tid == 0)
                issue_tile<S>(smem + (stage ^ 1) * Gm::STAGE, &bars[stage ^ 1], maps, par, xn, yn);
        }
        if (tile_is_fast(x0, y0, P)) {
            const uint32_t ph = stage ? phase1 : phase0;
            const bool ok = mbar_wait_bounded(&bars[stage], ph);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicExch(err, 1);
                if (next_issued)     // a copy of the next tile may still be landing here
                    mbar_wait_bounded(&bars[stage ^ 1], stage ? phase0 : phase1);
                return;
            }
            if (stage) phase1 ^= 1u; else phase0 ^= 1u;
            const unsigned char *base = smem + stage * Gm::STAGE;
            const S *GC = (const S *)(base + Gm::OFF_GC);
            const S *GL = (const S *)(base + Gm::OFF_GL);
            const S *GR = (const S *)(base + Gm::OFF_GR);
            const float *QC = (const float *)(base + Gm::OFF_QC);
            const float *QL = (const float *)(base + Gm::OFF_QL);
            const float *QR = (const float *)(base + Gm::OFF_QR);
            const S *F = (const S *)(base + Gm::OFF_F);
            const S *Sv = (const S *)(base + Gm::OFF_S);
            const float *PP = (const float *)(base + Gm::OFF_PP);
            // phi^n - phi_ref on the tile and its halo, from the staged boxes
            for (int sidx = tid; sidx < SX * SY; sidx += TX * TY) {
                const int sx = sidx % SX, sy = sidx / SX;
                const S *gb;
                int col, w;
                float qv;
                if (sx == 0) { gb = GL; col = Gm::SW - 1; w = Gm::SW; qv = QL[sy * Gm::QSW + Gm::QSW - 1]; }
                else if (sx == SX - 1) { gb = GR; col = 0; w = Gm::SW; qv = QR[sy * Gm::QSW]; }
                else { gb = GC; col = sx - 1; w = TX; qv = QC[sy * TX + sx - 1]; }
                const int gi = sy * w + col;
                const int plane = Gm::GH * w;
                float v[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i] = widen(gb[i * plane + gi]);
                sphi[sidx] = fmaf(0.5f, qv, set_sum2d<S>(v, P.set_isc[1]));
            }
            __syncthreads();
            float f[9], g[9], s[9];
            const int own = ty * TX + tx;
            const int gown = (ty + 1) * TX + tx;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f[i] = widen(F[i * TY * TX + own]);
                g[i] = widen(GC[i * Gm::GH * TX + gown]);
                s[i] = widen(Sv[i * TY * TX + own]);
            }
            const float phip = PP[own];
            const float qp = QC[(ty + 1) * TX + tx];
            const int x = x0 + tx, y = y0 + ty;
            const size_t c = (size_t)y * nx + x;
            cell_update2d<S, true>(sphi + (ty + 1) * SX + tx + 1, SX, f, g, s, phip, qp, x, y, c,
                                   pout, phi_prev, q_out, P);
        } else {
            step2d_tile<S, false>(pin, pout, phi_prev, q_in, q_out, P, sphi, x0, y0);
        }
        __syncthreads();      // stage buffers and the phi window are free again
        stage ^= 1;
    }
    (void)N;
}

// ------------------------------------------------------------------ host side
static cuuint32_t dtype_for(int es) {
    return es == 4 ? (cuuint32_t)CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : (cuuint32_t)CU_TENSOR_MAP_DATA_TYPE_UINT16;
}

bool tma2d_eligible(const DevParams &P, int elem_bytes) {
    const long long nx = P.n[0], ny = P.n[1];
    if (nx < 2 * TX + 2 || ny < 2 * TY + 2) return false;
    if ((nx * elem_bytes) % 16 != 0 || (nx * 4) % 16 != 0) return false;
    if ((P.N * elem_bytes) % 16 != 0) return false;
    return true;
}

int make_tma_maps2d(TmaMaps2d *M, const DevParams &P, int elem_bytes, void *const pops[2],
                    float *const q[2], float *phi_prev) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const cuuint64_t nx = (cuuint64_t)P.n[0], ny = (cuuint64_t)P.n[1], N = (cuuint64_t)P.N;
    const cuuint64_t es = (cuuint64_t)elem_bytes;
    const cuuint32_t sw = (cuuint32_t)(16 / elem_bytes);
    const cuuint32_t one[3] = {1, 1, 1};
    const CUtensorMapDataType dt = (CUtensorMapDataType)dtype_for(elem_bytes);
    auto map3 = [&](CUtensorMap *m, void *base, cuuint32_t bx, cuuint32_t by) {
        const cuuint64_t dims[3] = {nx, ny, 27};
        const cuuint64_t str[2] = {nx * es, N * es};
        const cuuint32_t box[3] = {bx, by, 9};
        return enc(m, dt, 3, base, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto map2 = [&](CUtensorMap *m, void *base, cuuint32_t bx, cuuint32_t by) {
        const cuuint64_t dims[2] = {nx, ny};
        const cuuint64_t str[1] = {nx * 4};
        const cuuint32_t box[2] = {bx, by};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, str, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
        if (!map3(&M->gc[b], pops[b], TX, TY + 2)) return -2;
        if (!map3(&M->gs[b], pops[b], sw, TY + 2)) return -3;
        if (!map3(&M->fs[b], pops[b], TX, TY)) return -4;
        if (!map2(&M->qc[b], q[b], TX, TY + 2)) return -5;
        if (!map2(&M->qs[b], q[b], 4, TY + 2)) return -6;
    }
    if (!map2(&M->pp, phi_prev, TX, TY)) return -7;
    return 0;
}

template <typename S>
cudaError_t launch_step2d_tma(const TmaMaps2d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, int nblocks, cudaStream_t st) {
    using Gm = TmaGeom<S>;
    const int dyn = 2 * Gm::STAGE + 128;  // attribute set by tma2d_blocks_per_sm
    dim3 block(TX, TY);
    step2d_tma_kernel<S><<<nblocks, block, dyn, st>>>(M, (const S *)pin, (S *)pout, phi_prev, q_in,
                                                       q_out, par, err, P);
    return cudaGetLastError();
}

int tma2d_blocks_per_sm(int elem_bytes) {
    int n = 0;
    cudaError_t e;
    if (elem_bytes == 4) {
        const int dyn = 2 * TmaGeom<float>::STAGE + 128;
        e = cudaFuncSetAttribute(step2d_tma_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step2d_tma_kernel<float>, TX * TY, dyn);
    } else {
        const int dyn = 2 * TmaGeom<__half>::STAGE + 128;
        e = cudaFuncSetAttribute(step2d_tma_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step2d_tma_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step2d_tma_kernel<__half>, TX * TY, dyn);
    }
    return e == cudaSuccess ? n : 0;
}

template cudaError_t launch_step2d_tma<float>(const TmaMaps2d &, int, const void *, void *, float *,
                                              const float *, float *, int *, const DevParams &, int,
                                              cudaStream_t);
template cudaError_t launch_step2d_tma<__half>(const TmaMaps2d &, int, const void *, void *, float *,
                                               const float *, float *, int *, const DevParams &, int,
                                               cudaStream_t);
template cudaError_t launch_step2d_tma<__nv_bfloat16>(const TmaMaps2d &, int, const void *, void *,
                                                      float *, const float *, float *, int *,
                                                      const DevParams &, int, cudaStream_t);

}  // namespace lbm
