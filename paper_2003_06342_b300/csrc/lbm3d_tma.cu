// 3D step with every tile layer staged by bulk tensor copies.
//
// Same update as step3d_kernel (lbm3d.cu): each block marches a 32x8 column
// tile through ZB layers.  For each layer L of its range (and the layer above
// the range), one thread issues five cp.async.bulk.tensor copies into a
// shared-memory stage:
//   f planes   32 x 8 x 1 x 19 from (x0, y0, L, 0)    4D map (x, y, z, plane)
//   s planes   32 x 8 x 1 x 19 from (x0, y0, L, 26)
//   g planes   32 x 8 x 1 x 7  from (x0, y0, L, 19)
//   q^{n-1}    32 x 8 x 1      from (x0, y0, L)       3D maps (x, y, z)
//   phi^{n-1}  32 x 8 x 1      from (x0, y0, L)
// completing on that stage's mbarrier (each box row is one whole 128-byte line
// of FP32, or 64 bytes of 16-bit values).  Two stages alternate: when layer z
// is computed, the copies of layer z+1 have landed (the phi window needs them
// first) and those of layer z+2 are issued as soon as layer z's stage is
// free, so the next layer's loads overlap this layer's arithmetic without
// holding the populations in registers.  The halo ring of the phi window is
// formed with plain loads, which find those cells in L2 (the neighbouring
// blocks stage them at about the same time).  A tile that does not fit the
// grid whole takes the plain-load column of step3d_kernel.
//
// Waits on the mbarriers are bounded: on expiry the block records an error in
// a device word, waits (bounded) for its copies in flight and returns; the
// host reports LBM_ETIMEOUT at the next sync.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm3d_cell.cuh"
#include "lbm3d_tma.h"
#include "tma_util.cuh"

namespace lbm {

template <typename S> struct Tma3Geom {
    static constexpr int ES = (int)sizeof(S);
    static constexpr int CELLS = TX * TY;
    static constexpr int al(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_BYTES = QF * CELLS * ES;
    static constexpr int G_BYTES = QG * CELLS * ES;
    static constexpr int Q_BYTES = CELLS * 4;
    static constexpr int OFF_F = 0;
    static constexpr int OFF_S = OFF_F + al(F_BYTES);
    static constexpr int OFF_G = OFF_S + al(F_BYTES);
    static constexpr int OFF_Q = OFF_G + al(G_BYTES);
    static constexpr int OFF_PP = OFF_Q + al(Q_BYTES);
    static constexpr int STAGE = OFF_PP + al(Q_BYTES);
    static constexpr unsigned TX_BYTES = 2 * F_BYTES + G_BYTES + 2 * Q_BYTES;
    static constexpr int DYN = 2 * STAGE + 128;     // two stages + alignment slack
};

template <typename S>
__device__ __forceinline__ void issue_layer(unsigned char *stage, uint64_t *bar, const TmaMaps3d &M,
                                            int par, int x0, int y0, int z) {
    using Gm = Tma3Geom<S>;
    // order earlier generic-proxy reads of this stage before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::TX_BYTES);
    tma_load_4d(stage + Gm::OFF_F, &M.fs[par], x0, y0, z, 0, bar);
    tma_load_4d(stage + Gm::OFF_S, &M.fs[par], x0, y0, z, S0, bar);
    tma_load_4d(stage + Gm::OFF_G, &M.g[par], x0, y0, z, G0, bar);
    tma_load_3d(stage + Gm::OFF_Q, &M.q[par], x0, y0, z, bar);
    tma_load_3d(stage + Gm::OFF_PP, &M.pp, x0, y0, z, bar);
}

// phi - phi_ref of the thread's own cell from a stage (same arithmetic as
// phid_at, so the halo ring of a neighbouring block sees the same float)
template <typename S>
__device__ __forceinline__ float staged_phid(const unsigned char *stage, int own, const DevParams &P) {
    using Gm = Tma3Geom<S>;
    const S *G = (const S *)(stage + Gm::OFF_G);
    float v[QG];
#pragma unroll
    for (int i = 0; i < QG; ++i) v[i] = widen(G[i * Gm::CELLS + own]);
    return fmaf(0.5f, ((const float *)(stage + Gm::OFF_Q))[own], set_sum7<S>(v, P.set_isc[1]));
}

template <typename S, bool FXY>
__device__ __forceinline__ void tma_column(const TmaMaps3d &M, int par, const S *__restrict__ pin,
                                           S *__restrict__ pout, float *__restrict__ phi_prev,
                                           const float *__restrict__ q_in, float *__restrict__ q_out,
                                           int *err, const DevParams &P, unsigned char *smem,
                                           uint64_t *bars, float *sphi) {
    using Gm = Tma3Geom<S>;
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int zlast = min(zend, nz - 1);          // last layer staged
    const int x = x0 + tx, y = y0 + ty;
    const size_t cxy = (size_t)y * nx + x;
    const size_t plane_cells = (size_t)nx * ny;

    // layer L lives in stage (L - zbeg) & 1; ph* = parity awaited next,
    // pend* = copies issued and not yet seen complete
    uint32_t ph0 = 0u, ph1 = 0u;
    bool pend0 = true, pend1 = zbeg + 1 <= zlast;
    if (tid == 0) {
        issue_layer<S>(smem, &bars[0], M, par, x0, y0, zbeg);
        if (pend1) issue_layer<S>(smem + Gm::STAGE, &bars[1], M, par, x0, y0, zbeg + 1);
    }
    auto wait_stage = [&](int st) -> bool {
        const bool ok = mbar_wait_bounded(&bars[st], st ? ph1 : ph0);
        if (ok) {
            if (st) { ph1 ^= 1u; pend1 = false; } else { ph0 ^= 1u; pend0 = false; }
        }
        return ok;
    };

    // window: plane zbeg - 1 with plain loads, plane zbeg from stage 0
    fill_plane<S, false>(sphi, zbeg % 3, zbeg - 1, false, false, 0.0f, pin, q_in, x0, y0, tid, tx, ty, P);
    bool ok = wait_stage(0);
    fill_plane<S, FXY>(sphi, (zbeg + 1) % 3, zbeg, true, true, staged_phid<S>(smem, tid, P), pin,
                       q_in, x0, y0, tid, tx, ty, P);

    for (int z = zbeg; z < zend; ++z) {
        const int st = (z - zbeg) & 1;
        const bool has_next = z + 1 < nz;
        float phn = 0.0f;
        if (has_next) {
            ok = wait_stage(st ^ 1) && ok;
            phn = staged_phid<S>(smem + (st ^ 1) * Gm::STAGE, tid, P);
        }
        fill_plane<S, FXY>(sphi, (z + 2) % 3, z + 1, true, has_next, phn, pin, q_in, x0, y0, tid,
                           tx, ty, P);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            if (pend0) mbar_wait_bounded(&bars[0], ph0);     // copies that may still land
            if (pend1) mbar_wait_bounded(&bars[1], ph1);
            return;
        }
        {
            const unsigned char *b = smem + st * Gm::STAGE;
            const S *F = (const S *)(b + Gm::OFF_F);
            const S *Sv = (const S *)(b + Gm::OFF_S);
            const S *G = (const S *)(b + Gm::OFF_G);
            float f[QF], s[QF], g[QG];
#pragma unroll
            for (int i = 0; i < QF; ++i) {
                f[i] = widen(F[i * Gm::CELLS + tid]);
                s[i] = widen(Sv[i * Gm::CELLS + tid]);
            }
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = widen(G[i * Gm::CELLS + tid]);
            const float qp = ((const float *)(b + Gm::OFF_Q))[tid];
            const float phip = ((const float *)(b + Gm::OFF_PP))[tid];
            const size_t c = (size_t)z * plane_cells + cxy;
            if (FXY && z >= 1 && z + 1 < nz)
                layer_update3d<S, true>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P);
            else
                layer_update3d<S, false>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P);
        }
        __syncthreads();      // stage st and window slot (z - 1) % 3 are free again
        if (z + 2 <= zlast) {
            if (tid == 0) issue_layer<S>(smem + st * Gm::STAGE, &bars[st], M, par, x0, y0, z + 2);
            if (st) pend1 = true; else pend0 = true;
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(TX * TY, 2)
step3d_tma_kernel(const __grid_constant__ TmaMaps3d maps, const S *__restrict__ pin,
                  S *__restrict__ pout, float *__restrict__ phi_prev,
                  const float *__restrict__ q_in, float *__restrict__ q_out, int par, int *err,
                  const DevParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies want 128-byte aligned destinations
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ float sphi[3 * PLANE];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    if (x0 + TX > P.n[0] || y0 + TY > P.n[1]) {          // ragged tile: plain loads
        step3d_column<S, false>(pin, pout, phi_prev, q_in, q_out, P, sphi);
        return;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool fxy = x0 >= 1 && x0 + TX + 1 <= P.n[0] && y0 >= 1 && y0 + TY + 1 <= P.n[1];
    if (fxy) tma_column<S, true>(maps, par, pin, pout, phi_prev, q_in, q_out, err, P, smem, bars, sphi);
    else tma_column<S, false>(maps, par, pin, pout, phi_prev, q_in, q_out, err, P, smem, bars, sphi);
}

// ------------------------------------------------------------------ host side
bool tma3d_eligible(const DevParams &P, int elem_bytes) {
    const long long nx = P.n[0], ny = P.n[1];
    if (nx < TX || ny < TY || P.n[2] < 1) return false;
    if ((nx * elem_bytes) % 16 != 0 || (nx * 4) % 16 != 0) return false;
    return true;
}

int make_tma_maps3d(TmaMaps3d *M, const DevParams &P, int elem_bytes, void *const pops[2],
                    float *const q[2], float *phi_prev) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const cuuint64_t nx = (cuuint64_t)P.n[0], ny = (cuuint64_t)P.n[1], nz = (cuuint64_t)P.n[2];
    const cuuint64_t N = (cuuint64_t)P.N, es = (cuuint64_t)elem_bytes;
    const cuuint32_t one[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    auto map4 = [&](CUtensorMap *m, void *base, cuuint32_t planes) {
        const cuuint64_t dims[4] = {nx, ny, nz, (cuuint64_t)(QF + QG + QF)};
        const cuuint64_t str[3] = {nx * es, nx * ny * es, N * es};
        const cuuint32_t box[4] = {TX, TY, 1, planes};
        return enc(m, dt, 4, base, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto map3 = [&](CUtensorMap *m, void *base) {
        const cuuint64_t dims[3] = {nx, ny, nz};
        const cuuint64_t str[2] = {nx * 4, nx * ny * 4};
        const cuuint32_t box[3] = {TX, TY, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, str, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
        if (!map4(&M->fs[b], pops[b], QF)) return -2;
        if (!map4(&M->g[b], pops[b], QG)) return -3;
        if (!map3(&M->q[b], q[b])) return -4;
    }
    if (!map3(&M->pp, phi_prev)) return -5;
    return 0;
}

template <typename S>
static int blocks_per_sm_for() {
    int n = 0;
    const int dyn = Tma3Geom<S>::DYN;
    if (cudaFuncSetAttribute(step3d_tma_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step3d_tma_kernel<S>, TX * TY, dyn) != cudaSuccess)
        return 0;
    return n;
}

int tma3d_blocks_per_sm(int elem_bytes) {
    if (elem_bytes == 4) return blocks_per_sm_for<float>();
    const int a = blocks_per_sm_for<__half>(), b = blocks_per_sm_for<__nv_bfloat16>();
    return a < b ? a : b;
}

template <typename S>
cudaError_t launch_step3d_tma(const TmaMaps3d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, cudaStream_t st) {
    dim3 block(TX, TY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, (P.n[2] + ZB - 1) / ZB);
    step3d_tma_kernel<S><<<grid, block, Tma3Geom<S>::DYN, st>>>(M, (const S *)pin, (S *)pout, phi_prev,
                                                                q_in, q_out, par, err, P);
    return cudaGetLastError();
}

#define LBM_INST3DTMA(S)                                                                        \
    template cudaError_t launch_step3d_tma<S>(const TmaMaps3d &, int, const void *, void *,     \
                                              float *, const float *, float *, int *,           \
                                              const DevParams &, cudaStream_t);
LBM_INST3DTMA(float)
LBM_INST3DTMA(__half)
LBM_INST3DTMA(__nv_bfloat16)

}  // namespace lbm
