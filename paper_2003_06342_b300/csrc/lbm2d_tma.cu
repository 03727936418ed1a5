// 2D step marching in y with every chunk staged by bulk tensor copies.
//
// Same update as step2d_kernel (lbm2d.cu), organised like the 3D z-march
// (lbm3d_tma.cu): each block owns a strip of 32 columns and walks YC chunks
// of 8 rows through it.  One thread issues cp.async.bulk.tensor copies of a
// chunk into shared-memory stages:
//   f/s stage  (f_i, s_i) pair planes 32 x 8 x 9 from (x0, y0, 0)
//                                                   3D map (x, y, pair plane)
//              phi^{n-1} 32 x 8    from (x0, y0)       2D map (x, y)
//   g stage    g planes 32 x 8 x 9 from (x0, y0, 0)    3D map (x, y, g plane)
//              q^{n-1}  32 x 8     from (x0, y0)
// completing on the stage's mbarrier.  Two f/s stages and three g stages
// rotate so that every copy is issued a whole chunk before it is awaited
// (chunk c needs f/s of c and g of c and c + 1, the latter for the row below
// it).  The phi window of a chunk (10 rows x 34 columns) takes its top row
// from the previous chunk's window, its own rows and the row below from the g
// stages, and only the 18 cells of the left and right halo columns from
// global memory, fetched a chunk ahead with cp.async.  So the populations
// never wait in registers and the halo costs 18 instead of 84 cells a tile.
// Strips whose halo leaves the grid in x, and chunks that touch the first or
// last row of the grid, take the generic path of the tiled kernel (plain
// loads, periodic wrap, wall links) on the same window buffer.
//
// Waits on the mbarriers are bounded: on expiry the block records an error in
// a device word, waits (bounded) for its copies in flight and returns; the
// host reports LBM_ETIMEOUT at the next sync.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm2d_cell.cuh"
#include "lbm2d_tma.h"
#include "tma_util.cuh"

namespace lbm {

constexpr int YC = 4;                       // chunks of TY rows per block
constexpr int RING2 = 2 * (TY + 1);         // halo-column cells of window rows 1..9
constexpr int RWORDS = 10 * RING2;          // 9 g words + q per cell

template <typename S> struct March2Geom {
    static constexpr int ES = (int)sizeof(S);
    static constexpr int CELLS = TX * TY;
    static constexpr int al(int b) { return (b + 127) / 128 * 128; }
    static constexpr int P_BYTES = 9 * CELLS * ES;        // one set of a chunk
    static constexpr int Q_BYTES = CELLS * 4;
    static constexpr int OFF_FS = 0;                       // pairs (f_i, s_i)
    static constexpr int OFF_PP = OFF_FS + al(2 * P_BYTES);
    static constexpr int FS_STAGE = OFF_PP + al(Q_BYTES);
    static constexpr int OFF_G = 0;
    static constexpr int OFF_Q = OFF_G + al(P_BYTES);
    static constexpr int G_STAGE = OFF_Q + al(Q_BYTES);
    static constexpr int NFS = 2, NG = 3;
    static constexpr int G_BASE = NFS * FS_STAGE;
    static constexpr unsigned FS_TX = 2 * P_BYTES + Q_BYTES;
    static constexpr unsigned G_TX = P_BYTES + Q_BYTES;
    static constexpr int DYN = NFS * FS_STAGE + NG * G_STAGE + 128;   // + alignment slack
};

template <typename S>
__device__ __forceinline__ void issue_fs2(unsigned char *stage, uint64_t *bar, const TmaMaps2d &M,
                                          int par, int x0, int y0) {
    using Gm = March2Geom<S>;
    // order earlier generic-proxy reads of this stage before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::FS_TX);
    tma_load_3d(stage + Gm::OFF_FS, &M.fs[par], x0, y0, 0, bar);
    tma_load_2d(stage + Gm::OFF_PP, &M.pp, x0, y0, bar);
}

template <typename S>
__device__ __forceinline__ void issue_g2(unsigned char *stage, uint64_t *bar, const TmaMaps2d &M,
                                         int par, int x0, int y0) {
    using Gm = March2Geom<S>;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::G_TX);
    tma_load_3d(stage + Gm::OFF_G, &M.g[par], x0, y0, 0, bar);
    tma_load_2d(stage + Gm::OFF_Q, &M.q[par], x0, y0, bar);
}

// phi - phi_ref of cell `k` of a staged chunk (same arithmetic as phid_cell2d)
template <typename S>
__device__ __forceinline__ float staged_phid2(const unsigned char *gstage, int k, const DevParams &P) {
    using Gm = March2Geom<S>;
    const S *G = (const S *)(gstage + Gm::OFF_G);
    float v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = widen(G[i * Gm::CELLS + k]);
    return fmaf(0.5f, ((const float *)(gstage + Gm::OFF_Q))[k], set_sum2d<S>(v, P.set_isc[1]));
}

// Polls allowed to the first mbarrier wait of every block (all later waits
// take WAIT_LIMIT).  The default is WAIT_LIMIT; the timeout test lowers it to
// zero through set_first_wait_limit2d, so that every block gives up at its
// first stage, waits for the copies it issued, records the timeout in the
// status word and returns (no copy is left in flight).
static __device__ int first_wait_limit = WAIT_LIMIT;

cudaError_t set_first_wait_limit2d(int polls) {
    const int v = polls < 0 ? WAIT_LIMIT : polls;
    return cudaMemcpyToSymbol(first_wait_limit, &v, sizeof(int));
}

struct StageBits {
    uint32_t par = 0u, pend = 0u;     // parity awaited next / copies in flight, per barrier
    __device__ __forceinline__ bool wait(uint64_t *bars, int b, int limit = WAIT_LIMIT) {
        const bool ok = mbar_wait_bounded(&bars[b], (par >> b) & 1u, limit);
        if (ok) { par ^= 1u << b; pend &= ~(1u << b); }
        return ok;
    }
    __device__ __forceinline__ void drain(uint64_t *bars, int n) {
        for (int b = 0; b < n; ++b)
            if ((pend >> b) & 1u) mbar_wait_bounded(&bars[b], (par >> b) & 1u);
    }
};

__device__ __forceinline__ void cp_async4_2d(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// halo-column cell r of a chunk starting at row y0 (rows y0 .. y0 + TY): its
// grid cell and its window slot
__device__ __forceinline__ size_t ring2_cell(int r, int x0, int y0, int nx, int &slot) {
    const int side = r / (TY + 1), row = r % (TY + 1);
    slot = (row + 1) * SX + (side ? SX - 1 : 0);
    return (size_t)(y0 + row) * nx + (side ? x0 + TX : x0 - 1);
}

// fetch the halo columns of the chunk at row y0 into buf (one cell per thread
// r < RING2; a 16-bit value as the aligned 32-bit word that holds it)
template <typename S>
__device__ __forceinline__ void ring2_prefetch(uint32_t *buf, const S *__restrict__ pin,
                                               const float *__restrict__ q_in, int x0, int y0,
                                               int tid, const DevParams &P) {
    if (tid >= RING2) return;
    int slot;
    const size_t cc = ring2_cell(tid, x0, y0, P.n[0], slot);
    const size_t N = (size_t)P.N;
    if (!in_bounds((long long)cc, (long long)N, P)) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const size_t e = off_g(9, i, cc, N);
        cp_async4_2d(&buf[i * RING2 + tid], pin + (IsNarrow<S>::value ? (e & ~(size_t)1) : e));
    }
    cp_async4_2d(&buf[9 * RING2 + tid], q_in + cc);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename S>
__device__ __forceinline__ void ring2_store(float *win, const uint32_t *buf, int x0, int y0, int tid,
                                            const DevParams &P) {
    if (tid >= RING2) return;
    int slot;
    const size_t cc = ring2_cell(tid, x0, y0, P.n[0], slot);
    const size_t N = (size_t)P.N;
    float v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const uint32_t w = buf[i * RING2 + tid];
        if (IsNarrow<S>::value) {
            const size_t e = off_g(9, i, cc, N);
            const unsigned short h = (unsigned short)((e & 1) ? (w >> 16) : (w & 0xffffu));
            S val;
            memcpy(&val, &h, 2);
            v[i] = widen(val);
        } else {
            v[i] = __uint_as_float(w);
        }
    }
    win[slot] = fmaf(0.5f, __uint_as_float(buf[9 * RING2 + tid]), set_sum2d<S>(v, P.set_isc[1]));
}

template <typename S, int COLL>
__global__ void __launch_bounds__(TX * TY, 3)
step2d_tma_kernel(const __grid_constant__ TmaMaps2d maps, const S *__restrict__ pin,
                  S *__restrict__ pout, float *__restrict__ phi_prev,
                  const float *__restrict__ q_in, float *__restrict__ q_out, int par, int *err,
                  const DevParams P, const __grid_constant__ Planes2d<S> PL) {
    using Gm = March2Geom<S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies want 128-byte aligned destinations
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t barF[Gm::NFS], barG[Gm::NG];
    pdl_wait();
    __shared__ float win[2][SY * SX];
    __shared__ uint32_t rbuf[2][RWORDS];
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX;
    const int ybeg = blockIdx.y * (TY * YC);
    const int nc = min(YC, (ny - ybeg + TY - 1) / TY);
    const bool xin = x0 >= 1 && x0 + TX + 1 <= nx;

    if (!xin) {     // strip at (or beyond) the x edges: generic tiles, plain loads
        for (int c = 0; c < nc; ++c) {
            step2d_tile<S, false, COLL>(pin, pout, phi_prev, q_in, q_out, P, win[0], x0, ybeg + c * TY, PL);
            __syncthreads();
        }
        return;
    }
    auto fast = [&](int c) {     // chunk c needs no wrap or wall (rows y0 - 1 .. y0 + TY inside)
        const int y0 = ybeg + c * TY;
        return y0 >= 1 && y0 + TY + 1 <= ny;
    };
    unsigned char *fs_base = smem;
    unsigned char *g_base = smem + Gm::G_BASE;
    if (tid == 0) {
        for (int k = 0; k < Gm::NFS; ++k) mbar_init(&barF[k], 1);
        for (int k = 0; k < Gm::NG; ++k) mbar_init(&barG[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // every chunk of the strip is staged (rows past the grid read as zero)
    StageBits F, G;
    for (int k = 0; k < Gm::NFS; ++k)
        if (k < nc) F.pend |= 1u << k;
    for (int k = 0; k < Gm::NG; ++k)
        if (k < nc) G.pend |= 1u << k;
    if (tid == 0) {
        for (int k = 0; k < Gm::NG; ++k)
            if (k < nc) issue_g2<S>(g_base + k * Gm::G_STAGE, &barG[k], maps, par, x0, ybeg + k * TY);
        for (int k = 0; k < Gm::NFS; ++k)
            if (k < nc) issue_fs2<S>(fs_base + k * Gm::FS_STAGE, &barF[k], maps, par, x0, ybeg + k * TY);
    }
    bool ok = G.wait(barG, 0, first_wait_limit);

    int fb = 0, gb = 0;                     // stages of chunk c
    for (int c = 0; c < nc; ++c) {
        const int y0 = ybeg + c * TY;
        const int gn = gb == Gm::NG - 1 ? 0 : gb + 1;
        const bool fc = fast(c);
        float *W = win[c & 1];
        if (c + 1 < nc) ok = G.wait(barG, gn) && ok;
        ok = F.wait(barF, fb) && ok;
        if (fc) {
            // top row: the previous chunk's row TY (its window row 8), or loaded
            if (tid < SX) {
                if (c > 0) {
                    W[tid] = win[(c - 1) & 1][TY * SX + tid];
                } else {
                    const size_t cc = (size_t)(y0 - 1) * nx + (x0 + tid - 1);
                    W[tid] = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
                }
            }
            // own rows from this chunk's g stage
            W[(ty + 1) * SX + tx + 1] = staged_phid2<S>(g_base + gb * Gm::G_STAGE, tid, P);
            // the row below: row 0 of the next chunk's stage, or loaded
            if (tid < TX) {
                float v;
                if (c + 1 < nc) {
                    v = staged_phid2<S>(g_base + gn * Gm::G_STAGE, tid, P);
                } else {
                    const size_t cc = (size_t)(y0 + TY) * nx + (x0 + tid);
                    v = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
                }
                W[(TY + 1) * SX + tid + 1] = v;
            }
            // halo columns of rows 1 .. TY + 1
            if (c > 0) {
                asm volatile("cp.async.wait_all;" ::: "memory");
                ring2_store<S>(W, rbuf[c & 1], x0, y0, tid, P);
            } else if (tid < RING2) {
                int slot;
                const size_t cc = ring2_cell(tid, x0, y0, nx, slot);
                W[slot] = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, 1);
            asm volatile("cp.async.wait_all;" ::: "memory");
            F.drain(barF, Gm::NFS);                 // copies that may still land
            G.drain(barG, Gm::NG);
            return;
        }
        // the next chunk's halo columns, a chunk ahead
        if (c + 1 < nc && fast(c + 1))
            ring2_prefetch<S>(rbuf[(c + 1) & 1], pin, q_in, x0, y0 + TY, tid, P);
        if (fc) {
            const unsigned char *b = fs_base + fb * Gm::FS_STAGE;
            const unsigned char *bg = g_base + gb * Gm::G_STAGE;
            const auto *FSp = (const typename PairOf<S>::T *)(b + Gm::OFF_FS);
            const S *Gp = (const S *)(bg + Gm::OFF_G);
            float f[9], g[9], s[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                unpack_pair(FSp[i * Gm::CELLS + tid], f[i], s[i]);
                g[i] = widen(Gp[i * Gm::CELLS + tid]);
            }
            const float qp = ((const float *)(bg + Gm::OFF_Q))[tid];
            const float phip = ((const float *)(b + Gm::OFF_PP))[tid];
            const int x = x0 + tx, y = y0 + ty;
            cell_update2d<S, true, COLL>(W + (ty + 1) * SX + tx + 1, SX, f, g, s, phip, qp, x, y,
                                   (size_t)y * nx + x, pout, phi_prev, q_out, P, PL);
        } else {
            // first or last rows of the grid (or a ragged chunk): generic tile
            // on the same window buffer, so the next chunk can take its top row
            step2d_tile<S, false, COLL>(pin, pout, phi_prev, q_in, q_out, P, W, x0, y0, PL);
        }
        __syncthreads();      // the stages of chunk c and window c - 1 are free again
        if (c + Gm::NFS < nc) {
            if (tid == 0)
                issue_fs2<S>(fs_base + fb * Gm::FS_STAGE, &barF[fb], maps, par, x0, ybeg + (c + Gm::NFS) * TY);
            F.pend |= 1u << fb;
        }
        if (c + Gm::NG < nc) {
            if (tid == 0)
                issue_g2<S>(g_base + gb * Gm::G_STAGE, &barG[gb], maps, par, x0, ybeg + (c + Gm::NG) * TY);
            G.pend |= 1u << gb;
        }
        fb ^= 1;
        gb = gn;
    }
}

// ------------------------------------------------------------------ host side
bool tma2d_eligible(const DevParams &P, int elem_bytes) {
    const long long nx = P.n[0], ny = P.n[1];
    if (nx < TX || ny < TY) return false;
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
    const cuuint32_t one[3] = {1, 1, 1};
    // a single value, and a (f_i, s_i) pair copied as one element of twice the size
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const CUtensorMapDataType dt2 = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    // 9 planes of `e` bytes per element, rows nx elements apart, planes pstride bytes apart
    auto map3 = [&](CUtensorMap *m, void *base, CUtensorMapDataType t, cuuint64_t e, cuuint64_t pstride) {
        const cuuint64_t dims[3] = {nx, ny, 9};
        const cuuint64_t str[2] = {nx * e, pstride};
        const cuuint32_t box[3] = {TX, TY, 9};
        return enc(m, t, 3, base, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto map2 = [&](CUtensorMap *m, void *base) {
        const cuuint64_t dims[2] = {nx, ny};
        const cuuint64_t str[1] = {nx * 4};
        const cuuint32_t box[2] = {TX, TY};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, str, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
        if (!map3(&M->fs[b], pops[b], dt2, 2 * es, 2 * N * es)) return -2;
        if (!map3(&M->g[b], (char *)pops[b] + off_g(9, 0, 0, N) * es, dt, es, N * es)) return -2;
        if (!map2(&M->q[b], q[b])) return -3;
    }
    if (!map2(&M->pp, phi_prev)) return -4;
    return 0;
}

template <typename S, int COLL>
static int blocks_per_sm_one2() {
    int n = 0;
    const int dyn = March2Geom<S>::DYN;
    if (cudaFuncSetAttribute(step2d_tma_kernel<S, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step2d_tma_kernel<S, COLL>, TX * TY, dyn) != cudaSuccess)
        return 0;
    return n;
}

// every collision instantiation gets the shared-memory limit
template <typename S>
static int blocks_per_sm_for2() {
    const int a = blocks_per_sm_one2<S, COLL_BGK>(), b = blocks_per_sm_one2<S, COLL_TRT>();
    const int c = blocks_per_sm_one2<S, COLL_MRT>();
    const int ab = a < b ? a : b;
    return ab < c ? ab : c;
}

int tma2d_blocks_per_sm(int elem_bytes) {
    if (elem_bytes == 4) return blocks_per_sm_for2<float>();
    const int a = blocks_per_sm_for2<__half>(), b = blocks_per_sm_for2<__nv_bfloat16>();
    return a < b ? a : b;
}

template <typename S>
cudaError_t launch_step2d_tma(const TmaMaps2d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, cudaStream_t st) {
    dim3 block(TX, TY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY * YC - 1) / (TY * YC));
    if (P.opts & OPT_TRT)
        pdl_launch(step2d_tma_kernel<S, COLL_TRT>, grid, block, March2Geom<S>::DYN, st, M, (const S *)pin,
                   (S *)pout, phi_prev, q_in, q_out, par, err, P, planes2d<S>(pin, pout, P));
    else if (P.opts & OPT_MRT)
        pdl_launch(step2d_tma_kernel<S, COLL_MRT>, grid, block, March2Geom<S>::DYN, st, M, (const S *)pin,
                   (S *)pout, phi_prev, q_in, q_out, par, err, P, planes2d<S>(pin, pout, P));
    else
        pdl_launch(step2d_tma_kernel<S, COLL_BGK>, grid, block, March2Geom<S>::DYN, st, M, (const S *)pin,
                   (S *)pout, phi_prev, q_in, q_out, par, err, P, planes2d<S>(pin, pout, P));
    return cudaGetLastError();
}

#define LBM_INST2DTMA(S)                                                                        \
    template cudaError_t launch_step2d_tma<S>(const TmaMaps2d &, int, const void *, void *,     \
                                              float *, const float *, float *, int *,           \
                                              const DevParams &, cudaStream_t);
LBM_INST2DTMA(float)
LBM_INST2DTMA(__half)
LBM_INST2DTMA(__nv_bfloat16)

}  // namespace lbm
