// 3D phase field alone in an imposed velocity field (LBM_MODEL_PHASE_FIELD).
//
// The conservative Allen-Cahn scheme of Sec. 3.2 on the D3Q7 lattice of the
// coupled 3D model (cs^2 = 1/4), without phase change (q = 0) and with the
// velocity u(x) c(n) prescribed -- the CAC validations of Sec. 4.1 run on
// thin 3D domains.  Each block marches a 32x8 column tile through ZB layers
// with a rolling phi window (four plane slots, one barrier per layer): before
// layer z is updated, plane z+1 is formed.  On tiles that need no wall test
// the loads run a layer ahead: while layer z is updated, the own cells' g of
// plane z+2 and the imposed velocity of layer z+1 are in flight in registers
// and the halo ring of plane z+2 is being copied into shared memory with
// cp.async (the per-layer work is small, so without the lookahead every
// layer waited for its loads).  There is no phase change, so phi = sum_i g_i
// and no lagged source is read.  Per cell:
// grad(phi) by Eqs. DerivDirec_Grad and Grad over the D3Q19 neighbours, the
// normal, Gamma(u) (Eq. FunctionGamma) and the collision of Eq. LBE with the
// source F^g of Eq. SourceTerm_AllenCahn in the even / odd form of the
// coupled step (E = Ag + Bg P_e, O = e.Vg, Ag = om (phi - phi_ref),
// Bg = om phi, Vg = 4 Bg u + (1 - om/2)(4/W) phi (1 - phi) n), then the push
// of the seven values.  Algorithmic bytes per cell: the g planes read and
// written and the three velocity components, 7 x 2 x (4 or 2) + 12.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm3d_cell.cuh"
#include "tma_util.cuh"

namespace lbm {

namespace {

// Slots of the phi window: plane p in slot (p + 1) % CW.  With four, the
// plane built for layer z + 1 never overwrites one that the slowest threads
// still read for layer z - 1, so one barrier per layer suffices (each
// thread reads back only the ring words it fetched itself).
constexpr int CW = 4;

// Column tile of this kernel: 32 x CTY cells (the coupled kernels use 32 x 4).
// The per-cell update is short, so the halo ring (84 cells for 256 owners
// here, 76 for 128 at a height of 4) is a large share of the work.
constexpr int CTY = 8, CSY = CTY + 2, CPLANE = SX * CSY, CTHREADS = TX * CTY;

// Halo ring of the phi window (one cell per thread r < CRING), fetched a
// layer ahead with 4-byte cp.async copies into shared memory: the 7 g values
// of ring cell r in words buf[i * CRING + r].  A 16-bit value is fetched as
// the aligned 32-bit word that holds it (the workspace is 256-byte aligned).
constexpr int CRING = 2 * SX + 2 * CTY;
constexpr int CRING_WORDS = QG * CRING;

__device__ __forceinline__ void cac_cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int XY>
__device__ __forceinline__ size_t cac_ring_cell(int r, int z, int x0, int y0, const DevParams &P, int &slot) {
    const int nx = P.n[0], ny = P.n[1];
    int sx, sy;
    if (r < SX) { sx = r; sy = 0; }
    else if (r < 2 * SX) { sx = r - SX; sy = CSY - 1; }
    else if (r < 2 * SX + CTY) { sx = 0; sy = 1 + r - 2 * SX; }
    else { sx = SX - 1; sy = 1 + r - 2 * SX - CTY; }
    slot = sy * SX + sx;
    int cx = x0 + sx - 1, cy = y0 + sy - 1;
    if (XY == XY_WRAP) {
        cx = cx < 0 ? cx + nx : (cx >= nx ? cx - nx : cx);
        cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
    }
    return ((size_t)z * ny + cy) * nx + cx;
}

// issue the ring copies of plane z (one commit group per call)
template <typename S, int XY>
__device__ __forceinline__ void cac_ring_prefetch(uint32_t *buf, const S *__restrict__ pin, int z, int x0,
                                                  int y0, int tid, const DevParams &P) {
    if (tid < CRING) {
        int slot;
        const size_t cc = cac_ring_cell<XY>(tid, z, x0, y0, P, slot);
        const size_t N = (size_t)P.N;
        if (in_bounds((long long)cc, (long long)N, P)) {
#pragma unroll
            for (int i = 0; i < QG; ++i) {
                const size_t e = off_g(QF, i, cc, N);
                const S *src = pin + (IsNarrow<S>::value ? (e & ~(size_t)1) : e);
                cac_cp_async4(&buf[i * CRING + tid], src);
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// phi - phi_ref of ring cell tid of plane z from its fetched words
template <typename S, int XY>
__device__ __forceinline__ void cac_ring_store(float *plane, const uint32_t *buf, int z, int x0, int y0,
                                               int tid, const DevParams &P) {
    if (tid >= CRING) return;
    int slot;
    const size_t cc = cac_ring_cell<XY>(tid, z, x0, y0, P, slot);
    const size_t N = (size_t)P.N;
    float v[QG];
    // element off_g(QF, i, cc, N) = (2 QF + i) N + cc sits in the high half of
    // its word when odd
    const uint32_t pc = (uint32_t)cc & 1u, pn = (uint32_t)N & 1u;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        const uint32_t w = buf[i * CRING + tid];
        if (IsNarrow<S>::value) {
            const uint32_t odd = pc ^ (pn & (uint32_t)((2 * QF + i) & 1));
            const unsigned short h = (unsigned short)(odd ? (w >> 16) : (w & 0xffffu));
            S val;
            memcpy(&val, &h, 2);
            v[i] = widen(val);
        } else {
            v[i] = __uint_as_float(w);
        }
    }
    plane[slot] = set_sum7<S>(v, P.set_isc[1]);
}

// Fast-path push of direction i's g value (tile class MODE = XY_IN or
// XY_WRAP): the x / y link as in the coupled kernel, and the z link moved by
// zup (ez = +1) or zdn (ez = -1) cells, +-N on the last / first layer of a
// periodic z axis and 0 elsewhere (N < 2^31, so the offsets fit an int).
template <typename S, int MODE>
__device__ __forceinline__ void cac_push_g(int i, float v, int x, int y, size_t c, int zup, int zdn,
                                           const DevParams &P, const Planes3d<S> &PL) {
    const int ex = LG::ex(i), ey = LG::ey(i), ez = LG::ez(i);
    int off = push_off3(ex, ey, ez, x, y, MODE == XY_WRAP, P);
    if (ez > 0) off += zup;
    if (ez < 0) off += zdn;
    if (!in_bounds((long long)c + off, (long long)P.N, P)) return;
    PL.out[G0 + i][(cidx)c + (cidx)off] = narrow<S>(v);
}

}  // namespace

// update of one cell of layer z from the phi window (planes z-1, z, z+1 in
// slots z % CW, (z+1) % CW, (z+2) % CW) and its g values (working representation)
template <typename S, int MODE>
__device__ __forceinline__ void cac3d_cell(const float *sphi, int z, int x, int y, size_t c,
                                           const float g[QG], const float *__restrict__ vel, float factor,
                                           const float uin[3], bool have_u, int zup, int zdn,
                                           S *__restrict__ pout, const DevParams &P, const Planes3d<S> &PL) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t N = (size_t)P.N;
    const int centre = (ty + 1) * SX + tx + 1;
    const float *pl[3] = {sphi + (z % CW) * CPLANE + centre, sphi + ((z + 1) % CW) * CPLANE + centre,
                          sphi + ((z + 2) % CW) * CPLANE + centre};
    const float phd = pl[1][0];
    const float ph = phd + P.g_ref;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k);
        const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
        const float d = pl[1 + ez][ey * SX + ex] - pl[1 - ez][-ey * SX - ex];
        if (ex != 0) gx += sgnv(ex, d) * LF::w(i);
        if (ey != 0) gy += sgnv(ey, d) * LF::w(i);
        if (ez != 0) gz += sgnv(ez, d) * LF::w(i);
    }
    gx *= 3.0f; gy *= 3.0f; gz *= 3.0f;
    const float inv_d = rsqrt_approx(fmaxf(fmaf(gz, gz, fmaf(gy, gy, gx * gx)), P.eps2));
    const float n[3] = {gx * inv_d, gy * inv_d, gz * inv_d};
    // the imposed velocity (already loaded a layer ahead when have_u)
    const float u[3] = {(have_u ? uin[0] : vel[c]) * factor, (have_u ? uin[1] : vel[N + c]) * factor,
                        (have_u ? uin[2] : vel[2 * N + c]) * factor};
    const float usq = fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));

    const float om = P.om_g, a_g = 1.0f - om, b_g = fmaf(-0.5f, om, 1.0f);
    // 16-bit storage: the set's scale folded into the coefficients
    const float sg = IsNarrow<S>::value ? P.set_sc[1] : 1.0f;
    const float Ag = sg * (om * phd), Bg = sg * (om * ph);
    const float bgi = sg * (b_g * (P.four_over_W * ph * (1.0f - ph)));
    const float Vg[3] = {fmaf(4.0f * Bg, u[0], bgi * n[0]), fmaf(4.0f * Bg, u[1], bgi * n[1]),
                         fmaf(4.0f * Bg, u[2], bgi * n[2])};
    const float usq2 = 2.0f * usq;
    auto push = [&](int i, float v) {
        if (MODE == XY_GEN) push3d_g<S, MODE>(i, v, x, y, z, c, pout, P, PL);
        else cac_push_g<S, MODE>(i, v, x, y, c, zup, zdn, P, PL);
    };
    push(0, fmaf(a_g, g[0], rep_mul3<S, LG>(0) * fmaf(Bg, -usq2, Ag)));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float Eg = fmaf(Bg, fmaf(8.0f * u[a], u[a], -usq2), Ag);
        const float mg = rep_mul3<S, LG>(a + 1);
        push(a + 1, fmaf(a_g, g[a + 1], mg * (Eg + Vg[a])));
        push(a + 4, fmaf(a_g, g[a + 4], mg * (Eg - Vg[a])));
    }
}

template <typename S, int XY>
__device__ __forceinline__ void cac3d_column(const S *__restrict__ pin, S *__restrict__ pout,
                                             const float *__restrict__ q_zero, const float *__restrict__ vel,
                                             float factor, const DevParams &P, float *sphi,
                                             uint32_t (*rbuf)[CRING_WORDS], const Planes3d<S> &PL) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * CTY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = XY != XY_GEN || ((x < nx) && (y < ny));
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;
    const size_t N = (size_t)P.N;
    const float isc = P.set_isc[1];
    // lookahead on tiles that need no wall test (q = 0: phi = sum_i g_i)
    constexpr bool PRE = XY != XY_GEN;

    // gn: the own g of plane z + 1 as stored (a 16-bit value is widened only
    // where it is used, so the load it came from is not waited for early)
    float g[QG], u[3] = {0.0f, 0.0f, 0.0f};
    S gn[QG];
    {
        float ph = 0.0f;
        if (col) {
            const size_t c = zbeg * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = load_raw(PL.in[G0 + i] + c);
            ph = PRE ? set_sum7<S>(g, isc) : fmaf(0.5f, q_zero[c], set_sum7<S>(g, isc));
            if (PRE) for (int a = 0; a < 3; ++a) u[a] = vel[a * N + c];
        }
        fill_plane<S, XY, CTY>(sphi, (zbeg + 1) % CW, zbeg, true, col, ph, pin, q_zero, x0, y0, tid, tx, ty, P);
        fill_plane<S, XY_GEN, CTY>(sphi, zbeg % CW, zbeg - 1, false, false, 0.0f, pin, q_zero, x0, y0, tid, tx, ty, P);
        if (PRE && zbeg + 1 < nz) {
            const size_t c = (size_t)(zbeg + 1) * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) gn[i] = __ldg(PL.in[G0 + i] + c);
            cac_ring_prefetch<S, XY>(rbuf[(zbeg + 1) & 1], pin, zbeg + 1, x0, y0, tid, P);
        }
    }
    for (int z = zbeg; z < zend; ++z) {
        S gnn[QG];
        float un[3] = {0.0f, 0.0f, 0.0f};
        if (PRE) {
            // in flight during this layer: plane z + 2 and the velocity of z + 1
            if (z + 2 < nz) {
                const size_t c2 = (size_t)(z + 2) * plane_cells + cxy;
#pragma unroll
                for (int i = 0; i < QG; ++i) gnn[i] = __ldg(PL.in[G0 + i] + c2);
                cac_ring_prefetch<S, XY>(rbuf[z & 1], pin, z + 2, x0, y0, tid, P);
            }
            if (z + 1 < zend) {
                const size_t c1 = (size_t)(z + 1) * plane_cells + cxy;
                for (int a = 0; a < 3; ++a) un[a] = vel[a * N + c1];
            }
            // plane z + 1 (in range: its own values and ring arrived a layer ago)
            if (z + 1 < nz) {
                float *plane = sphi + ((z + 2) % CW) * CPLANE;
                float v[QG];
#pragma unroll
                for (int i = 0; i < QG; ++i) v[i] = widen(gn[i]);
                plane[(ty + 1) * SX + tx + 1] = set_sum7<S>(v, isc);
                if (z + 2 < nz) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else asm volatile("cp.async.wait_group 0;" ::: "memory");
                cac_ring_store<S, XY>(plane, rbuf[(z + 1) & 1], z + 1, x0, y0, tid, P);
            } else {
                fill_plane<S, XY, CTY>(sphi, (z + 2) % CW, z + 1, true, false, 0.0f, pin, q_zero, x0, y0, tid, tx, ty, P);
            }
        } else {
            float ph = 0.0f;
            const bool ok = col && (z + 1 < nz);
            if (ok) {
                const size_t c = (size_t)(z + 1) * plane_cells + cxy;
                float v[QG];
#pragma unroll
                for (int i = 0; i < QG; ++i) { gn[i] = __ldg(PL.in[G0 + i] + c); v[i] = widen(gn[i]); }
                ph = fmaf(0.5f, q_zero[c], set_sum7<S>(v, isc));
            }
            fill_plane<S, XY, CTY>(sphi, (z + 2) % CW, z + 1, true, ok, ph, pin, q_zero, x0, y0, tid, tx, ty, P);
        }
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            // the first and last layers of a periodic z axis take the fast
            // push too, with the z link wrapped; beside a z wall the generic one
            if (XY != XY_GEN && ((z >= 1 && z + 1 < nz) || P.periodic[2])) {
                const int zup = z + 1 == nz ? -(int)N : 0, zdn = z == 0 ? (int)N : 0;
                cac3d_cell<S, XY>(sphi, z, x, y, c, g, vel, factor, u, PRE, zup, zdn, pout, P, PL);
            } else {
                cac3d_cell<S, XY_GEN>(sphi, z, x, y, c, g, vel, factor, u, PRE, 0, 0, pout, P, PL);
            }
        }
#pragma unroll
        for (int i = 0; i < QG; ++i) { g[i] = widen(gn[i]); if (PRE) gn[i] = gnn[i]; }
        if (PRE) for (int a = 0; a < 3; ++a) u[a] = un[a];
    }
    if (PRE) asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename S>
__global__ void __launch_bounds__(CTHREADS, 4)
cac3d_kernel(const S *__restrict__ pin, S *__restrict__ pout, const float *__restrict__ q_zero,
             const float *__restrict__ vel, float factor, const DevParams P,
             const __grid_constant__ Planes3d<S> PL) {
    __shared__ float sphi[CW * CPLANE];
    __shared__ uint32_t rbuf[2][CRING_WORDS];
    pdl_wait();
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * CTY;
    const int cls = tile_class3d<CTY>(x0, y0, P);
    if (cls == XY_IN) cac3d_column<S, XY_IN>(pin, pout, q_zero, vel, factor, P, sphi, rbuf, PL);
    else if (cls == XY_WRAP) cac3d_column<S, XY_WRAP>(pin, pout, q_zero, vel, factor, P, sphi, rbuf, PL);
    else cac3d_column<S, XY_GEN>(pin, pout, q_zero, vel, factor, P, sphi, rbuf, PL);
}

template <typename S>
cudaError_t launch_cac3d(const void *pin, void *pout, const float *q_zero, const float *vel, float factor,
                         const DevParams &P, cudaStream_t st) {
    dim3 block(TX, CTY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + CTY - 1) / CTY, (P.n[2] + ZB - 1) / ZB);
    pdl_launch(cac3d_kernel<S>, grid, block, 0, st, (const S *)pin, (S *)pout, q_zero, vel, factor, P,
               planes3d<S>(pin, pout, P));
    return cudaGetLastError();
}

template cudaError_t launch_cac3d<float>(const void *, void *, const float *, const float *, float,
                                         const DevParams &, cudaStream_t);
template cudaError_t launch_cac3d<__half>(const void *, void *, const float *, const float *, float,
                                          const DevParams &, cudaStream_t);
template cudaError_t launch_cac3d<__nv_bfloat16>(const void *, void *, const float *, const float *, float,
                                                 const DevParams &, cudaStream_t);

}  // namespace lbm
