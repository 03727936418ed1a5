// 3D phase field alone in an imposed velocity field (LBM_MODEL_PHASE_FIELD).
//
// The conservative Allen-Cahn scheme of Sec. 3.2 on the D3Q7 lattice of the
// coupled 3D model (cs^2 = 1/4), without phase change (q = 0) and with the
// velocity u(x) c(n) prescribed -- the CAC validations of Sec. 4.1 run on
// thin 3D domains.  Each block marches a 32x4 column tile through ZB layers
// with the rolling three-plane phi window of step3d_kernel: before layer z is
// updated, plane z+1 is formed (the own cell's g of plane z+1 stays in
// registers for the next layer, the halo ring comes from L2).  Per cell:
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

namespace lbm {

// update of one cell of layer z from the phi window (planes z-1, z, z+1 in
// slots z % 3, (z+1) % 3, (z+2) % 3) and its g values (working representation)
template <typename S, int MODE>
__device__ __forceinline__ void cac3d_cell(const float *sphi, int z, int x, int y, size_t c,
                                           const float g[QG], const float *__restrict__ vel, float factor,
                                           S *__restrict__ pout, const DevParams &P, const Planes3d<S> &PL) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t N = (size_t)P.N;
    const int centre = (ty + 1) * SX + tx + 1;
    const float *pl[3] = {sphi + (z % 3) * PLANE + centre, sphi + ((z + 1) % 3) * PLANE + centre,
                          sphi + ((z + 2) % 3) * PLANE + centre};
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
    const float u[3] = {vel[c] * factor, vel[N + c] * factor, vel[2 * N + c] * factor};
    const float usq = fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));

    const float om = P.om_g, a_g = 1.0f - om, b_g = fmaf(-0.5f, om, 1.0f);
    // 16-bit storage: the set's scale folded into the coefficients
    const float sg = IsNarrow<S>::value ? P.set_sc[1] : 1.0f;
    const float Ag = sg * (om * phd), Bg = sg * (om * ph);
    const float bgi = sg * (b_g * (P.four_over_W * ph * (1.0f - ph)));
    const float Vg[3] = {fmaf(4.0f * Bg, u[0], bgi * n[0]), fmaf(4.0f * Bg, u[1], bgi * n[1]),
                         fmaf(4.0f * Bg, u[2], bgi * n[2])};
    const float usq2 = 2.0f * usq;
    push3d_g<S, MODE>(0, fmaf(a_g, g[0], rep_mul3<S, LG>(0) * fmaf(Bg, -usq2, Ag)), x, y, z, c, pout, P, PL);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float Eg = fmaf(Bg, fmaf(8.0f * u[a], u[a], -usq2), Ag);
        const float mg = rep_mul3<S, LG>(a + 1);
        push3d_g<S, MODE>(a + 1, fmaf(a_g, g[a + 1], mg * (Eg + Vg[a])), x, y, z, c, pout, P, PL);
        push3d_g<S, MODE>(a + 4, fmaf(a_g, g[a + 4], mg * (Eg - Vg[a])), x, y, z, c, pout, P, PL);
    }
}

template <typename S, int XY>
__device__ __forceinline__ void cac3d_column(const S *__restrict__ pin, S *__restrict__ pout,
                                             const float *__restrict__ q_zero, const float *__restrict__ vel,
                                             float factor, const DevParams &P, float *sphi,
                                             const Planes3d<S> &PL) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = XY != XY_GEN || ((x < nx) && (y < ny));
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;
    const float isc = P.set_isc[1];

    float g[QG];
    {
        float ph = 0.0f;
        if (col) {
            const size_t c = zbeg * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = load_raw(PL.in[G0 + i] + c);
            ph = fmaf(0.5f, q_zero[c], set_sum7<S>(g, isc));
        }
        fill_plane<S, XY>(sphi, (zbeg + 1) % 3, zbeg, true, col, ph, pin, q_zero, x0, y0, tid, tx, ty, P);
        fill_plane<S, XY_GEN>(sphi, zbeg % 3, zbeg - 1, false, false, 0.0f, pin, q_zero, x0, y0, tid, tx, ty, P);
    }
    for (int z = zbeg; z < zend; ++z) {
        float gn[QG];
        {
            float ph = 0.0f;
            const bool ok = col && (z + 1 < nz);
            if (ok) {
                const size_t c = (size_t)(z + 1) * plane_cells + cxy;
#pragma unroll
                for (int i = 0; i < QG; ++i) gn[i] = load_raw(PL.in[G0 + i] + c);
                ph = fmaf(0.5f, q_zero[c], set_sum7<S>(gn, isc));
            }
            fill_plane<S, XY>(sphi, (z + 2) % 3, z + 1, true, ok, ph, pin, q_zero, x0, y0, tid, tx, ty, P);
        }
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            if (XY != XY_GEN && z >= 1 && z + 1 < nz)
                cac3d_cell<S, XY>(sphi, z, x, y, c, g, vel, factor, pout, P, PL);
            else
                cac3d_cell<S, XY_GEN>(sphi, z, x, y, c, g, vel, factor, pout, P, PL);
        }
#pragma unroll
        for (int i = 0; i < QG; ++i) g[i] = gn[i];
        __syncthreads();   // plane (z - 1) % 3 is overwritten next iteration
    }
}

template <typename S>
__global__ void __launch_bounds__(TX * TY, 8)
cac3d_kernel(const S *__restrict__ pin, S *__restrict__ pout, const float *__restrict__ q_zero,
             const float *__restrict__ vel, float factor, const DevParams P,
             const __grid_constant__ Planes3d<S> PL) {
    __shared__ float sphi[3 * PLANE];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int cls = tile_class3d(x0, y0, P);
    if (cls == XY_IN) cac3d_column<S, XY_IN>(pin, pout, q_zero, vel, factor, P, sphi, PL);
    else if (cls == XY_WRAP) cac3d_column<S, XY_WRAP>(pin, pout, q_zero, vel, factor, P, sphi, PL);
    else cac3d_column<S, XY_GEN>(pin, pout, q_zero, vel, factor, P, sphi, PL);
}

template <typename S>
cudaError_t launch_cac3d(const void *pin, void *pout, const float *q_zero, const float *vel, float factor,
                         const DevParams &P, cudaStream_t st) {
    dim3 block(TX, TY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, (P.n[2] + ZB - 1) / ZB);
    cac3d_kernel<S><<<grid, block, 0, st>>>((const S *)pin, (S *)pout, q_zero, vel, factor, P,
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
