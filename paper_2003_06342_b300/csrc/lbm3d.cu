// 3D kernels: D3Q19 for f and s, D3Q7 for the phase field g (Sec. 3
// lattices), stencils over the D3Q19 neighbours with factor 1/cs^2 = 3.
//
// The step kernel marches each 32x4 (x, y) column tile through a range of z
// planes.  Shared memory holds a rolling window of three planes of
// phi^n = sum_i gbar_i + q^{n-1}/2 (tile plus a one-cell halo ring): before
// layer z is updated, plane z+1 is computed; each thread keeps the gbar of
// its own cell of plane z+1 in registers for the next iteration.  The halo
// ring's gbar and q are re-read from L2, so populations cross HBM once.
// Everything else mirrors the 2D kernel (see lbm2d.cu): moments, closures,
// production rate, three BGK (or TRT / MRT) collisions and push streaming with wall
// links.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm3d.h"
#include "lbm3d_cell.cuh"

namespace lbm {

template <typename S, int COLL, bool BIASED>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
step3d_kernel(const S *__restrict__ pin, S *__restrict__ pout, float *__restrict__ phi_prev,
              const float *__restrict__ q_in, float *__restrict__ q_out, const DevParams P,
              const __grid_constant__ Planes3d<S> PL) {
    __shared__ float sphi[BIASED ? NWB * PLANEB : NW3 * PLANE];
    pdl_wait();
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int cls = tile_class3d(x0, y0, P);
    if (BIASED) {
        if (cls == XY_IN) step3d_column_biased<S, XY_IN, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
        else if (cls == XY_WRAP) step3d_column_biased<S, XY_WRAP, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
        else step3d_column_biased<S, XY_GEN, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
    } else {
        if (cls == XY_IN) step3d_column<S, XY_IN, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
        else if (cls == XY_WRAP) step3d_column<S, XY_WRAP, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
        else step3d_column<S, XY_GEN, COLL>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
    }
}

// ------------------------------------------------------------------ phi moment
template <typename S>
__global__ void phi3d_kernel(const S *__restrict__ pin, const float *__restrict__ q_in,
                             float *__restrict__ phi_out, const DevParams P) {
    const size_t N = (size_t)P.N;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x)
        phi_out[c] = phi_at<S>(pin, q_in, c, N, P);
}

__device__ __forceinline__ void gather_nb3d(const float *__restrict__ phi, int x, int y, int z,
                                            float nb[QF], const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    if (x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny && z >= 1 && z + 1 < nz) {
        // no neighbour wraps or lies beyond a wall
        const float *pc = phi + (((size_t)z * ny + y) * nx + x);
        const long long plane = (long long)nx * ny;
#pragma unroll
        for (int i = 0; i < QF; ++i) nb[i] = pc[LF::ez(i) * plane + LF::ey(i) * nx + LF::ex(i)];
        return;
    }
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        int cx = x + LF::ex(i), cy = y + LF::ey(i), cz = z + LF::ez(i);
        const int kx = wrap_coord(cx, nx, P.periodic[0]);
        const int ky = wrap_coord(cy, ny, P.periodic[1]);
        const int kz = wrap_coord(cz, nz, P.periodic[2]);
        if (kx >= 2) nb[i] = P.phi_wall[kx - 2];
        else if (ky >= 2) nb[i] = P.phi_wall[ky - 2];
        else if (kz >= 2) nb[i] = P.phi_wall[kz - 2];
        else nb[i] = phi[((size_t)cz * ny + cy) * nx + cx];
    }
}

// With the biased option, grad(phi) from the phi field by the second-order
// biased difference of Eq. Grad (two ghost layers: the wall value beyond a
// wall, wrapped on periodic axes); nb holds the values one cell away.
__device__ __forceinline__ void biased_grad_field3d(const float *__restrict__ phi, int x, int y, int z,
                                                    const float nb[QF], const DevParams &P, float g[3]) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    float q[QF];
#pragma unroll
    for (int i = 1; i < QF; ++i) {
        int cx = x + 2 * LF::ex(i), cy = y + 2 * LF::ey(i), cz = z + 2 * LF::ez(i);
        const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
        const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
        const int kz = wrap_coord_far(cz, nz, P.periodic[2]);
        if (kx >= 2) q[i] = P.phi_wall[kx - 2];
        else if (ky >= 2) q[i] = P.phi_wall[ky - 2];
        else if (kz >= 2) q[i] = P.phi_wall[kz - 2];
        else q[i] = phi[((size_t)cz * ny + cy) * nx + cx];
    }
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k), o = LF::opp(i);
        const float d = 0.5f * fmaf(4.0f, nb[i] - nb[o], -(q[i] - q[o]));
        if (LF::ex(i) != 0) gx += sgnv(LF::ex(i), d) * LF::w(i);
        if (LF::ey(i) != 0) gy += sgnv(LF::ey(i), d) * LF::w(i);
        if (LF::ez(i) != 0) gz += sgnv(LF::ez(i), d) * LF::w(i);
    }
    g[0] = 3.0f * gx; g[1] = 3.0f * gy; g[2] = 3.0f * gz;
}

template <typename S>
__global__ void __launch_bounds__(256)
macro3d_kernel(const S *__restrict__ pin, const float *__restrict__ phi_f,
               const float *__restrict__ phi_prev, const float *__restrict__ q_in,
               float *o_phi, float *o_T, float *o_ux, float *o_uy, float *o_uz, float *o_p,
               double *partial, double Cp, double Lh, const DevParams P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    double mass = 0.0, energy = 0.0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
        float nb[QF], f[QF], s[QF];
        gather_nb3d(phi_f, x, y, z, nb, P);
#pragma unroll
        for (int i = 0; i < QF; ++i) {
            f[i] = Codec<S>::load(pin + off_f(i, c, N), i, P);
            s[i] = Codec<S>::load_dev(pin + off_s(i, c, N), S0 + i, P);
        }
        Macro3 m;
        m.phi = nb[0];
        stencil3d(nb, m.g, m.lap);
        if (P.opts & OPT_BIASED) biased_grad_field3d(phi_f, x, y, z, nb, P, m.g);
        moments3d(m, f, s, phi_prev[c] + P.g_ref, q_in[c], P);
        if (o_phi) o_phi[c] = m.phi;
        if (o_T) o_T[c] = m.T;
        if (o_ux) o_ux[c] = m.u[0];
        if (o_uy) o_uy[c] = m.u[1];
        if (o_uz) o_uz[c] = m.u[2];
        if (o_p) o_p[c] = m.p;
        mass += (double)m.phi;
        energy += (double)m.rho * (Cp * (double)m.T + (double)m.phi * Lh);
    }
    if (partial) block_sum2(mass, energy, partial);
}

template <typename S>
__global__ void __launch_bounds__(256)
init3d_kernel(const float *__restrict__ phi0, const float *__restrict__ T0,
              const float *__restrict__ ux0, const float *__restrict__ uy0,
              const float *__restrict__ uz0, const float *__restrict__ p0, S *__restrict__ pout,
              float *__restrict__ phi_prev, float *__restrict__ q_out, const DevParams P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
    float nb[QF];
    gather_nb3d(phi0, x, y, z, nb, P);
    Macro3 m;
    m.phi = nb[0];
    stencil3d(nb, m.g, m.lap);
    if (P.opts & OPT_BIASED) biased_grad_field3d(phi0, x, y, z, nb, P, m.g);
    closures3d(m, P);
    m.u[0] = ux0 ? ux0[c] : 0.0f;
    m.u[1] = uy0 ? uy0[c] : 0.0f;
    m.u[2] = uz0 ? uz0[c] : 0.0f;
    m.p = p0 ? p0[c] : 0.0f;
    m.T = T0[c];
    m.Td = m.T - P.s_ref;
    const float q = production(m.phi, m.T, P);
    float n[3];
    normal3d(m.g, P.eps2, n);
    const float usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    const float D = (m.u[0] * m.g[0] + m.u[1] * m.g[1] + m.u[2] * m.g[2]) + m.phi * q * P.kappa;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        float eqb, src;
        g_eq_src(i, m, n, q, usq, P, eqb, src);
        Codec<S>::store_dev(pout + off_g(QF, i, c, N), eqb - LG::w(i) * P.g_ref, G0 + i, P);
    }
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        float feqb, fS, seqb, sS;
        fs_eq_src(i, m, q, D, usq, P, feqb, fS, seqb, sS);
        Codec<S>::store(pout + off_f(i, c, N), feqb, i, P);
        Codec<S>::store_dev(pout + off_s(i, c, N), seqb, S0 + i, P);
    }
    phi_prev[c] = m.phi - P.g_ref;
    q_out[c] = q;
}

// push emulation for the stream-map hook; set 0 = D3Q19 (f, s), 1 = D3Q7 (g)
template <class Lt>
__global__ void streammap3d_kernel(int32_t *src, int8_t *kind, const DevParams P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
    for (int i = 0; i < Lt::Q; ++i) {
        int dx = x + Lt::ex(i), dy = y + Lt::ey(i), dz = z + Lt::ez(i);
        const int kx = wrap_coord(dx, nx, P.periodic[0]);
        const int ky = wrap_coord(dy, ny, P.periodic[1]);
        const int kz = wrap_coord(dz, nz, P.periodic[2]);
        if (kx >= 2 || ky >= 2 || kz >= 2) {
            const int o = Lt::opp(i);
            src[o * N + c] = (int32_t)c;
            kind[o * N + c] = (int8_t)(kx >= 2 ? kx : (ky >= 2 ? ky : kz));
        } else {
            const size_t d = ((size_t)dz * ny + dy) * nx + dx;
            src[i * N + d] = (int32_t)c;
            kind[i * N + d] = (int8_t)((kx == 1 || ky == 1 || kz == 1) ? 1 : 0);
        }
    }
}

// ------------------------------------------------------------------ launchers
template <typename S>
cudaError_t launch_step3d(const void *pin, void *pout, float *phi_prev, const float *q_in,
                          float *q_out, const DevParams &P, cudaStream_t st) {
    dim3 block(TX, TY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, (P.n[2] + ZB - 1) / ZB);
    const S *in = (const S *)pin;
    S *out = (S *)pout;
    const Planes3d<S> PL = planes3d<S>(pin, pout, P);
    switch (P.opts & (OPT_TRT | OPT_MRT | OPT_BIASED)) {
    case 0: pdl_launch(step3d_kernel<S, COLL_BGK, false>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL); break;
    case OPT_TRT: pdl_launch(step3d_kernel<S, COLL_TRT, false>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL); break;
    case OPT_MRT: pdl_launch(step3d_kernel<S, COLL_MRT, false>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL); break;
    case OPT_BIASED: pdl_launch(step3d_kernel<S, COLL_BGK, true>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL); break;
    case OPT_TRT | OPT_BIASED:
        pdl_launch(step3d_kernel<S, COLL_TRT, true>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL);
        break;
    case OPT_MRT | OPT_BIASED:
        pdl_launch(step3d_kernel<S, COLL_MRT, true>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro3d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *const o_u[3],
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    phi3d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, q_in, phi_tmp, P);
    macro3d_kernel<S><<<moment_blocks(P.N), 256, 0, st>>>((const S *)pin, phi_tmp, phi_prev, q_in, o_phi,
                                                          o_T, o_u[0], o_u[1], o_u[2], o_p, partial, Cp,
                                                          Lh, P);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init3d(const float *phi0, const float *T0, const float *const u0[3],
                          const float *p0, void *pout, float *phi_prev, float *q_out,
                          const DevParams &P, cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    init3d_kernel<S><<<nb, 256, 0, st>>>(phi0, T0, u0[0], u0[1], u0[2], p0, (S *)pout, phi_prev,
                                         q_out, P);
    return cudaGetLastError();
}

cudaError_t launch_streammap3d(int set, int32_t *src, int8_t *kind, const DevParams &P,
                               cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    if (set == 0) streammap3d_kernel<LF><<<nb, 256, 0, st>>>(src, kind, P);
    else streammap3d_kernel<LG><<<nb, 256, 0, st>>>(src, kind, P);
    return cudaGetLastError();
}

#define LBM_INST3D(S)                                                                          \
    template cudaError_t launch_step3d<S>(const void *, void *, float *, const float *, float *, \
                                          const DevParams &, cudaStream_t);                    \
    template cudaError_t launch_macro3d<S>(const void *, float *, const float *, const float *, \
                                           float *, float *, float *const[3], float *, double *, \
                                           double, double, const DevParams &, cudaStream_t);    \
    template cudaError_t launch_init3d<S>(const float *, const float *, const float *const[3], \
                                          const float *, void *, float *, float *,             \
                                          const DevParams &, cudaStream_t);
LBM_INST3D(float)
LBM_INST3D(__half)
LBM_INST3D(__nv_bfloat16)

}  // namespace lbm
