// 2D D2Q9 kernels: the fused time step, the initialisation, the moments
// (fields and reductions) and the streaming-map test hook.
//
// State between steps (structure of arrays: the (f_i, s_i) pair planes, then
// the g planes, see off_f / off_g): the post-streaming populations of time n,
// phi^{n-1} and the lagged source q^{n-1} = mdot'''/rho_g of the previous
// collision.  One step is one launch of step2d_kernel:
//   1. every tile (32 x 4 cells for FP32, 64 x 4 for 16-bit storage)
//      computes phi^n = sum_i gbar_i + q^{n-1}/2 (Eq.
//      Moment_Phi) on the tile and a one-cell halo into shared memory; the
//      halo cells' gbar and q are re-read from L2, so each population
//      crosses HBM once per step;
//   2. each cell evaluates the stencils (Eqs. DerivDirec_Grad, Grad,
//      DerivDirect_Laplacian, Laplacian), the closures (Eqs. Density,
//      Viscosity, ChemicalPotential, SuperficialTensionForce, buoyancy), the
//      moments u, p, T (Eqs. Velocity, Pressure, Moment_Temp), the production
//      rate (Eq. ProductionRate) and the three BGK collisions in barred
//      variables (Eq. LBE with Eqs. Feq_NS_Incompr, Forcing, MicroProduction,
//      Geq_Allen-Cahn_Eq, SourceTerm_AllenCahn, Seq_Temp,
//      Def_SourceTerms_Temp), or their two-relaxation-time form (TRT
//      instantiation), or the multiple-relaxation-time collision of the
//      flow and phase-field sets with BGK for s (MRT instantiation), with the central
//      or the biased gradient (BIASED instantiation, a two-ring phi window);
//      The temperature set is advanced as deviations sbar_i - w_i T_ref
//      (the stored form), which keeps FP32 rounding relative to T - T_ref
//      rather than to T;
//   3. the post-collision values are pushed to x + e_i of the other
//      population buffer; a link that leaves through a wall comes back to the
//      same cell in the opposite direction, unchanged for f (half-way
//      bounce-back) and as -v + 2 w_i phi_w / T_w for g / s (anti
//      bounce-back, Sec. 3.3).
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm2d_cell.cuh"

namespace lbm {

// Tile of the tiled kernel per storage and gradient scheme, chosen by
// measurement on the 2048 x 4096 film (one thread per cell, 64 registers,
// 1024 threads per SM): FP32 32 x 4 (25.6k MLUPS against 24.9k for 32 x 8),
// 16-bit 64 x 4 (FP16 36.8k against 34.5k for 32 x 8, 33.0k for 64 x 8,
// 32.5k for 128 x 4) except with the MRT collision, which spills at 64
// registers and runs 32 x 4 (FP16 31.9k against 29.6k); the biased gradient
// 32 x 4 for 16-bit storage (FP16 32.7k against 31.0k for 64 x 4, 32.5k
// for 32 x 8) and 64 x 8 for FP32 (23.7k against 23.1k for 64 x 4, 22.5k
// for 32 x 8, 22.9k for 128 x 4).
template <typename S, bool BIASED, int COLL> struct StepTile { using T = Tile2<64, 4>; };
template <int COLL> struct StepTile<float, false, COLL> { using T = Tile2<32, 4>; };
template <int COLL> struct StepTile<float, true, COLL> { using T = Tile2<64, 8>; };
template <> struct StepTile<__half, false, COLL_MRT> { using T = Tile2<32, 4>; };
template <> struct StepTile<__nv_bfloat16, false, COLL_MRT> { using T = Tile2<32, 4>; };
template <int COLL> struct StepTile<__half, true, COLL> { using T = Tile2<32, 4>; };
template <int COLL> struct StepTile<__nv_bfloat16, true, COLL> { using T = Tile2<32, 4>; };

template <typename S, int COLL, bool BIASED>
__global__ void __launch_bounds__(StepTile<S, BIASED, COLL>::T::NT, 1024 / StepTile<S, BIASED, COLL>::T::NT)
step2d_kernel(const S *__restrict__ pin, S *__restrict__ pout, float *__restrict__ phi_prev,
              const float *__restrict__ q_in, float *__restrict__ q_out, const DevParams P,
              const __grid_constant__ Planes2d<S> PL) {
    using T = typename StepTile<S, BIASED, COLL>::T;
    __shared__ float sphi[BIASED ? (T::TY + 4) * (T::TX + 4) : T::SY * T::SX];
    pdl_wait();
    const int x0 = blockIdx.x * T::TX, y0 = blockIdx.y * T::TY;
    const bool fast = x0 >= 1 && x0 + T::TX + 1 <= P.n[0] && y0 >= 1 && y0 + T::TY + 1 <= P.n[1];
    if (BIASED) {
        if (fast) step2d_tile_biased<S, true, COLL, T>(pin, pout, phi_prev, q_in, q_out, P, sphi, x0, y0, PL);
        else step2d_tile_biased<S, false, COLL, T>(pin, pout, phi_prev, q_in, q_out, P, sphi, x0, y0, PL);
    } else {
        if (fast) step2d_tile<S, true, COLL, T>(pin, pout, phi_prev, q_in, q_out, P, sphi, x0, y0, PL);
        else step2d_tile<S, false, COLL, T>(pin, pout, phi_prev, q_in, q_out, P, sphi, x0, y0, PL);
    }
}

template <typename S, int COLL, bool BIASED>
static void launch_step2d_one(const S *in, S *out, float *phi_prev, const float *q_in, float *q_out,
                              const DevParams &P, const Planes2d<S> &PL, cudaStream_t st) {
    using T = typename StepTile<S, BIASED, COLL>::T;
    const dim3 block(T::TX, T::TY);
    const dim3 grid((P.n[0] + T::TX - 1) / T::TX, (P.n[1] + T::TY - 1) / T::TY);
    pdl_launch(step2d_kernel<S, COLL, BIASED>, grid, block, 0, st, in, out, phi_prev, q_in, q_out, P, PL);
}

// ------------------------------------------------------------------ phi moment
template <typename S>
__global__ void phi2d_kernel(const S *__restrict__ pin, const float *__restrict__ q_in,
                             float *__restrict__ phi_out, const DevParams P) {
    const size_t N = (size_t)P.N;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
        float v = Codec<S>::load(pin + off_g(9, 0, c, N), 9, P);
#pragma unroll
        for (int i = 1; i < 9; ++i) v += Codec<S>::load(pin + off_g(9, i, c, N), 9 + i, P);
        phi_out[c] = v + 0.5f * q_in[c];
    }
}

// phi(x + e_i) for i = 0..8 from a phi field, with wrap / wall ghosts
__device__ __forceinline__ void gather_nb2d(const float *__restrict__ phi, int x, int y, float nb[9],
                                            const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1];
    if (x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny) {
        // no neighbour wraps or lies beyond a wall
        const float *pc = phi + ((size_t)y * nx + x);
#pragma unroll
        for (int i = 0; i < 9; ++i) nb[i] = pc[L::ey(i) * nx + L::ex(i)];
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int cx = x + L::ex(i), cy = y + L::ey(i);
        const int kx = wrap_coord(cx, nx, P.periodic[0]);
        const int ky = wrap_coord(cy, ny, P.periodic[1]);
        if (kx >= 2) nb[i] = P.phi_wall[kx - 2];
        else if (ky >= 2) nb[i] = P.phi_wall[ky - 2];
        else nb[i] = phi[(size_t)cy * nx + cx];
    }
}

// With the biased option, grad(phi) from the phi field by the second-order
// biased difference (two ghost layers: the wall value beyond a wall,
// wrapped on periodic axes); nb holds the nine values one cell away.
__device__ __forceinline__ void biased_grad_field2d(const float *__restrict__ phi, int x, int y,
                                                    const float nb[9], const DevParams &P, float &gx,
                                                    float &gy) {
    const int nx = P.n[0], ny = P.n[1];
    float q[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int cx = x + 2 * L::ex(i), cy = y + 2 * L::ey(i);
        const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
        const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
        if (kx >= 2) q[i] = P.phi_wall[kx - 2];
        else if (ky >= 2) q[i] = P.phi_wall[ky - 2];
        else q[i] = phi[(size_t)cy * nx + cx];
    }
    // D2Q9 order: 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE
    biased_grad2d(nb[1], nb[3], nb[2], nb[4], nb[5], nb[6], nb[7], nb[8], q[1], q[3], q[2], q[4], q[5], q[6],
                  q[7], q[8], gx, gy);
}

// ------------------------------------------------------------------ moments
// Writes the requested fields (NULL pointers skipped) and, when partial is
// non-NULL, one FP64 (mass, enthalpy) pair per block.
template <typename S>
__global__ void __launch_bounds__(256)
macro2d_kernel(const S *__restrict__ pin, const float *__restrict__ phi_f,
               const float *__restrict__ phi_prev, const float *__restrict__ q_in,
               float *o_phi, float *o_T, float *o_ux, float *o_uy, float *o_p,
               double *partial, double Cp, double Lh, const DevParams P) {
    const int nx = P.n[0];
    const size_t N = (size_t)P.N;
    double mass = 0.0, energy = 0.0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        float nb[9], f[9], s[9];
        gather_nb2d(phi_f, x, y, nb, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = Codec<S>::load(pin + off_f(i, c, N), i, P);
            s[i] = Codec<S>::load_dev(pin + off_s(i, c, N), 18 + i, P);
        }
        Macro2 m;
        m.phi = nb[0];
        stencil2d(nb, m.gx, m.gy, m.lap);
        if (P.opts & OPT_BIASED) biased_grad_field2d(phi_f, x, y, nb, P, m.gx, m.gy);
        moments2d(m, f, s, phi_prev[c] + P.g_ref, q_in[c], P);
        if (o_phi) o_phi[c] = m.phi;
        if (o_T) o_T[c] = m.T;
        if (o_ux) o_ux[c] = m.ux;
        if (o_uy) o_uy[c] = m.uy;
        if (o_p) o_p[c] = m.p;
        mass += (double)m.phi;
        energy += (double)m.rho * (Cp * (double)m.T + (double)m.phi * Lh);
    }
    if (partial) block_sum2(mass, energy, partial);
}

// ------------------------------------------------------------------ init
template <typename S>
__global__ void __launch_bounds__(256)
init2d_kernel(const float *__restrict__ phi0, const float *__restrict__ T0,
              const float *__restrict__ ux0, const float *__restrict__ uy0,
              const float *__restrict__ p0, S *__restrict__ pout, float *__restrict__ phi_prev,
              float *__restrict__ q_out, const DevParams P) {
    const int nx = P.n[0];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % nx), y = (int)(c / nx);
    float nb[9];
    gather_nb2d(phi0, x, y, nb, P);
    Macro2 m;
    m.phi = nb[0];
    stencil2d(nb, m.gx, m.gy, m.lap);
    if (P.opts & OPT_BIASED) biased_grad_field2d(phi0, x, y, nb, P, m.gx, m.gy);
    closures2d(m, P);
    m.ux = ux0 ? ux0[c] : 0.0f;
    m.uy = uy0 ? uy0[c] : 0.0f;
    m.p = p0 ? p0[c] : 0.0f;
    m.T = T0[c];
    m.Td = m.T - P.s_ref;
    const float q = production(m.phi, m.T, P);
    float nx_, ny_;
    normal2d(m.gx, m.gy, P.eps2, nx_, ny_);
    const float D = (m.ux * m.gx + m.uy * m.gy) + m.phi * q * P.kappa;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const EqSrc e = eq_src2d(i, m, nx_, ny_, q, D, P);
        Codec<S>::store(pout + off_f(i, c, N), e.feq - 0.5f * e.fS, i, P);
        Codec<S>::store_dev(pout + off_g(9, i, c, N), e.geq - 0.5f * e.gS - L::w(i) * P.g_ref, 9 + i, P);
        Codec<S>::store_dev(pout + off_s(i, c, N), e.seq - 0.5f * e.sS, 18 + i, P);
    }
    phi_prev[c] = m.phi - P.g_ref;
    q_out[c] = q;
}

// ------------------------------------------------------------------ stream map
// Emulates the push of step2d_kernel for every (cell, direction) and records
// where each value lands, in pull form (see lbm_stream_map).
__global__ void streammap2d_kernel(int32_t *src, int8_t *kind, const DevParams P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % nx), y = (int)(c / nx);
    for (int i = 0; i < 9; ++i) {
        int dx = x + L::ex(i), dy = y + L::ey(i);
        const int kx = wrap_coord(dx, nx, P.periodic[0]);
        const int ky = wrap_coord(dy, ny, P.periodic[1]);
        if (kx >= 2 || ky >= 2) {
            const int o = L::opp(i);
            src[o * N + c] = (int32_t)c;
            kind[o * N + c] = (int8_t)(kx >= 2 ? kx : ky);
        } else {
            const size_t d = (size_t)dy * nx + dx;
            src[i * N + d] = (int32_t)c;
            kind[i * N + d] = (int8_t)((kx == 1 || ky == 1) ? 1 : 0);
        }
    }
}

// ------------------------------------------------------------------ launchers
template <typename S>
cudaError_t launch_step2d(const void *pin, void *pout, float *phi_prev, const float *q_in,
                          float *q_out, const DevParams &P, cudaStream_t st) {
    // the TRT and MRT collisions and the biased gradient are separate instantiations,
    // so the default kernel keeps its register allocation
    const S *in = (const S *)pin;
    S *out = (S *)pout;
    const Planes2d<S> PL = planes2d<S>(pin, pout, P);
    switch (P.opts & (OPT_TRT | OPT_MRT | OPT_BIASED)) {
    case 0: launch_step2d_one<S, COLL_BGK, false>(in, out, phi_prev, q_in, q_out, P, PL, st); break;
    case OPT_TRT: launch_step2d_one<S, COLL_TRT, false>(in, out, phi_prev, q_in, q_out, P, PL, st); break;
    case OPT_MRT: launch_step2d_one<S, COLL_MRT, false>(in, out, phi_prev, q_in, q_out, P, PL, st); break;
    case OPT_BIASED: launch_step2d_one<S, COLL_BGK, true>(in, out, phi_prev, q_in, q_out, P, PL, st); break;
    case OPT_TRT | OPT_BIASED:
        launch_step2d_one<S, COLL_TRT, true>(in, out, phi_prev, q_in, q_out, P, PL, st);
        break;
    case OPT_MRT | OPT_BIASED:
        launch_step2d_one<S, COLL_MRT, true>(in, out, phi_prev, q_in, q_out, P, PL, st);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro2d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *o_ux, float *o_uy,
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    phi2d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, q_in, phi_tmp, P);
    macro2d_kernel<S><<<moment_blocks(P.N), 256, 0, st>>>((const S *)pin, phi_tmp, phi_prev, q_in, o_phi,
                                                          o_T, o_ux, o_uy, o_p, partial, Cp, Lh, P);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init2d(const float *phi0, const float *T0, const float *ux0, const float *uy0,
                          const float *p0, void *pout, float *phi_prev, float *q_out,
                          const DevParams &P, cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    init2d_kernel<S><<<nb, 256, 0, st>>>(phi0, T0, ux0, uy0, p0, (S *)pout, phi_prev, q_out, P);
    return cudaGetLastError();
}

cudaError_t launch_streammap2d(int32_t *src, int8_t *kind, const DevParams &P, cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    streammap2d_kernel<<<nb, 256, 0, st>>>(src, kind, P);
    return cudaGetLastError();
}

#define LBM_INST2D(S)                                                                          \
    template cudaError_t launch_step2d<S>(const void *, void *, float *, const float *, float *, \
                                          const DevParams &, cudaStream_t);                    \
    template cudaError_t launch_macro2d<S>(const void *, float *, const float *, const float *, \
                                           float *, float *, float *, float *, float *, double *, \
                                           double, double, const DevParams &, cudaStream_t);    \
    template cudaError_t launch_init2d<S>(const float *, const float *, const float *,         \
                                          const float *, const float *, void *, float *, float *, \
                                          const DevParams &, cudaStream_t);
LBM_INST2D(float)
LBM_INST2D(__half)
LBM_INST2D(__nv_bfloat16)

}  // namespace lbm
