// 3D kernels: D3Q19 for f and s, D3Q7 for the phase field g (Sec. 3
// lattices), stencils over the D3Q19 neighbours with factor 1/cs^2 = 3.
//
// The step kernel marches each 32x8 (x, y) column tile through a range of z
// planes.  Shared memory holds a rolling window of three planes of
// phi^n = sum_i gbar_i + q^{n-1}/2 (tile plus a one-cell halo ring): before
// layer z is updated, plane z+1 is computed; each thread keeps the gbar of
// its own cell of plane z+1 in registers for the next iteration.  The halo
// ring's gbar and q are re-read from L2, so populations cross HBM once.
// Everything else mirrors the 2D kernel (see lbm2d.cu): moments, closures,
// production rate, three BGK collisions and push streaming with wall links.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm3d.h"

namespace lbm {

using LF = D3Q19L;   // f and s
using LG = D3Q7L;    // g
constexpr int TX = 32, TY = 8, SX = TX + 2, SY = TY + 2, PLANE = SX * SY;
constexpr int ZB = 32;                       // z planes per block
constexpr int QF = 19, QG = 7;
constexpr int G0 = QF, S0 = QF + QG;         // first plane of g and of s

struct Macro3 {
    float phi, g[3], lap, rho, gr[3], F[3], u[3], p, T, Td;   // Td = T - T_ref
};

// nb[i] = phi(x + e_i) over the D3Q19 directions
__device__ __forceinline__ void stencil3d(const float nb[QF], float g[3], float &lap) {
    const float phi = nb[0];
    g[0] = g[1] = g[2] = 0.0f;
    lap = 0.0f;
#pragma unroll
    for (int i = 1; i < QF; ++i) {
        const float plus = nb[i], minus = nb[LF::opp(i)];
        const float dir = (plus - minus) * 0.5f;
        const float sec = plus - 2.0f * phi + minus;
        if (LF::ex(i) != 0) g[0] += (LF::w(i) * (float)LF::ex(i)) * dir;
        if (LF::ey(i) != 0) g[1] += (LF::w(i) * (float)LF::ey(i)) * dir;
        if (LF::ez(i) != 0) g[2] += (LF::w(i) * (float)LF::ez(i)) * dir;
        lap += LF::w(i) * sec;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] *= LF::inv_cs2;
    lap *= LF::inv_cs2;
}

__device__ __forceinline__ void closures3d(Macro3 &m, const DevParams &P) {
    const float phi = m.phi;
    m.rho = density(phi, P);
    const float mu = 4.0f * P.H * phi * (phi - 1.0f) * (phi - 0.5f) - P.K * m.lap;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.gr[a] = P.drho * m.g[a];
        m.F[a] = mu * m.g[a] + (m.rho - P.rho_l) * P.gravity[a] + P.body[a];
    }
}

__device__ __forceinline__ void moments3d(Macro3 &m, const float f[QF], const float s[QF],
                                          float phi_prev, float q_prev, const DevParams &P) {
    closures3d(m, P);
    float j[3] = {0.0f, 0.0f, 0.0f};
    float sf = f[0], ss = s[0];
#pragma unroll
    for (int i = 1; i < QF; ++i) {
        if (LF::ex(i) != 0) j[0] += (float)LF::ex(i) * f[i];
        if (LF::ey(i) != 0) j[1] += (float)LF::ey(i) * f[i];
        if (LF::ez(i) != 0) j[2] += (float)LF::ez(i) * f[i];
        sf += f[i];
        ss += s[i];
    }
    float ugr = 0.0f, ug = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.u[a] = (j[a] * LF::inv_cs2 + 0.5f * m.F[a]) / m.rho;
        ugr += m.u[a] * m.gr[a];
        ug += m.u[a] * m.g[a];
    }
    m.p = sf + 0.5f * (LF::cs2 * ugr + m.rho * LF::cs2 * q_prev * P.kappa);
    m.Td = ss - 0.5f * P.L_over_Cp * ((m.phi - phi_prev) + ug + m.phi * q_prev * P.kappa);
    m.T = m.Td + P.s_ref;
}

__device__ __forceinline__ void normal3d(const float g[3], float eps2, float n[3]) {
    const float d = sqrtf(fmaxf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2], eps2));
    n[0] = g[0] / d; n[1] = g[1] / d; n[2] = g[2] / d;
}

// Gamma_i (Eq. FunctionGamma) on lattice Lt with its own cs^2
template <class Lt>
__device__ __forceinline__ float gamma_i(int i, const float u[3], float usq) {
    const float cu = (float)Lt::ex(i) * u[0] + (float)Lt::ey(i) * u[1] + (float)Lt::ez(i) * u[2];
    return Lt::w(i) * (1.0f + cu * Lt::inv_cs2 + cu * cu * (0.5f * Lt::inv_cs2 * Lt::inv_cs2)
                       - usq * (0.5f * Lt::inv_cs2));
}

// barred equilibrium and source of g (D3Q7)
__device__ __forceinline__ void g_eq_src(int i, const Macro3 &m, const float n[3], float q, float usq,
                                         const DevParams &P, float &eqb, float &src) {
    const float G = gamma_i<LG>(i, m.u, usq);
    const float en = (float)LG::ex(i) * n[0] + (float)LG::ey(i) * n[1] + (float)LG::ez(i) * n[2];
    src = P.four_over_W * m.phi * (1.0f - m.phi) * LG::w(i) * en + LG::w(i) * q;
    eqb = m.phi * G - 0.5f * src;
}

// barred equilibria and sources of f and s (D3Q19)
__device__ __forceinline__ void fs_eq_src(int i, const Macro3 &m, float q, float D, float usq,
                                          const DevParams &P, float &feqb, float &fS, float &seqb,
                                          float &sS) {
    const float w = LF::w(i);
    const float e[3] = {(float)LF::ex(i), (float)LF::ey(i), (float)LF::ez(i)};
    const float cu = e[0] * m.u[0] + e[1] * m.u[1] + e[2] * m.u[2];
    const float poly = 3.0f * cu + 4.5f * cu * cu - 1.5f * usq;
    const float G = w * (1.0f + poly);
    const float Gw = G - w;
    float F = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) F += (e[a] - m.u[a]) * (Gw * m.gr[a] * LF::cs2 + G * m.F[a]);
    fS = F + w * m.rho * LF::cs2 * q * P.kappa;
    feqb = w * (m.p + m.rho * LF::cs2 * poly) - 0.5f * fS;
    sS = -w * P.L_over_Cp * D;
    seqb = m.Td * G + P.s_ref * (w * poly) - 0.5f * sS;   // deviation from w_i T_ref
}

// ------------------------------------------------------------------ step
template <typename S>
__device__ __forceinline__ float phi_at(const S *__restrict__ pin, const float *__restrict__ q_in,
                                        size_t cc, size_t N, const DevParams &P) {
    float v = Codec<S>::load(pin + G0 * N + cc, G0, P);
#pragma unroll
    for (int i = 1; i < QG; ++i) v += Codec<S>::load(pin + (G0 + i) * N + cc, G0 + i, P);
    return v + 0.5f * q_in[cc];
}

// Fill window slot `slot` with phi of plane z (tile + halo ring).  When
// owners_write is set, each thread whose column is inside the grid has
// already stored its own cell of an in-range plane (own_ok, own_phi);
// every other slot is computed here: phi of the wrapped cell, or the wall's
// Dirichlet value beyond a wall.
template <typename S>
__device__ __forceinline__ void fill_plane(float *sphi, int slot, int z, bool owners_write,
                                           bool own_ok, float own_phi, const S *__restrict__ pin,
                                           const float *__restrict__ q_in, int x0, int y0, int tid,
                                           int tx, int ty, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    float *plane = sphi + slot * PLANE;
    const bool z_in = z >= 0 && z < nz;
    if (owners_write && own_ok) plane[(ty + 1) * SX + tx + 1] = own_phi;
    for (int sidx = tid; sidx < PLANE; sidx += TX * TY) {
        const int sx = sidx % SX, sy = sidx / SX;
        int cx = x0 + sx - 1, cy = y0 + sy - 1, cz = z;
        const bool inner = sx >= 1 && sx <= TX && sy >= 1 && sy <= TY;
        if (owners_write && z_in && inner && cx < nx && cy < ny) continue;   // owner wrote it
        if (cx < -1 || cx > nx || cy < -1 || cy > ny || cz < -1 || cz > nz) { plane[sidx] = 0.0f; continue; }
        const int kx = wrap_coord(cx, nx, P.periodic[0]);
        const int ky = wrap_coord(cy, ny, P.periodic[1]);
        const int kz = wrap_coord(cz, nz, P.periodic[2]);
        float v;
        if (kx >= 2) v = P.phi_wall[kx - 2];
        else if (ky >= 2) v = P.phi_wall[ky - 2];
        else if (kz >= 2) v = P.phi_wall[kz - 2];
        else v = phi_at<S>(pin, q_in, ((size_t)cz * ny + cy) * nx + cx, N, P);
        plane[sidx] = v;
    }
}

template <typename S>
__global__ void __launch_bounds__(TX * TY, 1)
step3d_kernel(const S *__restrict__ pin, S *__restrict__ pout, float *__restrict__ phi_prev,
              const float *__restrict__ q_in, float *__restrict__ q_out, const DevParams P) {
    __shared__ float sphi[3 * PLANE];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = (x < nx) && (y < ny);
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;

    float g[QG], gn[QG], qcur = 0.0f, qnext = 0.0f;
    // prologue: plane zbeg (own cells kept in registers) and plane zbeg-1;
    // plane p lives in window slot (p + 1) % 3
    {
        float ph = 0.0f;
        if (col) {
            const size_t c = zbeg * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = Codec<S>::load(pin + (G0 + i) * N + c, G0 + i, P);
            qcur = q_in[c];
            ph = g[0];
#pragma unroll
            for (int i = 1; i < QG; ++i) ph += g[i];
            ph += 0.5f * qcur;
        }
        fill_plane<S>(sphi, (zbeg + 1) % 3, zbeg, true, col, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        fill_plane<S>(sphi, zbeg % 3, zbeg - 1, false, false, 0.0f, pin, q_in, x0, y0, tid, tx, ty, P);
    }

    for (int z = zbeg; z < zend; ++z) {
        // plane z+1 into the window
        {
            float ph = 0.0f;
            const bool ok = col && (z + 1 < nz);
            if (ok) {
                const size_t c = (size_t)(z + 1) * plane_cells + cxy;
#pragma unroll
                for (int i = 0; i < QG; ++i) gn[i] = Codec<S>::load(pin + (G0 + i) * N + c, G0 + i, P);
                qnext = q_in[c];
                ph = gn[0];
#pragma unroll
                for (int i = 1; i < QG; ++i) ph += gn[i];
                ph += 0.5f * qnext;
            }
            fill_plane<S>(sphi, (z + 2) % 3, z + 1, true, ok, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        }
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            float f[QF], s[QF];
#pragma unroll
            for (int i = 0; i < QF; ++i) f[i] = Codec<S>::load(pin + i * N + c, i, P);
#pragma unroll
            for (int i = 0; i < QF; ++i) s[i] = Codec<S>::load_dev(pin + (S0 + i) * N + c, S0 + i, P);
            const float phip = phi_prev[c];
            float nb[QF];
#pragma unroll
            for (int i = 0; i < QF; ++i) {
                const int slot = (z + 1 + LF::ez(i)) % 3;
                nb[i] = sphi[slot * PLANE + (ty + 1 + LF::ey(i)) * SX + tx + 1 + LF::ex(i)];
            }
            Macro3 m;
            m.phi = nb[0];
            stencil3d(nb, m.g, m.lap);
            moments3d(m, f, s, phip, qcur, P);
            const float q = production(m.phi, m.T, P);
            float n[3];
            normal3d(m.g, P.eps2, n);
            const float usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
            const float om_g = 1.0f / (P.tau_g + 0.5f);
            const float om_f = 1.0f / (viscosity(m.phi, P) * LF::inv_cs2 + 0.5f);
            const float om_s = 1.0f / (diffusivity(m.phi, P) * LF::inv_cs2 + 0.5f);
            const float D = (m.phi - phip) + (m.u[0] * m.g[0] + m.u[1] * m.g[1] + m.u[2] * m.g[2])
                          + m.phi * q * P.kappa;
            phi_prev[c] = m.phi;
            q_out[c] = q;
            // g on D3Q7
#pragma unroll
            for (int i = 0; i < QG; ++i) {
                float eqb, src;
                g_eq_src(i, m, n, q, usq, P, eqb, src);
                const float gs = g[i] - om_g * (g[i] - eqb) + src;
                int dx = x + LG::ex(i), dy = y + LG::ey(i), dz = z + LG::ez(i);
                const int kx = wrap_coord(dx, nx, P.periodic[0]);
                const int ky = wrap_coord(dy, ny, P.periodic[1]);
                const int kz = wrap_coord(dz, nz, P.periodic[2]);
                if (kx >= 2 || ky >= 2 || kz >= 2) {
                    const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
                    const int o = LG::opp(i);
                    Codec<S>::store(pout + (G0 + o) * N + c, -gs + 2.0f * LG::w(i) * P.phi_wall[side], G0 + o, P);
                } else {
                    const size_t d = ((size_t)dz * ny + dy) * nx + dx;
                    Codec<S>::store(pout + (G0 + i) * N + d, gs, G0 + i, P);
                }
            }
            // f and s on D3Q19
#pragma unroll
            for (int i = 0; i < QF; ++i) {
                float feqb, fS, seqb, sS;
                fs_eq_src(i, m, q, D, usq, P, feqb, fS, seqb, sS);
                const float fs = f[i] - om_f * (f[i] - feqb) + fS;
                const float sv = s[i] - om_s * (s[i] - seqb) + sS;
                int dx = x + LF::ex(i), dy = y + LF::ey(i), dz = z + LF::ez(i);
                const int kx = wrap_coord(dx, nx, P.periodic[0]);
                const int ky = wrap_coord(dy, ny, P.periodic[1]);
                const int kz = wrap_coord(dz, nz, P.periodic[2]);
                if (kx >= 2 || ky >= 2 || kz >= 2) {
                    const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
                    const int o = LF::opp(i);
                    Codec<S>::store(pout + o * N + c, fs, o, P);
                    Codec<S>::store_dev(pout + (S0 + o) * N + c, -sv + 2.0f * LF::w(i) * (P.T_wall[side] - P.s_ref), S0 + o, P);
                } else {
                    const size_t d = ((size_t)dz * ny + dy) * nx + dx;
                    Codec<S>::store(pout + i * N + d, fs, i, P);
                    Codec<S>::store_dev(pout + (S0 + i) * N + d, sv, S0 + i, P);
                }
            }
        }
        // rotate the own-cell registers to the next layer
#pragma unroll
        for (int i = 0; i < QG; ++i) g[i] = gn[i];
        qcur = qnext;
        __syncthreads();   // plane (z-1)%3 is overwritten next iteration
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

template <typename S>
__global__ void __launch_bounds__(256)
macro3d_kernel(const S *__restrict__ pin, const float *__restrict__ phi_f,
               const float *__restrict__ phi_prev, const float *__restrict__ q_in,
               float *o_phi, float *o_T, float *o_ux, float *o_uy, float *o_uz, float *o_p,
               double *partial, double Cp, double Lh, const DevParams P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double mass = 0.0, energy = 0.0;
    if (c < N) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((size_t)nx * ny));
        float nb[QF], f[QF], s[QF];
        gather_nb3d(phi_f, x, y, z, nb, P);
#pragma unroll
        for (int i = 0; i < QF; ++i) {
            f[i] = Codec<S>::load(pin + i * N + c, i, P);
            s[i] = Codec<S>::load_dev(pin + (S0 + i) * N + c, S0 + i, P);
        }
        Macro3 m;
        m.phi = nb[0];
        stencil3d(nb, m.g, m.lap);
        moments3d(m, f, s, phi_prev[c], q_in[c], P);
        if (o_phi) o_phi[c] = m.phi;
        if (o_T) o_T[c] = m.T;
        if (o_ux) o_ux[c] = m.u[0];
        if (o_uy) o_uy[c] = m.u[1];
        if (o_uz) o_uz[c] = m.u[2];
        if (o_p) o_p[c] = m.p;
        mass = (double)m.phi;
        energy = (double)m.rho * (Cp * (double)m.T + (double)m.phi * Lh);
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
        Codec<S>::store(pout + (G0 + i) * N + c, eqb, G0 + i, P);
    }
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        float feqb, fS, seqb, sS;
        fs_eq_src(i, m, q, D, usq, P, feqb, fS, seqb, sS);
        Codec<S>::store(pout + i * N + c, feqb, i, P);
        Codec<S>::store_dev(pout + (S0 + i) * N + c, seqb, S0 + i, P);
    }
    phi_prev[c] = m.phi;
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
    step3d_kernel<S><<<grid, block, 0, st>>>((const S *)pin, (S *)pout, phi_prev, q_in, q_out, P);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro3d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *const o_u[3],
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    phi3d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, q_in, phi_tmp, P);
    macro3d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, phi_tmp, phi_prev, q_in, o_phi, o_T,
                                          o_u[0], o_u[1], o_u[2], o_p, partial, Cp, Lh, P);
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
