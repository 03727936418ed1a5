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
// phi - phi_ref at one cell (the step works on the phase field's deviation)
template <typename S>
__device__ __forceinline__ float phid_at(const S *__restrict__ pin, const float *__restrict__ q_in,
                                         size_t cc, size_t N, const DevParams &P) {
    float v = Codec<S>::load_dev(pin + G0 * N + cc, G0, P);
#pragma unroll
    for (int i = 1; i < QG; ++i) v += Codec<S>::load_dev(pin + (G0 + i) * N + cc, G0 + i, P);
    return v + 0.5f * q_in[cc];
}

template <typename S>
__device__ __forceinline__ float phi_at(const S *__restrict__ pin, const float *__restrict__ q_in,
                                        size_t cc, size_t N, const DevParams &P) {
    return phid_at<S>(pin, q_in, cc, N, P) + P.g_ref;
}

// Fill window slot `slot` with phi of plane z (tile + halo ring).  When
// owners_write is set, each thread whose column is inside the grid has
// already stored its own cell of an in-range plane (own_ok, own_phi); every
// other slot is computed here: phi of the wrapped cell, or the wall's
// Dirichlet value beyond a wall.  FXY: the tile's halo ring lies inside the
// grid in x and y, so an in-range plane needs no wrap or wall test.
template <typename S, bool FXY>
__device__ __forceinline__ void fill_plane(float *sphi, int slot, int z, bool owners_write,
                                           bool own_ok, float own_phi, const S *__restrict__ pin,
                                           const float *__restrict__ q_in, int x0, int y0, int tid,
                                           int tx, int ty, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    float *plane = sphi + slot * PLANE;
    const bool z_in = z >= 0 && z < nz;
    if (owners_write && own_ok) plane[(ty + 1) * SX + tx + 1] = own_phi;
    if (FXY && z_in && owners_write) {
        constexpr int RING = 2 * SX + 2 * TY;
        if (tid < RING) {
            int sx, sy;
            if (tid < SX) { sx = tid; sy = 0; }
            else if (tid < 2 * SX) { sx = tid - SX; sy = SY - 1; }
            else if (tid < 2 * SX + TY) { sx = 0; sy = 1 + tid - 2 * SX; }
            else { sx = SX - 1; sy = 1 + tid - 2 * SX - TY; }
            const size_t cc = ((size_t)z * ny + (y0 + sy - 1)) * nx + (x0 + sx - 1);
            plane[sy * SX + sx] = phid_at<S>(pin, q_in, cc, N, P);
        }
        return;
    }
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
        if (kx >= 2) v = P.phi_wall[kx - 2] - P.g_ref;
        else if (ky >= 2) v = P.phi_wall[ky - 2] - P.g_ref;
        else if (kz >= 2) v = P.phi_wall[kz - 2] - P.g_ref;
        else v = phid_at<S>(pin, q_in, ((size_t)cz * ny + cy) * nx + cx, N, P);
        plane[sidx] = v;
    }
}

__device__ __forceinline__ float sgnv(int e, float v) { return e > 0 ? v : -v; }
// e.(a, b, c) for e in {-1, 0, 1}^3 without multiplications
__device__ __forceinline__ float edot3(int ex, int ey, int ez, float a, float b, float c) {
    float r = 0.0f;
    bool any = false;
    if (ex != 0) { r = sgnv(ex, a); any = true; }
    if (ey != 0) { r = any ? r + sgnv(ey, b) : sgnv(ey, b); any = true; }
    if (ez != 0) { r = any ? r + sgnv(ez, c) : sgnv(ez, c); }
    return r;
}

// positive half of the D3Q19 directions: each pair (i, opposite) once
__device__ __forceinline__ constexpr int half19(int k) {
    return k < 3 ? k + 1 : (k < 5 ? k + 4 : (k < 7 ? k + 6 : k + 8));   // 1,2,3,7,8,11,12,15,16
}

// Update of one cell of layer z: stencils from the three window planes,
// moments, closures, production, the three collisions (theta* = (1 - om)
// theta + om theta_eq + (1 - om/2) S, identical to Eq. LBE), then the push.
// FAST: no link of this cell wraps or meets a wall.
template <typename S, bool FAST>
__device__ __forceinline__ void layer_update3d(const float *sphi, int z, int x, int y, size_t c,
                                               const float f[QF], const float s[QF],
                                               const float g[QG], float qp,
                                               S *__restrict__ pout, float *__restrict__ phi_prev,
                                               float *__restrict__ q_out, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int centre = (ty + 1) * SX + tx + 1;
    const float *pl[3] = {sphi + (z % 3) * PLANE + centre, sphi + ((z + 1) % 3) * PLANE + centre,
                          sphi + ((z + 2) % 3) * PLANE + centre};   // planes z-1, z, z+1
    Macro3 m;
    const float phd = pl[1][0];              // the window holds phi - phi_ref
    const float ph = phd + P.g_ref;
    m.phi = ph;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f, la = 0.0f, ld = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k);
        const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
        const float a = pl[1 + ez][ey * SX + ex], b = pl[1 - ez][-ey * SX - ex];
        const float d = a - b, sm = a + b;
        if (ex != 0) gx += sgnv(ex, d) * LF::w(i);
        if (ey != 0) gy += sgnv(ey, d) * LF::w(i);
        if (ez != 0) gz += sgnv(ez, d) * LF::w(i);
        if (i <= 6) la += sm; else ld += sm;
    }
    m.g[0] = 3.0f * gx; m.g[1] = 3.0f * gy; m.g[2] = 3.0f * gz;
    m.lap = 6.0f * ((1.0f / 18.0f) * (la - 6.0f * phd) + (1.0f / 36.0f) * (ld - 12.0f * phd));
    closures3d(m, P);
    float jx = 0.0f, jy = 0.0f, jz = 0.0f, sf = f[0], ss = s[0];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k), o = LF::opp(i);
        const float d = f[i] - f[o];
        if (LF::ex(i) != 0) jx += sgnv(LF::ex(i), d);
        if (LF::ey(i) != 0) jy += sgnv(LF::ey(i), d);
        if (LF::ez(i) != 0) jz += sgnv(LF::ez(i), d);
    }
#pragma unroll
    for (int i = 1; i < QF; ++i) { sf += f[i]; ss += s[i]; }
    const float inv_rho = __frcp_rn(m.rho);
    m.u[0] = (3.0f * jx + 0.5f * m.F[0]) * inv_rho;
    m.u[1] = (3.0f * jy + 0.5f * m.F[1]) * inv_rho;
    m.u[2] = (3.0f * jz + 0.5f * m.F[2]) * inv_rho;
    const float rcs2 = m.rho * LF::cs2;
    const float ugr = m.u[0] * m.gr[0] + m.u[1] * m.gr[1] + m.u[2] * m.gr[2];
    const float ug = m.u[0] * m.g[0] + m.u[1] * m.g[1] + m.u[2] * m.g[2];
    const float phip = phi_prev[c];
    m.p = sf + 0.5f * (LF::cs2 * ugr + rcs2 * qp * P.kappa);
    m.Td = ss - 0.5f * P.L_over_Cp * ((phd - phip) + ug + ph * qp * P.kappa);
    m.T = m.Td + P.s_ref;
    const float q = production(ph, m.T, P);
    const float inv_d = __frcp_rn(sqrtf(fmaxf(m.g[0] * m.g[0] + m.g[1] * m.g[1] + m.g[2] * m.g[2], P.eps2)));
    const float n0 = m.g[0] * inv_d, n1 = m.g[1] * inv_d, n2 = m.g[2] * inv_d;
    const float om_g = P.om_g;
    const float om_f = __frcp_rn(viscosity(ph, P) * LF::inv_cs2 + 0.5f);
    const float om_s = __frcp_rn(diffusivity(ph, P) * LF::inv_cs2 + 0.5f);
    const float D = (phd - phip) + ug + ph * q * P.kappa;
    phi_prev[c] = phd;           // stored as phi - phi_ref
    q_out[c] = q;

    const float usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    const float iface = P.four_over_W * ph * (1.0f - ph);
    const float a_g = 1.0f - om_g, b_g = 1.0f - 0.5f * om_g;
    const float a_f = 1.0f - om_f, b_f = 1.0f - 0.5f * om_f;
    const float a_s = 1.0f - om_s, b_s = 1.0f - 0.5f * om_s;

    // phase field on D3Q7 (cs^2 = 1/4): Gamma_i = w (1 + 4 cu + 8 cu^2 - 2 u^2)
    const float usq2 = 2.0f * usq;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        const int ex = LG::ex(i), ey = LG::ey(i), ez = LG::ez(i);
        const float w = LG::w(i);
        const float cu = edot3(ex, ey, ez, m.u[0], m.u[1], m.u[2]);
        const float poly = cu * fmaf(8.0f, cu, 4.0f) - usq2;
        const float G = fmaf(w, poly, w);
        const float Sg = w * (i == 0 ? q : fmaf(iface, edot3(ex, ey, ez, n0, n1, n2), q));
        const float gs = fmaf(a_g, g[i], fmaf(om_g, fmaf(phd, G, P.g_ref * (G - w)), b_g * Sg));
        int dx = x + ex, dy = y + ey, dz = z + ez;
        if (FAST) {
            const long long off = ((long long)ez * ny + ey) * nx + ex;
            Codec<S>::store_dev(pout + (G0 + i) * N + c + off, gs, G0 + i, P);
        } else {
            const int kx = wrap_coord(dx, nx, P.periodic[0]);
            const int ky = wrap_coord(dy, ny, P.periodic[1]);
            const int kz = wrap_coord(dz, nz, P.periodic[2]);
            if (kx >= 2 || ky >= 2 || kz >= 2) {
                const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
                const int o = LG::opp(i);
                Codec<S>::store_dev(pout + (G0 + o) * N + c, -gs + 2.0f * w * (P.phi_wall[side] - P.g_ref), G0 + o, P);
            } else {
                const size_t d = ((size_t)dz * ny + dy) * nx + dx;
                Codec<S>::store_dev(pout + (G0 + i) * N + d, gs, G0 + i, P);
            }
        }
    }

    // flow and temperature on D3Q19 (cs^2 = 1/3)
    const float usq15 = 1.5f * usq;
    const float gA0 = LF::cs2 * m.gr[0], gA1 = LF::cs2 * m.gr[1], gA2 = LF::cs2 * m.gr[2];
    const float uA = m.u[0] * gA0 + m.u[1] * gA1 + m.u[2] * gA2;
    const float uB = m.u[0] * m.F[0] + m.u[1] * m.F[1] + m.u[2] * m.F[2];
    const float pf = rcs2 * q * P.kappa;
    const float bsw = b_s * (-P.L_over_Cp * D);
    const float Tref = P.s_ref;
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
        const float w = LF::w(i);
        const float cu = edot3(ex, ey, ez, m.u[0], m.u[1], m.u[2]);
        const float poly = cu * fmaf(4.5f, cu, 3.0f) - usq15;
        const float G = fmaf(w, poly, w);
        const float Gw = w * poly;
        const float feq = w * fmaf(rcs2, poly, m.p);
        const float eA = (i == 0) ? 0.0f : edot3(ex, ey, ez, gA0, gA1, gA2);
        const float eB = (i == 0) ? 0.0f : edot3(ex, ey, ez, m.F[0], m.F[1], m.F[2]);
        const float fS = fmaf(Gw, eA - uA, fmaf(G, eB - uB, w * pf));
        const float fs = fmaf(a_f, f[i], fmaf(om_f, feq, b_f * fS));
        const float seq = fmaf(m.Td, G, Tref * Gw);
        const float sv = fmaf(a_s, s[i], fmaf(om_s, seq, w * bsw));
        int dx = x + ex, dy = y + ey, dz = z + ez;
        if (FAST) {
            const long long off = ((long long)ez * ny + ey) * nx + ex;
            S *dst = pout + c + off;
            Codec<S>::store(dst + i * N, fs, i, P);
            Codec<S>::store_dev(dst + (S0 + i) * N, sv, S0 + i, P);
        } else {
            const int kx = wrap_coord(dx, nx, P.periodic[0]);
            const int ky = wrap_coord(dy, ny, P.periodic[1]);
            const int kz = wrap_coord(dz, nz, P.periodic[2]);
            if (kx >= 2 || ky >= 2 || kz >= 2) {
                const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
                const int o = LF::opp(i);
                Codec<S>::store(pout + o * N + c, fs, o, P);
                Codec<S>::store_dev(pout + (S0 + o) * N + c, -sv + 2.0f * w * (P.T_wall[side] - P.s_ref), S0 + o, P);
            } else {
                const size_t d = ((size_t)dz * ny + dy) * nx + dx;
                Codec<S>::store(pout + i * N + d, fs, i, P);
                Codec<S>::store_dev(pout + (S0 + i) * N + d, sv, S0 + i, P);
            }
        }
    }
}

template <typename S, bool FXY>
__device__ __forceinline__ void step3d_column(const S *__restrict__ pin, S *__restrict__ pout,
                                              float *__restrict__ phi_prev,
                                              const float *__restrict__ q_in,
                                              float *__restrict__ q_out, const DevParams &P,
                                              float *sphi) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = FXY || ((x < nx) && (y < ny));
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;

    float g[QG], qcur = 0.0f;
    // prologue: plane zbeg (own cells kept in registers) and plane zbeg-1;
    // plane p lives in window slot (p + 1) % 3
    {
        float ph = 0.0f;
        if (col) {
            const size_t c = zbeg * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = Codec<S>::load_dev(pin + (G0 + i) * N + c, G0 + i, P);
            qcur = q_in[c];
            ph = g[0];
#pragma unroll
            for (int i = 1; i < QG; ++i) ph += g[i];
            ph += 0.5f * qcur;
        }
        fill_plane<S, FXY>(sphi, (zbeg + 1) % 3, zbeg, true, col, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        fill_plane<S, false>(sphi, zbeg % 3, zbeg - 1, false, false, 0.0f, pin, q_in, x0, y0, tid, tx, ty, P);
    }

    for (int z = zbeg; z < zend; ++z) {
        float gn[QG], qnext = 0.0f;
        {
            float ph = 0.0f;
            const bool ok = col && (z + 1 < nz);
            if (ok) {
                const size_t c = (size_t)(z + 1) * plane_cells + cxy;
#pragma unroll
                for (int i = 0; i < QG; ++i) gn[i] = Codec<S>::load_dev(pin + (G0 + i) * N + c, G0 + i, P);
                qnext = q_in[c];
                ph = gn[0];
#pragma unroll
                for (int i = 1; i < QG; ++i) ph += gn[i];
                ph += 0.5f * qnext;
            }
            fill_plane<S, FXY>(sphi, (z + 2) % 3, z + 1, true, ok, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        }
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            float f[QF], s[QF];
#pragma unroll
            for (int i = 0; i < QF; ++i) f[i] = Codec<S>::load(pin + i * N + c, i, P);
#pragma unroll
            for (int i = 0; i < QF; ++i) s[i] = Codec<S>::load_dev(pin + (S0 + i) * N + c, S0 + i, P);
            if (FXY && z >= 1 && z + 1 < nz)
                layer_update3d<S, true>(sphi, z, x, y, c, f, s, g, qcur, pout, phi_prev, q_out, P);
            else
                layer_update3d<S, false>(sphi, z, x, y, c, f, s, g, qcur, pout, phi_prev, q_out, P);
        }
#pragma unroll
        for (int i = 0; i < QG; ++i) g[i] = gn[i];
        qcur = qnext;
        __syncthreads();   // plane (z - 1) % 3 is overwritten next iteration
    }
}

template <typename S>
__global__ void __launch_bounds__(TX * TY, 2)
step3d_kernel(const S *__restrict__ pin, S *__restrict__ pout, float *__restrict__ phi_prev,
              const float *__restrict__ q_in, float *__restrict__ q_out, const DevParams P) {
    __shared__ float sphi[3 * PLANE];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool fxy = x0 >= 1 && x0 + TX + 1 <= P.n[0] && y0 >= 1 && y0 + TY + 1 <= P.n[1];
    if (fxy) step3d_column<S, true>(pin, pout, phi_prev, q_in, q_out, P, sphi);
    else step3d_column<S, false>(pin, pout, phi_prev, q_in, q_out, P, sphi);
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
        moments3d(m, f, s, phi_prev[c] + P.g_ref, q_in[c], P);
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
        Codec<S>::store_dev(pout + (G0 + i) * N + c, eqb - LG::w(i) * P.g_ref, G0 + i, P);
    }
#pragma unroll
    for (int i = 0; i < QF; ++i) {
        float feqb, fS, seqb, sS;
        fs_eq_src(i, m, q, D, usq, P, feqb, fS, seqb, sS);
        Codec<S>::store(pout + i * N + c, feqb, i, P);
        Codec<S>::store_dev(pout + (S0 + i) * N + c, seqb, S0 + i, P);
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
