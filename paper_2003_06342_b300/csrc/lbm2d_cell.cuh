// Per-cell pieces of the 2D (D2Q9) step shared by the tiled kernel
// (lbm2d.cu) and the TMA-staged persistent kernel (lbm2d_tma.cu).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

using L = D2Q9L;
constexpr int TX = 32, TY = 8, SX = TX + 2, SY = TY + 2;

struct Macro2 {
    float phi, gx, gy, lap, rho, grx, gry, Fx, Fy, ux, uy, p, T, Td;   // Td = T - T_ref
};

// Stencils of Sec. 3.4 from the nine values nb[i] = phi(x + e_i).
__device__ __forceinline__ void stencil2d(const float nb[9], float &gx, float &gy, float &lap) {
    const float phi = nb[0];
    gx = 0.0f; gy = 0.0f; lap = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const float plus = nb[i], minus = nb[L::opp(i)];
        const float dir = (plus - minus) * 0.5f;
        const float sec = plus - 2.0f * phi + minus;
        if (L::ex(i) != 0) gx += (L::w(i) * (float)L::ex(i)) * dir;
        if (L::ey(i) != 0) gy += (L::w(i) * (float)L::ey(i)) * dir;
        lap += L::w(i) * sec;
    }
    gx *= L::inv_cs2; gy *= L::inv_cs2; lap *= L::inv_cs2;
}

// Closures shared by the step, the moments and the initialisation.
__device__ __forceinline__ void closures2d(Macro2 &m, const DevParams &P) {
    const float phi = m.phi;
    m.rho = density(phi, P);
    m.grx = P.drho * m.gx;
    m.gry = P.drho * m.gy;
    const float mu = 4.0f * P.H * phi * (phi - 1.0f) * (phi - 0.5f) - P.K * m.lap;
    m.Fx = mu * m.gx + (m.rho - P.rho_l) * P.gravity[0] + P.body[0];
    m.Fy = mu * m.gy + (m.rho - P.rho_l) * P.gravity[1] + P.body[1];
}

// Moments of the post-streaming populations (Eqs. Velocity, Pressure,
// Moment_Temp); s holds the temperature populations as deviations
// sbar_i - w_i T_ref, so their sum is T - T_ref.
__device__ __forceinline__ void moments2d(Macro2 &m, const float f[9], const float s[9],
                                          float phi_prev, float q_prev, const DevParams &P) {
    closures2d(m, P);
    float jx = 0.0f, jy = 0.0f, sf = f[0], ss = s[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (L::ex(i) != 0) jx += (float)L::ex(i) * f[i];
        if (L::ey(i) != 0) jy += (float)L::ey(i) * f[i];
        sf += f[i];
        ss += s[i];
    }
    m.ux = (jx * L::inv_cs2 + 0.5f * m.Fx) / m.rho;
    m.uy = (jy * L::inv_cs2 + 0.5f * m.Fy) / m.rho;
    m.p = sf + 0.5f * (L::cs2 * (m.ux * m.grx + m.uy * m.gry) + m.rho * L::cs2 * q_prev * P.kappa);
    m.Td = ss - 0.5f * P.L_over_Cp * ((m.phi - phi_prev) + (m.ux * m.gx + m.uy * m.gy) + m.phi * q_prev * P.kappa);
    m.T = m.Td + P.s_ref;
}

// Unbarred equilibria and sources of the three sets for direction i; seq is
// the temperature equilibrium T Gamma_i as a deviation from w_i T_ref:
// (T - T_ref) Gamma_i + T_ref (Gamma_i - w_i).
struct EqSrc { float geq, gS, feq, fS, seq, sS; };

__device__ __forceinline__ EqSrc eq_src2d(int i, const Macro2 &m, float nx_, float ny_, float q,
                                          float D, const DevParams &P) {
    const float w = L::w(i);
    const float cu = (float)L::ex(i) * m.ux + (float)L::ey(i) * m.uy;
    const float usq = m.ux * m.ux + m.uy * m.uy;
    const float poly = 3.0f * cu + 4.5f * cu * cu - 1.5f * usq;
    const float G = w * (1.0f + poly);                               // Eq. FunctionGamma
    EqSrc r;
    const float en = (float)L::ex(i) * nx_ + (float)L::ey(i) * ny_;
    r.geq = m.phi * G;
    r.gS = P.four_over_W * m.phi * (1.0f - m.phi) * w * en + w * q;  // F^g + P^g
    r.feq = w * (m.p + m.rho * L::cs2 * poly);                       // Eq. Feq_NS_Incompr
    const float Gw = G - w;
    r.fS = ((float)L::ex(i) - m.ux) * (Gw * m.grx * L::cs2 + G * m.Fx)
         + ((float)L::ey(i) - m.uy) * (Gw * m.gry * L::cs2 + G * m.Fy)
         + w * m.rho * L::cs2 * q * P.kappa;                         // F^f + P^f
    r.seq = m.Td * G + P.s_ref * (w * poly);
    r.sS = -w * P.L_over_Cp * D;                                     // F^s + P^s
    return r;
}

__device__ __forceinline__ void normal2d(float gx, float gy, float eps2, float &nx_, float &ny_) {
    const float d = sqrtf(fmaxf(gx * gx + gy * gy, eps2));
    nx_ = gx / d;
    ny_ = gy / d;
}

// ------------------------------------------------------------------ step
// +-v or 0 for a lattice component e in {-1, 0, 1}, and e.(a, b) without
// multiplications (e is a compile-time constant once the loops are unrolled)
__device__ __forceinline__ float sgnv(int e, float v) { return e > 0 ? v : -v; }
__device__ __forceinline__ float edot(int ex, int ey, float a, float b) {
    return ex == 0 ? (ey == 0 ? 0.0f : sgnv(ey, b))
                   : (ey == 0 ? sgnv(ex, a) : sgnv(ex, a) + sgnv(ey, b));
}

// Update of one cell from a window of phi - phi_ref (`sp` points at the
// cell, rows `pitch` floats apart) and the cell's own populations: stencils,
// closures, moments, production rate, the three collisions and the push into
// pout.  FAST: no link of the cell wraps or meets a wall.
template <typename S, bool FAST>
__device__ __forceinline__ void cell_update2d(const float *sp, int pitch, const float f[9],
                                              const float g[9], const float s[9], float phip,
                                              float qp, int x, int y, size_t c,
                                              S *__restrict__ pout, float *__restrict__ phi_prev,
                                              float *__restrict__ q_out, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    // stencils, pair-folded: each (i, opposite) pair of Eqs. Grad and
    // Laplacian contributes w_i e_i (phi_i - phi_i') and 2 w_i (phi_i + phi_i' - 2 phi)
    // the window holds phi - phi_ref; differences are unaffected by the shift
    const float phd = sp[0];
    const float ph = phd + P.g_ref;
    const float pE = sp[1], pW = sp[-1], pN = sp[pitch], pS = sp[-pitch];
    const float pNE = sp[pitch + 1], pNW = sp[pitch - 1], pSW = sp[-pitch - 1], pSE = sp[-pitch + 1];
    Macro2 m;
    m.phi = ph;
    {
        const float dA = pNE - pSW, dB = pSE - pNW;
        m.gx = 3.0f * ((1.0f / 9.0f) * (pE - pW) + (1.0f / 36.0f) * (dA + dB));
        m.gy = 3.0f * ((1.0f / 9.0f) * (pN - pS) + (1.0f / 36.0f) * (dA - dB));
        m.lap = 6.0f * ((1.0f / 9.0f) * ((pE + pW) + (pN + pS) - 4.0f * phd)
                      + (1.0f / 36.0f) * ((pNE + pSW) + (pNW + pSE) - 4.0f * phd));
    }
    closures2d(m, P);
    // moments (Eqs. Velocity, Pressure, Moment_Temp)
    const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
    const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    float sf = f[0], ss = s[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) { sf += f[i]; ss += s[i]; }
    const float inv_rho = __frcp_rn(m.rho);
    m.ux = (3.0f * jx + 0.5f * m.Fx) * inv_rho;
    m.uy = (3.0f * jy + 0.5f * m.Fy) * inv_rho;
    const float rcs2 = m.rho * L::cs2;
    m.p = sf + 0.5f * (L::cs2 * (m.ux * m.grx + m.uy * m.gry) + rcs2 * qp * P.kappa);
    const float ug = m.ux * m.gx + m.uy * m.gy;
    m.Td = ss - 0.5f * P.L_over_Cp * ((phd - phip) + ug + ph * qp * P.kappa);
    m.T = m.Td + P.s_ref;

    const float q = production(ph, m.T, P);
    const float inv_d = __frcp_rn(sqrtf(fmaxf(m.gx * m.gx + m.gy * m.gy, P.eps2)));
    const float nx_ = m.gx * inv_d, ny_ = m.gy * inv_d;
    const float om_g = P.om_g;
    const float om_f = __frcp_rn(viscosity(ph, P) * L::inv_cs2 + 0.5f);
    const float om_s = __frcp_rn(diffusivity(ph, P) * L::inv_cs2 + 0.5f);
    const float D = (phd - phip) + ug + ph * q * P.kappa;

    phi_prev[c] = phd;          // stored as phi - phi_ref
    q_out[c] = q;

    // collision in the form theta* = (1 - om) theta + om theta_eq + (1 - om/2) S,
    // algebraically identical to Eq. LBE with theta_eq_bar = theta_eq - S/2
    const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
    const float iface = P.four_over_W * ph * (1.0f - ph);
    const float gAx = L::cs2 * m.grx, gAy = L::cs2 * m.gry;
    const float uA = m.ux * gAx + m.uy * gAy;
    const float uB = m.ux * m.Fx + m.uy * m.Fy;
    const float pf = rcs2 * q * P.kappa;                 // P^f_i / w_i
    const float a_g = 1.0f - om_g, b_g = 1.0f - 0.5f * om_g;
    const float a_f = 1.0f - om_f, b_f = 1.0f - 0.5f * om_f;
    const float a_s = 1.0f - om_s, b_s = 1.0f - 0.5f * om_s;
    const float bsw = b_s * (-P.L_over_Cp * D);          // (1 - om_s/2) S^s_i / w_i
    const float Tref = P.s_ref;

#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ex = L::ex(i), ey = L::ey(i);
        const float w = L::w(i);
        const float cu = edot(ex, ey, m.ux, m.uy);
        const float poly = cu * fmaf(4.5f, cu, 3.0f) - usq15;     // Gamma_i / w_i - 1
        const float G = fmaf(w, poly, w);                          // Eq. FunctionGamma
        const float Gw = w * poly;
        // phase field: F^g + P^g = w (iface e.n + q)
        const float Sg = w * (ex == 0 && ey == 0 ? q : fmaf(iface, edot(ex, ey, nx_, ny_), q));
        // phase field in deviation form: g_eq - w phi_ref = (phi - phi_ref) G + phi_ref (G - w)
        const float gs = fmaf(a_g, g[i], fmaf(om_g, fmaf(phd, G, P.g_ref * Gw), b_g * Sg));
        // flow: f_eq = w (p + rho cs2 poly), F^f + P^f
        const float feq = w * fmaf(rcs2, poly, m.p);
        const float fS = fmaf(Gw, edot(ex, ey, gAx, gAy) - uA, fmaf(G, edot(ex, ey, m.Fx, m.Fy) - uB, w * pf));
        const float fs = fmaf(a_f, f[i], fmaf(om_f, feq, b_f * fS));
        // temperature, deviation form: s_eq - w T_ref = (T - T_ref) G + T_ref (G - w)
        const float seq = fmaf(m.Td, G, Tref * Gw);
        const float ssv = fmaf(a_s, s[i], fmaf(om_s, seq, w * bsw));
        if (FAST) {
            const long long off = (long long)ey * nx + ex;
            S *dst = pout + c + off;
            Codec<S>::store(dst + i * N, fs, i, P);
            Codec<S>::store_dev(dst + (9 + i) * N, gs, 9 + i, P);
            Codec<S>::store_dev(dst + (18 + i) * N, ssv, 18 + i, P);
        } else {
            int dx = x + ex, dy = y + ey;
            const int kx = wrap_coord(dx, nx, P.periodic[0]);
            const int ky = wrap_coord(dy, ny, P.periodic[1]);
            if (kx >= 2 || ky >= 2) {
                const int side = (kx >= 2 ? kx : ky) - 2;
                const int o = L::opp(i);
                const float w2 = 2.0f * w;
                Codec<S>::store(pout + o * N + c, fs, o, P);
                Codec<S>::store_dev(pout + (9 + o) * N + c, -gs + w2 * (P.phi_wall[side] - P.g_ref), 9 + o, P);
                Codec<S>::store_dev(pout + (18 + o) * N + c, -ssv + w2 * (P.T_wall[side] - P.s_ref), 18 + o, P);
            } else {
                const size_t d = (size_t)dy * nx + dx;
                Codec<S>::store(pout + i * N + d, fs, i, P);
                Codec<S>::store_dev(pout + (9 + i) * N + d, gs, 9 + i, P);
                Codec<S>::store_dev(pout + (18 + i) * N + d, ssv, 18 + i, P);
            }
        }
    }
}

// The whole update of one tile.  FAST: the tile and its halo ring lie inside
// the grid, so no halo cell and no streaming link wraps or meets a wall.
template <typename S, bool FAST>
__device__ __forceinline__ void step2d_tile(const S *__restrict__ pin, S *__restrict__ pout,
                                            float *__restrict__ phi_prev,
                                            const float *__restrict__ q_in,
                                            float *__restrict__ q_out, const DevParams &P,
                                            float *sphi, int x0, int y0) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = FAST || ((x < nx) && (y < ny));
    const size_t c = active ? (size_t)y * nx + x : 0;

    float f[9], g[9], s[9], phip = 0.0f, qp = 0.0f;
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Codec<S>::load_dev(pin + (9 + i) * N + c, 9 + i, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = Codec<S>::load(pin + i * N + c, i, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) s[i] = Codec<S>::load_dev(pin + (18 + i) * N + c, 18 + i, P);
        phip = phi_prev[c];
        qp = q_in[c];
        float ph = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) ph += g[i];
        sphi[(ty + 1) * SX + tx + 1] = ph + 0.5f * qp;      // phi - phi_ref
    }
    if (FAST) {
        // the 2*SX + 2*TY halo cells, one per thread
        constexpr int RING = 2 * SX + 2 * TY;
        if (tid < RING) {
            int sx, sy;
            if (tid < SX) { sx = tid; sy = 0; }
            else if (tid < 2 * SX) { sx = tid - SX; sy = SY - 1; }
            else if (tid < 2 * SX + TY) { sx = 0; sy = 1 + tid - 2 * SX; }
            else { sx = SX - 1; sy = 1 + tid - 2 * SX - TY; }
            const size_t cc = (size_t)(y0 + sy - 1) * nx + (x0 + sx - 1);
            float v = Codec<S>::load_dev(pin + 9 * N + cc, 9, P);
#pragma unroll
            for (int i = 1; i < 9; ++i) v += Codec<S>::load_dev(pin + (9 + i) * N + cc, 9 + i, P);
            sphi[sy * SX + sx] = v + 0.5f * q_in[cc];
        }
    } else {
        // halo ring and ragged-tile slots: phi at the (wrapped) neighbour
        // cell, or the wall's Dirichlet value beyond a wall
        for (int sidx = tid; sidx < SX * SY; sidx += TX * TY) {
            const int sx = sidx % SX, sy = sidx / SX;
            int cx = x0 + sx - 1, cy = y0 + sy - 1;
            const bool inner = sx >= 1 && sx <= TX && sy >= 1 && sy <= TY;
            if (inner && cx < nx && cy < ny) continue;               // owned by a thread
            if (cx < -1 || cx > nx || cy < -1 || cy > ny) { sphi[sidx] = 0.0f; continue; }
            const int kx = wrap_coord(cx, nx, P.periodic[0]);
            const int ky = wrap_coord(cy, ny, P.periodic[1]);
            float v;
            if (kx >= 2) v = P.phi_wall[kx - 2] - P.g_ref;
            else if (ky >= 2) v = P.phi_wall[ky - 2] - P.g_ref;
            else {
                const size_t cc = (size_t)cy * nx + cx;
                v = Codec<S>::load_dev(pin + 9 * N + cc, 9, P);
#pragma unroll
                for (int i = 1; i < 9; ++i) v += Codec<S>::load_dev(pin + (9 + i) * N + cc, 9 + i, P);
                v += 0.5f * q_in[cc];
            }
            sphi[sidx] = v;
        }
    }
    __syncthreads();
    if (!active) return;

    cell_update2d<S, FAST>(sphi + (ty + 1) * SX + tx + 1, SX, f, g, s, phip, qp, x, y, c, pout,
                           phi_prev, q_out, P);
}

}  // namespace lbm
