// 2D D2Q9 kernels: the fused time step, the initialisation, the moments
// (fields and reductions) and the streaming-map test hook.
//
// State between steps (per cell, structure of arrays, plane k = set*9 + i with
// set 0 = f, 1 = g, 2 = s): the post-streaming populations of time n,
// phi^{n-1} and the lagged source q^{n-1} = mdot'''/rho_g of the previous
// collision.  One step is one launch of step2d_kernel:
//   1. every 32x8 tile computes phi^n = sum_i gbar_i + q^{n-1}/2 (Eq.
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
//      Def_SourceTerms_Temp);
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

// The whole update of one tile.  FAST: the tile and its halo ring lie inside
// the grid, so no halo cell and no streaming link wraps or meets a wall.
template <typename S, bool FAST>
__device__ __forceinline__ void step2d_tile(const S *__restrict__ pin, S *__restrict__ pout,
                                            float *__restrict__ phi_prev,
                                            const float *__restrict__ q_in,
                                            float *__restrict__ q_out, const DevParams &P,
                                            float *sphi) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
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

    // stencils, pair-folded: each (i, opposite) pair of Eqs. Grad and
    // Laplacian contributes w_i e_i (phi_i - phi_i') and 2 w_i (phi_i + phi_i' - 2 phi)
    // the window holds phi - phi_ref; differences are unaffected by the shift
    const float *sp = sphi + (ty + 1) * SX + tx + 1;
    const float phd = sp[0];
    const float ph = phd + P.g_ref;
    const float pE = sp[1], pW = sp[-1], pN = sp[SX], pS = sp[-SX];
    const float pNE = sp[SX + 1], pNW = sp[SX - 1], pSW = sp[-SX - 1], pSE = sp[-SX + 1];
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

template <typename S>
__global__ void __launch_bounds__(TX * TY, 3)
step2d_kernel(const S *__restrict__ pin, S *__restrict__ pout, float *__restrict__ phi_prev,
              const float *__restrict__ q_in, float *__restrict__ q_out, const DevParams P) {
    __shared__ float sphi[SY * SX];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool fast = x0 >= 1 && x0 + TX + 1 <= P.n[0] && y0 >= 1 && y0 + TY + 1 <= P.n[1];
    if (fast) step2d_tile<S, true>(pin, pout, phi_prev, q_in, q_out, P, sphi);
    else step2d_tile<S, false>(pin, pout, phi_prev, q_in, q_out, P, sphi);
}

// ------------------------------------------------------------------ phi moment
template <typename S>
__global__ void phi2d_kernel(const S *__restrict__ pin, const float *__restrict__ q_in,
                             float *__restrict__ phi_out, const DevParams P) {
    const size_t N = (size_t)P.N;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
        float v = Codec<S>::load(pin + 9 * N + c, 9, P);
#pragma unroll
        for (int i = 1; i < 9; ++i) v += Codec<S>::load(pin + (9 + i) * N + c, 9 + i, P);
        phi_out[c] = v + 0.5f * q_in[c];
    }
}

// phi(x + e_i) for i = 0..8 from a phi field, with wrap / wall ghosts
__device__ __forceinline__ void gather_nb2d(const float *__restrict__ phi, int x, int y, float nb[9],
                                            const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1];
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
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double mass = 0.0, energy = 0.0;
    if (c < N) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        float nb[9], f[9], s[9];
        gather_nb2d(phi_f, x, y, nb, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = Codec<S>::load(pin + i * N + c, i, P);
            s[i] = Codec<S>::load_dev(pin + (18 + i) * N + c, 18 + i, P);
        }
        Macro2 m;
        m.phi = nb[0];
        stencil2d(nb, m.gx, m.gy, m.lap);
        moments2d(m, f, s, phi_prev[c] + P.g_ref, q_in[c], P);
        if (o_phi) o_phi[c] = m.phi;
        if (o_T) o_T[c] = m.T;
        if (o_ux) o_ux[c] = m.ux;
        if (o_uy) o_uy[c] = m.uy;
        if (o_p) o_p[c] = m.p;
        mass = (double)m.phi;
        energy = (double)m.rho * (Cp * (double)m.T + (double)m.phi * Lh);
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
        Codec<S>::store(pout + i * N + c, e.feq - 0.5f * e.fS, i, P);
        Codec<S>::store_dev(pout + (9 + i) * N + c, e.geq - 0.5f * e.gS - L::w(i) * P.g_ref, 9 + i, P);
        Codec<S>::store_dev(pout + (18 + i) * N + c, e.seq - 0.5f * e.sS, 18 + i, P);
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
    dim3 block(TX, TY);
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY);
    step2d_kernel<S><<<grid, block, 0, st>>>((const S *)pin, (S *)pout, phi_prev, q_in, q_out, P);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro2d(const void *pin, float *phi_tmp, const float *phi_prev,
                           const float *q_in, float *o_phi, float *o_T, float *o_ux, float *o_uy,
                           float *o_p, double *partial, double Cp, double Lh, const DevParams &P,
                           cudaStream_t st) {
    const int nb = (int)((P.N + 255) / 256);
    phi2d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, q_in, phi_tmp, P);
    macro2d_kernel<S><<<nb, 256, 0, st>>>((const S *)pin, phi_tmp, phi_prev, q_in, o_phi, o_T,
                                          o_ux, o_uy, o_p, partial, Cp, Lh, P);
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
