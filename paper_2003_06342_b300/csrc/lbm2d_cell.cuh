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
    const float mu = fmaf(-P.K, m.lap, 4.0f * P.H * phi * (phi - 1.0f) * (phi - 0.5f));
    m.Fx = fmaf(mu, m.gx, fmaf(m.rho - P.rho_l, P.gravity[0], P.body[0]));
    m.Fy = fmaf(mu, m.gy, fmaf(m.rho - P.rho_l, P.gravity[1], P.body[1]));
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

// grad(phi) by Eq. Grad with the second-order biased directional difference
// [-phi(x + 2e) + 4 phi(x + e) - 3 phi(x)] / 2 (Sec. 3.4), from the values one
// (p*) and two (q*) cells away in each D2Q9 direction.  Pair-folded: a
// direction and its opposite contribute w e (4 (p+ - p-) - (q+ - q-)) / 2.
__device__ __forceinline__ void biased_grad2d(float pE, float pW, float pN, float pS, float pNE, float pNW,
                                              float pSW, float pSE, float qE, float qW, float qN, float qS,
                                              float qNE, float qNW, float qSW, float qSE, float &gx, float &gy) {
    const float bx = 0.5f * fmaf(4.0f, pE - pW, -(qE - qW));
    const float by = 0.5f * fmaf(4.0f, pN - pS, -(qN - qS));
    const float bA = 0.5f * fmaf(4.0f, pNE - pSW, -(qNE - qSW));     // along (1, 1)
    const float bB = 0.5f * fmaf(4.0f, pSE - pNW, -(qSE - qNW));     // along (1, -1)
    gx = 3.0f * fmaf(1.0f / 9.0f, bx, (1.0f / 36.0f) * (bA + bB));
    gy = 3.0f * fmaf(1.0f / 9.0f, by, (1.0f / 36.0f) * (bA - bB));
}

__device__ __forceinline__ void normal2d(float gx, float gy, float eps2, float &nx_, float &ny_) {
    const float d = sqrtf(fmaxf(gx * gx + gy * gy, eps2));
    nx_ = gx / d;
    ny_ = gy / d;
}

// Base pointers of the population planes of the buffer read and of the
// buffer written, passed to the kernels as a parameter: entries 0..8 are the
// (f_i, s_i) pair planes, 9..17 the g planes.  A fast-path load or store then
// addresses its plane as base + cell, with no per-plane offset arithmetic
// (measured: 2.8% faster 2D FP32 step).
template <typename S> struct Planes2d {
    const S *in[18];
    S *out[18];
};

template <typename S>
inline Planes2d<S> planes2d(const void *pin, void *pout, const DevParams &P) {
    Planes2d<S> PL;
    const size_t N = (size_t)P.N;
    for (int i = 0; i < 9; ++i) {
        PL.in[i] = (const S *)pin + off_f(i, 0, N);
        PL.out[i] = (S *)pout + off_f(i, 0, N);
        PL.in[9 + i] = (const S *)pin + off_g(9, i, 0, N);
        PL.out[9 + i] = (S *)pout + off_g(9, i, 0, N);
    }
    return PL;
}

// ------------------------------------------------------------------ step
// Sums over one D2Q9 set in the working representation v (see IsNarrow):
// sum_i mu_i v_i = sum_i theta_i - ref and sum_i mu_i e_i v_i, with mu_i = 1
// for FP32 and w_i / scale for the 16-bit formats.  Every kernel that forms
// phi from the stored g uses set_sum2d, so a cell's phi is the same float
// wherever it is computed.
template <typename S>
__device__ __forceinline__ float set_sum2d(const float v[9], float inv_sc) {
    const float ax = (v[1] + v[3]) + (v[2] + v[4]);
    const float dg = (v[5] + v[7]) + (v[6] + v[8]);
    if (!IsNarrow<S>::value) return v[0] + (ax + dg);
    return fmaf(4.0f / 9.0f, v[0], fmaf(1.0f / 9.0f, ax, (1.0f / 36.0f) * dg)) * inv_sc;
}

// set_sum2d of the flow (x) and temperature (y) sets at once, with the same
// sum tree (packed FP32x2), so each lane equals set_sum2d of its set
template <typename S>
__device__ __forceinline__ float2 set_sum2dx2(const float f[9], const float s[9], float2 inv_sc) {
    float2 v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = make_float2(f[i], s[i]);
    const float2 ax = fadd2(fadd2(v[1], v[3]), fadd2(v[2], v[4]));
    const float2 dg = fadd2(fadd2(v[5], v[7]), fadd2(v[6], v[8]));
    if (!IsNarrow<S>::value) return fadd2(v[0], fadd2(ax, dg));
    return fmul2(ffma2(splat2(4.0f / 9.0f), v[0], ffma2(splat2(1.0f / 9.0f), ax, fmul2(splat2(1.0f / 36.0f), dg))),
                 inv_sc);
}

template <typename S>
__device__ __forceinline__ void set_flux2d(const float v[9], float inv_sc, float &jx, float &jy) {
    const float ax = v[1] - v[3], ay = v[2] - v[4];
    const float d57 = v[5] - v[7], d86 = v[8] - v[6];        // e5 = (1,1), e8 = (1,-1)
    if (!IsNarrow<S>::value) {
        jx = ax + (d57 + d86);
        jy = ay + (d57 - d86);
    } else {
        jx = fmaf(1.0f / 9.0f, ax, (1.0f / 36.0f) * (d57 + d86)) * inv_sc;
        jy = fmaf(1.0f / 9.0f, ay, (1.0f / 36.0f) * (d57 - d86)) * inv_sc;
    }
}

// Multiplier taking a per-weight post-collision increment to the working
// representation: w_i for FP32 deviations, the set's scale for 16-bit values.
template <typename S>
__device__ __forceinline__ float rep_mul(int i, int set, const DevParams &P) {
    return IsNarrow<S>::value ? P.set_sc[set] : L::w(i);
}

// A per-weight increment x taken to the working representation: w_i x (the
// split-weight product of weighted()) for FP32, x times the set's scale for
// 16-bit storage.
template <typename S>
__device__ __forceinline__ float to_rep(int i, int set, float x, const DevParams &P) {
    return IsNarrow<S>::value ? P.set_sc[set] * x : weighted<L>(i, x);
}

// Push of direction i's three post-collision values (working representation)
// from cell c = (x, y).  FAST: the link neither wraps nor meets a wall.
// PART: all three values, g alone (PUSH_G) or the (f, s) pair alone (PUSH_FS).
constexpr int PUSH_ALL = 0, PUSH_G = 1, PUSH_FS = 2;
template <typename S, bool FAST, int PART = PUSH_ALL>
__device__ __forceinline__ void push2d(int i, float vf, float vg, float vs, int x, int y, size_t c,
                                       S *__restrict__ pout, const DevParams &P,
                                       const Planes2d<S> &PL) {
    constexpr bool DO_FS = PART != PUSH_G, DO_G = PART != PUSH_FS;
    const int ex = L::ex(i), ey = L::ey(i);
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    if (FAST) {
        const long long d = (long long)c + ((long long)ey * nx + ex);
        if (in_bounds(d, (long long)N, P)) {
            if (DO_FS) store_pair<S>(PL.out[i], d, vf, vs);
            if (DO_G) PL.out[9 + i][d] = narrow<S>(vg);
        }
        return;
    }
    int dx = x + ex, dy = y + ey;
    const int kx = wrap_coord(dx, nx, P.periodic[0]);
    const int ky = wrap_coord(dy, ny, P.periodic[1]);
    if (kx >= 2 || ky >= 2) {
        // half-way bounce-back (f) and anti-bounce-back (g, s): back into c,
        // opposite direction; the Dirichlet term 2 w (value - ref) in the
        // working representation
        const int side = (kx >= 2 ? kx : ky) - 2;
        const int o = L::opp(i);
        if (!in_bounds((long long)c, (long long)N, P)) return;
        if (DO_FS)
            store_pair<S>(pout + off_f(o, 0, N), (long long)c, vf,
                          fmaf(2.0f * rep_mul<S>(i, 2, P), P.T_wall[side] - P.s_ref, -vs));
        if (DO_G)
            pout[off_g(9, o, c, N)] = narrow<S>(fmaf(2.0f * rep_mul<S>(i, 1, P), P.phi_wall[side] - P.g_ref, -vg));
    } else {
        const size_t d = (size_t)dy * nx + dx;
        if (!in_bounds((long long)d, (long long)N, P)) return;
        if (DO_FS) store_pair<S>(pout + off_f(i, 0, N), (long long)d, vf, vs);
        if (DO_G) pout[off_g(9, i, d, N)] = narrow<S>(vg);
    }
}

// Per-cell coefficients of the three collisions.  With poly_i = Gamma_i/w_i - 1
// = 3 e.u + P_e, P_e = 4.5 (e.u)^2 - 1.5 u^2 (even in e), the post-collision
// value of direction i of each set, in the form
//   theta*_i - w_i ref = (1 - om)(theta_i - w_i ref) + w_i [E(e_i) + O(e_i)]
// (algebraically Eq. LBE with theta_eq_bar = theta_eq - S/2), splits into a
// part E even in e_i and a part O odd in e_i, so a direction and its opposite
// share every product:
//   g: E = Ag + Bg P_e,                     O = e.Vg
//   f: E = K0 + K1 P_e + 3 (e.u)(e.Hf),     O = e.Vf + P_e (e.Hf)
//   s: E = As + Bs P_e,                     O = e.Ws
struct Coef2 {
    float a_g, a_f, a_s;
    float Ag, Bg, Vgx, Vgy;
    float K0, K1, Hx, Hy, Vfx, Vfy;
    float As, Bs, Wx, Wy;
};

// MRT correction of one D2Q9 set: -(M^-1 diag(s - om) M d)_i for the
// non-conserved moments of the orthogonal basis (rows rho, e, eps, j_x, q_x,
// j_y, q_y, p_xx, p_xy; squared norms 9, 36, 36, 6, 12, 6, 12, 4, 4), given
// d_i = theta_i - theta_eq_bar_i in population units and the rate
// differences s_k - om:
//   de: e,  dp: eps,  dq: q (and j when J: the flow set relaxes j with q),
//   ds: the stress moments p_xx, p_xy (read when PS: the phase-field set).
// Without J, j keeps om; without PS, p_xx and p_xy keep om.  The result is
// in the set's working representation (x 1 for FP32, x scale / w_i for
// 16-bit storage); __fmul_rn / __fadd_rn keep every product out of later
// sums, so each kernel that runs this correction produces the same bits.
template <typename S, bool J, bool PS>
__device__ __forceinline__ void mrt_correction2d(const float dd[9], float de, float dp, float dq,
                                                 float ds, float sc, float out[9]) {
    const float ce = __fmul_rn(de, 1.0f / 36.0f), cp = __fmul_rn(dp, 1.0f / 36.0f);
    const float cj = J ? __fmul_rn(dq, 1.0f / 6.0f) : 0.0f;
    const float cq = __fmul_rn(dq, 1.0f / 12.0f);
    const float cs = PS ? __fmul_rn(ds, 0.25f) : 0.0f;
    // moments of d (e5 = (1,1), e6 = (-1,1), e7 = (-1,-1), e8 = (1,-1))
    const float s13 = dd[1] + dd[3], s24 = dd[2] + dd[4];
    const float s57 = dd[5] + dd[7], s68 = dd[6] + dd[8];
    const float sa = s13 + s24, sd = s57 + s68;
    const float me = fmaf(2.0f, sd, fmaf(-4.0f, dd[0], -sa));
    const float meps = fmaf(4.0f, dd[0], fmaf(-2.0f, sa, sd));
    const float ax = dd[1] - dd[3], ay = dd[2] - dd[4];
    const float dx = (dd[5] - dd[7]) + (dd[8] - dd[6]), dy = (dd[5] - dd[7]) - (dd[8] - dd[6]);
    const float mqx = fmaf(-2.0f, ax, dx), mqy = fmaf(-2.0f, ay, dy);
    // by direction class: rest, axis (even, odd), diagonal (even, odd)
    const float r0 = 4.0f * fmaf(ce, me, -cp * meps);
    const float rA = fmaf(ce, me, 2.0f * cp * meps);
    const float rD = -fmaf(2.0f * ce, me, cp * meps);
    float Ox = __fmul_rn(2.0f * cq, mqx), Oy = __fmul_rn(2.0f * cq, mqy);
    float Bx = __fmul_rn(-cq, mqx), By = __fmul_rn(-cq, mqy);
    if (J) {
        const float mjx = ax + dx, mjy = ay + dy;
        Ox = fmaf(2.0f * cq, mqx, -cj * mjx);
        Oy = fmaf(2.0f * cq, mqy, -cj * mjy);
        Bx = -fmaf(cj, mjx, cq * mqx);
        By = -fmaf(cj, mjy, cq * mqy);
    }
    // stress moments: p_xx = +1 on x-axis links, -1 on y-axis links; p_xy = +1
    // on the (1,1) / (-1,-1) diagonals, -1 on the others
    const float pxx = PS ? __fmul_rn(cs, s13 - s24) : 0.0f;
    const float pxy = PS ? __fmul_rn(cs, s57 - s68) : 0.0f;
    const float rAx = PS ? rA - pxx : rA, rAy = PS ? rA + pxx : rA;
    const float rD57 = PS ? rD - pxy : rD, rD68 = PS ? rD + pxy : rD;
    const bool nar = IsNarrow<S>::value;
    const float k0 = nar ? sc * 2.25f : 1.0f, kA = nar ? sc * 9.0f : 1.0f, kD = nar ? sc * 36.0f : 1.0f;
    out[0] = __fmul_rn(k0, r0);
    out[1] = __fmul_rn(kA, rAx + Ox); out[3] = __fmul_rn(kA, rAx - Ox);
    out[2] = __fmul_rn(kA, rAy + Oy); out[4] = __fmul_rn(kA, rAy - Oy);
    out[5] = __fmul_rn(kD, rD57 + (Bx + By)); out[7] = __fmul_rn(kD, rD57 - (Bx + By));
    out[6] = __fmul_rn(kD, rD68 + (By - Bx)); out[8] = __fmul_rn(kD, rD68 - (By - Bx));
}

// Update of one cell from a window of phi - phi_ref (`sp` points at the
// cell, rows `pitch` floats apart) and the cell's own populations in the
// working representation: stencils, closures, moments, production rate, the
// three collisions and the push into pout.  FAST: no link of the cell wraps or
// meets a wall.
// COLL selects the collision of Eq. LBE (COLL_BGK) or one of two extensions
// outside the paper.  COLL_TRT: the BGK relaxation (1 - om) v_i becomes
// v_i - w+ (v_i + v_o)/2 - w- (v_i - v_o)/2 = a1 v_i + a2 v_o (o = opposite).
// COLL_MRT (flow and phase-field sets; s keeps BGK): with d = theta -
// theta_eq_bar and the orthogonal D2Q9 moment basis M (rows rho, e, eps, j_x,
// q_x, j_y, q_y, p_xx, p_xy), theta*_i = theta_i - (M^-1 diag(s) M d)_i + S_i;
// for f the conserved and stress moments relax at the BGK rate om_f, e and
// eps at s_e and s_eps, j and q at s_q; for g phi and j relax at om_g (the
// mobility), e, eps, q and the stress moments at their own rates.  Computed
// as the BGK update plus -(M^-1 diag(s - om) M d)_i (mrt_correction2d).
// BIASED: the gradient of Eq. Grad from the second-order biased difference
// (the window then holds two rings around the tile).
template <typename S, int COLL, bool BIASED, class Sink>
__device__ __forceinline__ void cell_core2d(const float *sp, int pitch, const float f[9],
                                            const float g[9], const float s[9], float phip,
                                            float qp, const DevParams &P, Sink &sink) {
    constexpr bool TRT = COLL == COLL_TRT, MRT = COLL == COLL_MRT;
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
        if (BIASED) {
            const int p2 = 2 * pitch;
            biased_grad2d(pE, pW, pN, pS, pNE, pNW, pSW, pSE, sp[2], sp[-2], sp[p2], sp[-p2], sp[p2 + 2],
                          sp[p2 - 2], sp[-p2 - 2], sp[-p2 + 2], m.gx, m.gy);
        } else {
            m.gx = 3.0f * fmaf(1.0f / 9.0f, pE - pW, (1.0f / 36.0f) * (dA + dB));
            m.gy = 3.0f * fmaf(1.0f / 9.0f, pN - pS, (1.0f / 36.0f) * (dA - dB));
        }
        const float la = fmaf(-4.0f, phd, (pE + pW) + (pN + pS));
        const float ld = fmaf(-4.0f, phd, (pNE + pSW) + (pNW + pSE));
        m.lap = 6.0f * fmaf(1.0f / 9.0f, la, (1.0f / 36.0f) * ld);
    }
    closures2d(m, P);
    // moments (Eqs. Velocity, Pressure, Moment_Temp)
    float jx, jy;
    set_flux2d<S>(f, P.set_isc[0], jx, jy);
    const float2 sfs = set_sum2dx2<S>(f, s, make_float2(P.set_isc[0], P.set_isc[2]));
    const float sf = sfs.x + P.set_ref[0];
    const float ss = sfs.y;                                          // T - T_ref
    const float inv_rho = rcp_approx(m.rho);
    m.ux = fmaf(0.5f, m.Fx, 3.0f * jx) * inv_rho;
    m.uy = fmaf(0.5f, m.Fy, 3.0f * jy) * inv_rho;
    const float rcs2 = m.rho * L::cs2;
    const float ugr = fmaf(m.ux, m.grx, m.uy * m.gry);
    m.p = fmaf(0.5f, fmaf(L::cs2, ugr, (rcs2 * qp) * P.kappa), sf);
    const float ug = fmaf(m.ux, m.gx, m.uy * m.gy);
    m.Td = fmaf(-0.5f * P.L_over_Cp, fmaf(ph * qp, P.kappa, (phd - phip) + ug), ss);
    m.T = m.Td + P.s_ref;

    const float q = production(ph, m.T, P);
    const float inv_d = rsqrt_approx(fmaxf(fmaf(m.gx, m.gx, m.gy * m.gy), P.eps2));
    const float nx_ = m.gx * inv_d, ny_ = m.gy * inv_d;
    const float phu = unit_phi(ph);
    float om_f;
    if (P.visc_interp == 0) {
        // 1 / (nu / cs2 + 1/2) with the harmonic nu = nu_l nu_g / den
        const float den = fmaf(phu, P.nu_l - P.nu_g, P.nu_g);
        om_f = den * rcp_approx(fmaf(0.5f, den, 3.0f * P.nu_l * P.nu_g));
    } else {
        om_f = rcp_approx(fmaf(L::inv_cs2, fmaf(phu, P.nu_g - P.nu_l, P.nu_l), 0.5f));
    }
    const float om_s = rcp_approx(fmaf(L::inv_cs2, diffusivity(ph, P), 0.5f));
    const float om_g = P.om_g;
    const float D = fmaf(ph * q, P.kappa, (phd - phip) + ug);

    sink.scalars(phd, q);      // phi^{n-1} stored as phi - phi_ref

    const float ux = m.ux, uy = m.uy;
    // rates of the symmetric (p) and antisymmetric (m) parts: the BGK rate on
    // both, or with TRT the BGK rate on the part carrying the transport
    // coefficient (f: symmetric; g, s: antisymmetric) and the magic-parameter
    // rate on the other
    const float omp_f = om_f, omm_g = om_g, omm_s = om_s;
    const float omm_f = TRT ? trt_other_rate(om_f, P.trt_magic[0]) : om_f;
    const float omp_g = TRT ? trt_other_rate(om_g, P.trt_magic[1]) : om_g;
    const float omp_s = TRT ? trt_other_rate(om_s, P.trt_magic[2]) : om_s;
    const float b_g = fmaf(-0.5f, omp_g, 1.0f), b_f = fmaf(-0.5f, omp_f, 1.0f);
    const float b_s = fmaf(-0.5f, omp_s, 1.0f);
    const float bm_g = TRT ? fmaf(-0.5f, omm_g, 1.0f) : b_g;
    const float bm_f = TRT ? fmaf(-0.5f, omm_f, 1.0f) : b_f;
    Coef2 k;
    k.a_g = 1.0f - omp_g; k.a_f = 1.0f - omp_f; k.a_s = 1.0f - omp_s;    // rest direction
    // g: F^g + P^g = w (iface e.n + q); g_eq - w phi_ref = w (phd + phi poly)
    const float iface = P.four_over_W * ph * (1.0f - ph);
    k.Ag = fmaf(omp_g, phd, b_g * q);
    k.Bg = omp_g * ph;
    const float Bgo = TRT ? omm_g * ph : k.Bg;
    const float bgi = bm_g * iface;
    k.Vgx = fmaf(3.0f * Bgo, ux, bgi * nx_);
    k.Vgy = fmaf(3.0f * Bgo, uy, bgi * ny_);
    // f: f_eq = w (p + rho cs2 poly); F^f + P^f = w [(e.F - u.F + pf) + poly (e.H - u.H)]
    // with H = cs2 grad(rho) + F (Eq. Forcing with Gamma_i = w_i (1 + poly_i))
    const float hx = fmaf(L::cs2, m.grx, m.Fx), hy = fmaf(L::cs2, m.gry, m.Fy);
    const float hU = fmaf(ux, hx, uy * hy);
    const float uB = fmaf(ux, m.Fx, uy * m.Fy);
    // P^f_i / w_i = rho cs2 q kappa, here minus u.F
    k.K0 = fmaf(omp_f, m.p - P.set_ref[0], b_f * fmaf(rcs2 * q, P.kappa, -uB));
    k.K1 = fmaf(omp_f, rcs2, -b_f * hU);
    k.Hx = b_f * hx; k.Hy = b_f * hy;
    // the odd part: K1 and H with the antisymmetric rate
    const float K1o = TRT ? fmaf(omm_f, rcs2, -bm_f * hU) : k.K1;
    const float Hox = TRT ? bm_f * hx : k.Hx, Hoy = TRT ? bm_f * hy : k.Hy;
    k.Vfx = fmaf(3.0f * K1o, ux, bm_f * m.Fx);
    k.Vfy = fmaf(3.0f * K1o, uy, bm_f * m.Fy);
    // s: s_eq - w T_ref = w (Td + T poly); S^s = -w (L/Cp) D
    k.As = fmaf(omp_s, m.Td, -b_s * P.L_over_Cp * D);
    k.Bs = omp_s * m.T;
    const float Bso = TRT ? omm_s * m.T : k.Bs;
    // __fmul_rn: W enters E +- W as a finished product, never fused into the sum
    k.Wx = __fmul_rn(3.0f * Bso, ux); k.Wy = __fmul_rn(3.0f * Bso, uy);
    // TRT: out_i = a1 v_i + a2 v_o + ...
    const float a1_f = 1.0f - 0.5f * (omp_f + omm_f), a2_f = 0.5f * (omm_f - omp_f);
    const float a1_g = 1.0f - 0.5f * (omp_g + omm_g), a2_g = 0.5f * (omm_g - omp_g);
    const float a1_s = 1.0f - 0.5f * (omp_s + omm_s), a2_s = 0.5f * (omm_s - omp_s);

    // even parts P_e of poly: rest, x axis, y axis, diagonals (1,1) and (-1,1)
    const float uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const float usq = fmaf(ux, ux, uyy);
    const float P0 = -1.5f * usq;
    const float Pxa = fmaf(3.0f, uxx, -1.5f * uyy), Pya = fmaf(3.0f, uyy, -1.5f * uxx);
    const float Pd0 = 3.0f * usq;

    const float2 a_fs = make_float2(k.a_f, k.a_s);
    const float2 a1_fs = make_float2(a1_f, a1_s), a2_fs = make_float2(a2_f, a2_s);
    // a direction i with e = (ex, ey) and its opposite o.  With MRT the sets
    // go out in two passes, each with its own correction c (working
    // representation), so only one set's correction is live at a time:
    // part 1 pushes g, part 2 pushes f and s.
    auto pair = [&](int part, const float *c, int i, int o, float cu, float Pe, float eVg, float eH,
                    float eHo, float eVf, float eW) {
        const float Eg = fmaf(k.Bg, Pe, k.Ag);
        const float Ef = fmaf(3.0f * cu, eH, fmaf(k.K1, Pe, k.K0));
        const float Of = fmaf(Pe, eHo, eVf);
        const float Es = fmaf(k.Bs, Pe, k.As);
        // w_i = w_o: the increments of i and o share the weight of i
        auto rg = [&](float v) { return to_rep<S>(i, 1, v, P); };
        // f and s as one FP32x2 pair (x: f, y: s): E + O and E - O of both
        // sets, taken to the working representation (to_rep on each lane)
        auto rfs = [&](float2 v) {
            return IsNarrow<S>::value ? fmul2(make_float2(P.set_sc[0], P.set_sc[2]), v) : weighted2<L>(i, v);
        };
        const float2 ri = rfs(fadd2(make_float2(Ef, Es), make_float2(Of, eW)));
        const float2 ro = rfs(fadd2(make_float2(Ef, Es), make_float2(-Of, -eW)));
        const float2 fsi = make_float2(f[i], s[i]), fso = make_float2(f[o], s[o]);
        if (MRT) {
            if (part == 1) {
                sink.put_g(i, __fadd_rn(fmaf(k.a_g, g[i], rg(Eg + eVg)), c[i]));
                sink.put_g(o, __fadd_rn(fmaf(k.a_g, g[o], rg(Eg - eVg)), c[o]));
            } else {
                const float2 vi = ffma2(a_fs, fsi, ri), vo = ffma2(a_fs, fso, ro);
                sink.put_fs(i, __fadd_rn(vi.x, c[i]), vi.y);
                sink.put_fs(o, __fadd_rn(vo.x, c[o]), vo.y);
            }
        } else if (!TRT) {
            const float2 vi = ffma2(a_fs, fsi, ri), vo = ffma2(a_fs, fso, ro);
            sink.put(i, vi.x, fmaf(k.a_g, g[i], rg(Eg + eVg)), vi.y);
            sink.put(o, vo.x, fmaf(k.a_g, g[o], rg(Eg - eVg)), vo.y);
        } else {
            const float2 vi = ffma2(a1_fs, fsi, ffma2(a2_fs, fso, ri));
            const float2 vo = ffma2(a1_fs, fso, ffma2(a2_fs, fsi, ro));
            sink.put(i, vi.x, fmaf(a1_g, g[i], fmaf(a2_g, g[o], rg(Eg + eVg))), vi.y);
            sink.put(o, vo.x, fmaf(a1_g, g[o], fmaf(a2_g, g[i], rg(Eg - eVg))), vo.y);
        }
    };
    auto pairs = [&](int part, const float *c) {
        pair(part, c, 1, 3, ux, Pxa, k.Vgx, k.Hx, Hox, k.Vfx, k.Wx);                 // (1, 0)
        pair(part, c, 2, 4, uy, Pya, k.Vgy, k.Hy, Hoy, k.Vfy, k.Wy);                 // (0, 1)
        // the diagonal components are sums of products: __fadd_rn / __fsub_rn
        // keep the compiler from fusing one of the products into the sum
        pair(part, c, 5, 7, __fadd_rn(ux, uy), fmaf(9.0f, uxy, Pd0), __fadd_rn(k.Vgx, k.Vgy),
             __fadd_rn(k.Hx, k.Hy), __fadd_rn(Hox, Hoy), __fadd_rn(k.Vfx, k.Vfy),
             __fadd_rn(k.Wx, k.Wy));                                                 // (1, 1)
        pair(part, c, 6, 8, __fsub_rn(uy, ux), fmaf(-9.0f, uxy, Pd0), __fsub_rn(k.Vgy, k.Vgx),
             __fsub_rn(k.Hy, k.Hx), __fsub_rn(Hoy, Hox), __fsub_rn(k.Vfy, k.Vfx),
             __fsub_rn(k.Wy, k.Wx));                                                 // (-1, 1)
    };

    if constexpr (MRT) {
        // the phase-field set: g_eq_bar - w phi_ref per weight is
        // (phd - q/2) + phi P_e + e.(3 phi u - iface n / 2) (the coefficient
        // form above at om = 1 and b = -1/2)
        {
            float dd[9], cg[9];
            const float Agb = fmaf(-0.5f, q, phd);
            const float hif = __fmul_rn(-0.5f, iface);
            const float Vgbx = fmaf(3.0f * ph, ux, __fmul_rn(hif, nx_));
            const float Vgby = fmaf(3.0f * ph, uy, __fmul_rn(hif, ny_));
            auto devg = [&](int i, float eqw) {
                return IsNarrow<S>::value ? __fmul_rn(L::w(i), fmaf(g[i], P.set_isc[1], -eqw))
                                          : fmaf(-L::w(i), eqw, g[i]);
            };
            dd[0] = devg(0, fmaf(ph, P0, Agb));
            auto gpair = [&](int i, int o, float Pe, float eV) {
                const float Eb = fmaf(ph, Pe, Agb);
                dd[i] = devg(i, Eb + eV);
                dd[o] = devg(o, Eb - eV);
            };
            gpair(1, 3, Pxa, Vgbx);
            gpair(2, 4, Pya, Vgby);
            gpair(5, 7, fmaf(9.0f, uxy, Pd0), __fadd_rn(Vgbx, Vgby));
            gpair(6, 8, fmaf(-9.0f, uxy, Pd0), __fsub_rn(Vgby, Vgbx));
            // phi and j relax at om_g (the mobility); e, eps, q, p_xx, p_xy at
            // their own rates (the host stores om_g for a rate given as 0)
            mrt_correction2d<S, false, true>(dd, P.mrt_rates_g[0] - om_g, P.mrt_rates_g[1] - om_g,
                                             P.mrt_rates_g[2] - om_g, P.mrt_rates_g[3] - om_g,
                                             P.set_sc[1], cg);
            sink.put_g(0, __fadd_rn(fmaf(k.a_g, g[0], to_rep<S>(0, 1, fmaf(k.Bg, P0, k.Ag), P)), cg[0]));
            pairs(1, cg);
        }
        // the flow set (s keeps BGK): f_eq_bar - w ref per weight, the same
        // coefficient form at om = 1 and b = -1/2
        {
            float dd[9], cf[9];
            const float K0b = fmaf(-0.5f, fmaf(rcs2 * q, P.kappa, -uB), m.p - P.set_ref[0]);
            const float K1b = fmaf(0.5f, hU, rcs2);
            const float Hbx = __fmul_rn(-0.5f, hx), Hby = __fmul_rn(-0.5f, hy);
            const float Vbx = fmaf(3.0f * K1b, ux, -0.5f * m.Fx), Vby = fmaf(3.0f * K1b, uy, -0.5f * m.Fy);
            // d_i = f_i - f_eq_bar_i (population units)
            auto devf = [&](int i, float eqw) {
                return IsNarrow<S>::value ? __fmul_rn(L::w(i), fmaf(f[i], P.set_isc[0], -eqw))
                                          : fmaf(-L::w(i), eqw, f[i]);
            };
            dd[0] = devf(0, fmaf(K1b, P0, K0b));
            auto dpair = [&](int i, int o, float cu, float Pe, float eHb, float eVb) {
                const float Eb = fmaf(3.0f * cu, eHb, fmaf(K1b, Pe, K0b));
                const float Ob = fmaf(Pe, eHb, eVb);
                dd[i] = devf(i, Eb + Ob);
                dd[o] = devf(o, Eb - Ob);
            };
            dpair(1, 3, ux, Pxa, Hbx, Vbx);
            dpair(2, 4, uy, Pya, Hby, Vby);
            dpair(5, 7, __fadd_rn(ux, uy), fmaf(9.0f, uxy, Pd0), __fadd_rn(Hbx, Hby), __fadd_rn(Vbx, Vby));
            dpair(6, 8, __fsub_rn(uy, ux), fmaf(-9.0f, uxy, Pd0), __fsub_rn(Hby, Hbx), __fsub_rn(Vby, Vbx));
            // e, eps, j and q relax at their own rates; rho, p_xx, p_xy at om_f
            mrt_correction2d<S, true, false>(dd, P.mrt_rates[0] - om_f, P.mrt_rates[1] - om_f,
                                             P.mrt_rates[2] - om_f, 0.0f, P.set_sc[0], cf);
            sink.put_fs(0, __fadd_rn(fmaf(k.a_f, f[0], to_rep<S>(0, 0, fmaf(k.K1, P0, k.K0), P)), cf[0]),
                        fmaf(k.a_s, s[0], to_rep<S>(0, 2, fmaf(k.Bs, P0, k.As), P)));
            pairs(2, cf);
        }
    } else {
        // rest
        sink.put(0, fmaf(k.a_f, f[0], to_rep<S>(0, 0, fmaf(k.K1, P0, k.K0), P)),
                 fmaf(k.a_g, g[0], to_rep<S>(0, 1, fmaf(k.Bg, P0, k.Ag), P)),
                 fmaf(k.a_s, s[0], to_rep<S>(0, 2, fmaf(k.Bs, P0, k.As), P)));
        pairs(0, nullptr);
    }
}


// Where a cell update's results go: PushSink2 pushes them into the other
// population buffer and writes phi^{n-1} and the lagged source (the tiled and
// TMA kernels); a sink gets scalars(phd, q) once and put(i, f, g, s) for every
// direction i, or with MRT put_g(i, g) for every i and then put_fs(i, f, s).
template <typename S, bool FAST>
struct PushSink2 {
    int x, y;
    size_t c;
    S *__restrict__ pout;
    float *__restrict__ phi_prev;
    float *__restrict__ q_out;
    const DevParams &P;
    const Planes2d<S> &PL;
    __device__ __forceinline__ void scalars(float phd, float q) {
        if (in_bounds((long long)c, P.N, P)) {
            phi_prev[c] = phd;
            q_out[c] = q;
        }
    }
    __device__ __forceinline__ void put(int i, float vf, float vg, float vs) {
        push2d<S, FAST>(i, vf, vg, vs, x, y, c, pout, P, PL);
    }
    __device__ __forceinline__ void put_g(int i, float vg) {
        push2d<S, FAST, PUSH_G>(i, 0.0f, vg, 0.0f, x, y, c, pout, P, PL);
    }
    __device__ __forceinline__ void put_fs(int i, float vf, float vs) {
        push2d<S, FAST, PUSH_FS>(i, vf, 0.0f, vs, x, y, c, pout, P, PL);
    }
};

template <typename S, bool FAST, int COLL = COLL_BGK, bool BIASED = false>
__device__ __forceinline__ void cell_update2d(const float *sp, int pitch, const float f[9],
                                              const float g[9], const float s[9], float phip,
                                              float qp, int x, int y, size_t c,
                                              S *__restrict__ pout, float *__restrict__ phi_prev,
                                              float *__restrict__ q_out, const DevParams &P,
                                              const Planes2d<S> &PL) {
    PushSink2<S, FAST> sink{x, y, c, pout, phi_prev, q_out, P, PL};
    cell_core2d<S, COLL, BIASED>(sp, pitch, f, g, s, phip, qp, P, sink);
}

// phi - phi_ref of one cell from its nine stored g values and lagged source
template <typename S>
__device__ __forceinline__ float phid_cell2d(const S *__restrict__ pin, size_t cc, size_t N,
                                             float qv, const DevParams &P) {
    float v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = load_raw(pin + off_g(9, i, cc, N));
    (void)in_bounds((long long)cc, (long long)N, P);
    return fmaf(0.5f, qv, set_sum2d<S>(v, P.set_isc[1]));
}

// Geometry of a tile of the tiled 2D kernels: TX_ x TY_ cells, one thread
// each, and a phi window with a one-cell halo ring of RING cells.
template <int TX_, int TY_> struct Tile2 {
    static constexpr int TX = TX_, TY = TY_, SX = TX_ + 2, SY = TY_ + 2, NT = TX_ * TY_;
    static constexpr int RING = 2 * SX + 2 * TY_;
};
using Tile2Default = Tile2<TX, TY>;

// window slot (sx, sy) of ring cell r: the top row, the bottom row, then the
// left and right columns
template <class T>
__device__ __forceinline__ void ring_slot(int r, int &sx, int &sy) {
    if (r < T::SX) { sx = r; sy = 0; }
    else if (r < 2 * T::SX) { sx = r - T::SX; sy = T::SY - 1; }
    else if (r < 2 * T::SX + T::TY) { sx = 0; sy = 1 + r - 2 * T::SX; }
    else { sx = T::SX - 1; sy = 1 + r - 2 * T::SX - T::TY; }
}

// The whole update of one tile of geometry T (blockDim = T::TX x T::TY).
// FAST: the tile and its halo ring lie inside the grid, so no halo cell and
// no streaming link wraps or meets a wall.
template <typename S, bool FAST, int COLL = COLL_BGK, class T = Tile2Default>
__device__ __forceinline__ void step2d_tile(const S *__restrict__ pin, S *__restrict__ pout,
                                            float *__restrict__ phi_prev,
                                            const float *__restrict__ q_in,
                                            float *__restrict__ q_out, const DevParams &P,
                                            float *sphi, int x0, int y0, const Planes2d<S> &PL) {
    constexpr int SXT = T::SX, SYT = T::SY, TXT = T::TX, TYT = T::TY, NT = T::NT, RING = T::RING;
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TXT + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = FAST || ((x < nx) && (y < ny));
    const size_t c = active ? (size_t)y * nx + x : 0;

    float f[9], g[9], s[9], phip = 0.0f, qp = 0.0f;
    (void)in_bounds(active ? (long long)c : 0, P.N, P);
    // FAST: the ring cells' g and q come from L2 (the neighbouring tiles load
    // the same lines), one ring cell per thread held in registers.  FP32
    // requests them before the tile's own values, so their latency overlaps
    // the own loads; the 16-bit formats after them (measured on 32 x 8 tiles:
    // ring first is 3.8% faster for FP32, own first 2.4% / 4.4% faster for
    // FP16 / BF16).  Ring cells beyond the block's thread count follow.
    constexpr bool RING_FIRST = !IsNarrow<S>::value;
    float rv[9], rq = 0.0f;
    int rslot = 0;
    auto load_ring = [&]() {
        if (FAST && tid < RING) {
            int sx, sy;
            ring_slot<T>(tid, sx, sy);
            rslot = sy * SXT + sx;
            const size_t cc = (size_t)(y0 + sy - 1) * nx + (x0 + sx - 1);
            const bool ok = in_bounds((long long)cc, (long long)N, P);
#pragma unroll
            for (int i = 0; i < 9; ++i) rv[i] = ok ? load_raw(PL.in[9 + i] + cc) : 0.0f;
            rq = ok ? q_in[cc] : 0.0f;
        }
    };
    if (RING_FIRST) load_ring();
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = load_raw(PL.in[9 + i] + c);
#pragma unroll
        for (int i = 0; i < 9; ++i) load_pair<S>(PL.in[i], (long long)c, f[i], s[i]);
        phip = phi_prev[c];
        qp = q_in[c];
        sphi[(ty + 1) * SXT + tx + 1] = fmaf(0.5f, qp, set_sum2d<S>(g, P.set_isc[1]));   // phi - phi_ref
    }
    if (!RING_FIRST) load_ring();
    if (FAST) {
        // the ring's halo cells (same arithmetic as phid_cell2d)
        if (tid < RING) sphi[rslot] = fmaf(0.5f, rq, set_sum2d<S>(rv, P.set_isc[1]));
        if (RING > NT) {
            for (int r = tid + NT; r < RING; r += NT) {
                int sx, sy;
                ring_slot<T>(r, sx, sy);
                const size_t cc = (size_t)(y0 + sy - 1) * nx + (x0 + sx - 1);
                const bool ok = in_bounds((long long)cc, (long long)N, P);
                sphi[sy * SXT + sx] = ok ? phid_cell2d<S>(pin, cc, N, q_in[cc], P) : 0.0f;
            }
        }
    } else {
        // halo ring and ragged-tile slots: phi at the (wrapped) neighbour
        // cell, or the wall's Dirichlet value beyond a wall
        for (int sidx = tid; sidx < SXT * SYT; sidx += NT) {
            const int sx = sidx % SXT, sy = sidx / SXT;
            int cx = x0 + sx - 1, cy = y0 + sy - 1;
            const bool inner = sx >= 1 && sx <= TXT && sy >= 1 && sy <= TYT;
            if (inner && cx < nx && cy < ny) continue;               // owned by a thread
            if (cx < -1 || cx > nx || cy < -1 || cy > ny) { sphi[sidx] = 0.0f; continue; }
            const int kx = wrap_coord(cx, nx, P.periodic[0]);
            const int ky = wrap_coord(cy, ny, P.periodic[1]);
            float v;
            if (kx >= 2) v = P.phi_wall[kx - 2] - P.g_ref;
            else if (ky >= 2) v = P.phi_wall[ky - 2] - P.g_ref;
            else {
                const size_t cc = (size_t)cy * nx + cx;
                v = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
            }
            sphi[sidx] = v;
        }
    }
    __syncthreads();
    if (!active) return;

    cell_update2d<S, FAST, COLL>(sphi + (ty + 1) * SXT + tx + 1, SXT, f, g, s, phip, qp, x, y, c, pout,
                                phi_prev, q_out, P, PL);
}

// The update of one tile with the biased gradient: the phi window holds two
// rings around the tile ((TY + 4) x (TX + 4) values, formed with
// plain loads; beyond a wall both ghost layers take the wall's Dirichlet
// value, periodic axes wrap).  FAST: no streaming link of the tile wraps or
// meets a wall.
template <typename S, bool FAST, int COLL, class T = Tile2Default>
__device__ __forceinline__ void step2d_tile_biased(const S *__restrict__ pin, S *__restrict__ pout,
                                                   float *__restrict__ phi_prev,
                                                   const float *__restrict__ q_in,
                                                   float *__restrict__ q_out, const DevParams &P,
                                                   float *sphi, int x0, int y0, const Planes2d<S> &PL) {
    constexpr int TX = T::TX, TY = T::TY, SXB = TX + 4, SYB = TY + 4;
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = FAST || ((x < nx) && (y < ny));
    const size_t c = active ? (size_t)y * nx + x : 0;
    float f[9], g[9], s[9], phip = 0.0f, qp = 0.0f;
    if (active) {
        (void)in_bounds((long long)c, (long long)N, P);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = load_raw(PL.in[9 + i] + c);
#pragma unroll
        for (int i = 0; i < 9; ++i) load_pair<S>(PL.in[i], (long long)c, f[i], s[i]);
        phip = phi_prev[c];
        qp = q_in[c];
        sphi[(ty + 2) * SXB + tx + 2] = fmaf(0.5f, qp, set_sum2d<S>(g, P.set_isc[1]));
    }
    // 16-bit storage, both rings inside the grid: no wrap or wall test per
    // slot (FP16 +6.5% on 2048 x 4096; FP32 measured -2.3% and keeps the
    // generic fill)
    const bool in2 = IsNarrow<S>::value && x0 >= 2 && x0 + TX + 2 <= nx && y0 >= 2 && y0 + TY + 2 <= ny;
    for (int sidx = tid; sidx < SXB * SYB; sidx += TX * TY) {
        const int sx = sidx % SXB, sy = sidx / SXB;
        int cx = x0 + sx - 2, cy = y0 + sy - 2;
        const bool inner = sx >= 2 && sx < TX + 2 && sy >= 2 && sy < TY + 2;
        if (inner && cx < nx && cy < ny) continue;                   // owned by a thread
        if (in2) {
            const size_t cc = (size_t)cy * nx + cx;
            sphi[sidx] = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
            continue;
        }
        if (cx < -2 || cx > nx + 1 || cy < -2 || cy > ny + 1) { sphi[sidx] = 0.0f; continue; }
        const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
        const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
        float v;
        if (kx >= 2) v = P.phi_wall[kx - 2] - P.g_ref;
        else if (ky >= 2) v = P.phi_wall[ky - 2] - P.g_ref;
        else {
            const size_t cc = (size_t)cy * nx + cx;
            v = phid_cell2d<S>(pin, cc, N, q_in[cc], P);
        }
        sphi[sidx] = v;
    }
    __syncthreads();
    if (!active) return;
    cell_update2d<S, FAST, COLL, true>(sphi + (ty + 2) * SXB + tx + 2, SXB, f, g, s, phip, qp, x, y, c, pout,
                                      phi_prev, q_out, P, PL);
}

}  // namespace lbm
