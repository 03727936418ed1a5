// Discrete adjoint of the 2D (D2Q9) time step, FP32 storage.
//
// The forward step (lbm2d.cu) maps the stored state X^n = (populations,
// phi^{n-1} - phi_ref, q^{n-1}) to X^{n+1}.  For a scalar loss J of the final
// state, the adjoint state Lambda^n = dJ/dX^n (same layout as the state) is
// obtained backwards, Lambda^n = (dX^{n+1}/dX^n)^T Lambda^{n+1}, in two
// kernels per step:
//   A. per cell x: recompute the forward update of x from X^n; gather the
//      adjoint of every value x pushed (the transpose of the push is a pull;
//      a bounced link maps back with +1 for f and -1 for the anti-bounce-back
//      sets g, s); back-propagate by hand through the collision, sources,
//      production rate, moments, closures and stencils.  Writes the adjoint
//      of x's own populations, of phi^{n-1} and of q^{n-1}, plus four planes
//      that give every stencil contribution c_j(x) = dJ/dphi^n(x + e_j)
//      (the own-cell part c_0 and the adjoints of grad phi and lap phi;
//      c_j = 3 w_j e_j.l_grad + 6 w_j l_lap for j >= 1), and accumulates
//      dJ/dL, dJ/dM_phi, dJ/dsigma (FP64 block sums, one atomic per block).
//   B. per cell y: lambda_phi(y) = sum_j c_j(y - e_j) (transpose of the
//      stencil gather) into plane 29 of the adjoint state.
// The transpose of phi^n = sum_i g_i + q^{n-1}/2 is left implicit: the
// adjoint of g_i(y) is plane 9 + i plus lambda_phi(y), that of q^{n-1}(y)
// plane 28 plus lambda_phi(y)/2, and each reader (kernel A of the next
// reverse step when it pulls, the init kernel) adds the share itself, so B
// moves 20 bytes per cell instead of rewriting ten adjoint planes.
// The terminal kernel seeds Lambda^N for J = 1/2 sum (phi^N - phi_target)^2,
// and the init kernel maps Lambda^0 to dJ/dT_0 (and the init's share of
// dJ/dL, dJ/dsigma) through the barred-equilibrium initialisation.
// Derivatives of the clip of phi to [0, 1] and of the regularised norm are
// taken piecewise (zero / 1/eps on the flat branches).  With the biased
// gradient (LBM_GRAD_BIASED2) the window holds two rings and kernel B also
// gathers from the cells two links away.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "adjoint.h"

namespace lbm {

using L = D2Q9L;

// ------------------------------------------------------------------ helpers
// Element of flat plane k of cell c in a state or adjoint-state buffer: the
// population layout of off_f / off_g (f_i = plane i, g_i = 9 + i, s_i =
// 18 + i), then phi^{n-1} (plane 27) and the lagged source (plane 28).
__device__ __forceinline__ size_t st_idx(int k, size_t c, size_t N) {
    return k < 9 ? off_f(k, c, N) : k < 18 ? off_g(9, k - 9, c, N) : k < 27 ? off_s(k - 18, c, N)
                                                                              : (size_t)k * N + c;
}

// plane of an adjoint state holding lambda_phi = dJ/dphi^n: the adjoint of a
// stored g_i adds it, that of the lagged source half of it
constexpr int LPHI = 29;

// the (f_i, s_i) pair of cell c as one 8-byte load
__device__ __forceinline__ float2 pair_at(const float *__restrict__ buf, int i, size_t c, size_t N) {
    return __ldg(reinterpret_cast<const float2 *>(buf) + ((size_t)i * N + c));
}

// phi - phi_ref from a cell's nine g deviations and its lagged source
__device__ __forceinline__ float phid_sum(const float g[9], float q) {
    float v = g[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) v = __fadd_rn(v, g[i]);
    return fmaf(0.5f, q, v);
}

__device__ __forceinline__ float phid_cell(const float *__restrict__ st, size_t c, size_t N,
                                           const DevParams &P) {
    // phi - phi_ref of a cell from the stored state (g planes 9..17 hold
    // deviations, the lagged source is plane 28)
    float g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = st[st_idx(9 + i, c, N)];
    return phid_sum(g, st[st_idx(28, c, N)]);
}

__device__ __forceinline__ float edot2(int ex, int ey, float a, float b) {
    return (float)ex * a + (float)ey * b;
}

// ------------------------------------------------------------------ terminal
// Lambda^N for J = 1/2 sum_x (phi^N(x) - target(x))^2; J accumulated in FP64.
__global__ void __launch_bounds__(256)
adj_terminal2d_kernel(const float *__restrict__ st, const float *__restrict__ target,
                      float *__restrict__ adj, double *J, const DevParams P) {
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double part = 0.0;
    if (c < N) {
        const float r = phid_cell(st, c, N, P) + P.g_ref - target[c];
        for (int k = 0; k < 29; ++k) adj[st_idx(k, c, N)] = 0.0f;
        adj[(size_t)LPHI * N + c] = r;           // dJ/dphi^N
        part = 0.5 * (double)r * (double)r;
    }
    block_sum3_atomic(part, 0.0, 0.0, J);
}

// ------------------------------------------------------------------ step A
// two blocks per SM: 128 registers, no spills (at one block the kernel is
// latency bound with 8 warps per SM)
// tile of kernel A: 32 x ADJ_TY cells, one thread each (128 registers, 512
// threads per SM)
constexpr int ADJ_TY = 4;

// phi window of a tile with R rings (R = 1 for the central gradient, 2 for
// the biased one)
template <int R> struct AdjWin {
    static constexpr int WX = 32 + 2 * R, WY = ADJ_TY + 2 * R;
};
constexpr int ADJ_WMAX = AdjWin<2>::WX * AdjWin<2>::WY;

// The reverse step of one 32 x ADJ_TY tile.  FAST: the tile and its rings lie
// inside the grid, so no pulled link and no window cell wraps or meets a
// wall.  BIASED: the gradient of Eq. Grad from the second-order biased
// difference (two rings).  Adds the cell's dJ/dL, dJ/dM_phi, dJ/dsigma terms
// to dL, dM, dS.
template <bool FAST, bool BIASED>
__device__ __forceinline__ void adj_a_tile(const float *__restrict__ st, const float *__restrict__ lam_next,
                                           float *__restrict__ lam, float *__restrict__ cst,
                                           const DevParams &P, float *sphi, int x0, int y0,
                                           float &dL, float &dM, float &dS) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    // phi - phi_ref of the tile and its rings in shared memory (each window
    // value formed once, not once per neighbour)
    constexpr int R = BIASED ? 2 : 1;
    constexpr int WX = AdjWin<R>::WX, WY = AdjWin<R>::WY;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < nx && y < ny;
    const size_t c = active ? (size_t)y * nx + x : 0;
    // the cell's own stored state first: its window slot comes from the g
    // values it needs anyway, the ring and ragged slots from plain loads
    float f[9], g[9], s[9], phip = 0.0f, qp = 0.0f;
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float2 fs = pair_at(st, i, c, N);
            f[i] = fs.x + P.enc_c[i];
            g[i] = st[st_idx(9 + i, c, N)];
            s[i] = fs.y;
        }
        phip = st[st_idx(27, c, N)];
        qp = st[st_idx(28, c, N)];
        sphi[(ty + R) * WX + tx + R] = phid_sum(g, qp);
    }
    float lf[9], lg[9], ls[9], l_phip_new = 0.0f, l_q_new = 0.0f;
    if (active) {
        // ---------------- adjoints of the pushed values (pull of Lambda^{n+1})
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // the adjoint of a g value at its target cell adds that cell's
            // lambda_phi (plane LPHI)
            if (FAST) {
                const size_t d = c + (long long)L::ey(i) * nx + L::ex(i);
                const float2 fs = pair_at(lam_next, i, d, N);
                lf[i] = fs.x;
                lg[i] = lam_next[st_idx(9 + i, d, N)] + lam_next[(size_t)LPHI * N + d];
                ls[i] = fs.y;
                continue;
            }
            int dx = x + L::ex(i), dy = y + L::ey(i);
            const int kx = wrap_coord(dx, nx, P.periodic[0]);
            const int ky = wrap_coord(dy, ny, P.periodic[1]);
            if (kx >= 2 || ky >= 2) {
                const int o = L::opp(i);
                const float2 fs = pair_at(lam_next, o, c, N);
                lf[i] = fs.x;
                lg[i] = -(lam_next[st_idx(9 + o, c, N)] + lam_next[(size_t)LPHI * N + c]);
                ls[i] = -fs.y;
            } else {
                const size_t d = (size_t)dy * nx + dx;
                const float2 fs = pair_at(lam_next, i, d, N);
                lf[i] = fs.x;
                lg[i] = lam_next[st_idx(9 + i, d, N)] + lam_next[(size_t)LPHI * N + d];
                ls[i] = fs.y;
            }
        }
        l_phip_new = lam_next[st_idx(27, c, N)];
        l_q_new = fmaf(0.5f, lam_next[(size_t)LPHI * N + c], lam_next[st_idx(28, c, N)]);

    }
    if (FAST && !BIASED) {
        // the ring: the top and bottom rows, then the left and right columns
        constexpr int RING = 2 * WX + 2 * ADJ_TY;
        const int r = threadIdx.x;
        if (r < RING) {
            int wx, wy;
            if (r < WX) { wx = r; wy = 0; }
            else if (r < 2 * WX) { wx = r - WX; wy = WY - 1; }
            else if (r < 2 * WX + ADJ_TY) { wx = 0; wy = 1 + r - 2 * WX; }
            else { wx = WX - 1; wy = 1 + r - 2 * WX - ADJ_TY; }
            sphi[wy * WX + wx] = phid_cell(st, (size_t)(y0 + wy - 1) * nx + (x0 + wx - 1), N, P);
        }
    } else {
        for (int sidx = threadIdx.x; sidx < WX * WY; sidx += blockDim.x) {
            const int wx = sidx % WX, wy = sidx / WX;
            int cx = x0 + wx - R, cy = y0 + wy - R;
            if (wx >= R && wx < 32 + R && wy >= R && wy < ADJ_TY + R && cx < nx && cy < ny) continue;  // owned
            if (FAST) {
                sphi[sidx] = phid_cell(st, (size_t)cy * nx + cx, N, P);
                continue;
            }
            if (cx > nx + R - 1 || cy > ny + R - 1) { sphi[sidx] = 0.0f; continue; }   // beyond a ragged tile
            const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
            const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
            sphi[sidx] = kx >= 2 ? P.phi_wall[kx - 2] - P.g_ref
                       : (ky >= 2 ? P.phi_wall[ky - 2] - P.g_ref : phid_cell(st, (size_t)cy * nx + cx, N, P));
        }
    }
    __syncthreads();
    if (active) {
        // ---------------- forward recomputation
        const float *sp = sphi + (ty + R) * WX + tx + R;
        float nb[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) nb[j] = sp[L::ey(j) * WX + L::ex(j)];
        const float phd = nb[0];
        const float ph = phd + P.g_ref;
        const float nE = nb[1], nN = nb[2], nW = nb[3], nS = nb[4];
        const float nNE = nb[5], nNW = nb[6], nSW = nb[7], nSE = nb[8];
        const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
        const float dA = nNE - nSW, dB = nSE - nNW;
        float gx, gy;
        if (BIASED) {
            // Eq. Grad with [-phi(x + 2e) + 4 phi(x + e) - 3 phi(x)] / 2, pair-folded
            const int W2 = 2 * WX;
            const float bx = 0.5f * fmaf(4.0f, nE - nW, -(sp[2] - sp[-2]));
            const float by = 0.5f * fmaf(4.0f, nN - nS, -(sp[W2] - sp[-W2]));
            const float bA = 0.5f * fmaf(4.0f, dA, -(sp[W2 + 2] - sp[-W2 - 2]));
            const float bB = 0.5f * fmaf(4.0f, dB, -(sp[-W2 + 2] - sp[W2 - 2]));
            gx = 3.0f * fmaf(w1, bx, w5 * (bA + bB));
            gy = 3.0f * fmaf(w1, by, w5 * (bA - bB));
        } else {
            gx = 3.0f * (w1 * (nE - nW) + w5 * (dA + dB));
            gy = 3.0f * (w1 * (nN - nS) + w5 * (dA - dB));
        }
        const float lap = 6.0f * (w1 * ((nE + nW) + (nN + nS) - 4.0f * phd)
                                + w5 * ((nNE + nSW) + (nNW + nSE) - 4.0f * phd));
        const bool inside = ph > 0.0f && ph < 1.0f;
        const float pc = unit_phi(ph);
        const float rho = pc * P.rho_g + (1.0f - pc) * P.rho_l;
        const float grx = P.drho * gx, gry = P.drho * gy;
        const float m3 = ph * (ph - 1.0f) * (ph - 0.5f);
        const float mu = 4.0f * P.H * m3 - P.K * lap;
        const float Fx = mu * gx + (rho - P.rho_l) * P.gravity[0] + P.body[0];
        const float Fy = mu * gy + (rho - P.rho_l) * P.gravity[1] + P.body[1];
        const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
        const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
        float sf = f[0], ss = s[0];
        for (int i = 1; i < 9; ++i) { sf += f[i]; ss += s[i]; }
        // reciprocals and 1/|grad phi| by the one-instruction approximations
        // the forward step uses (rcp.approx / rsqrt.approx)
        const float ir = rcp_approx(rho);
        const float ux = (3.0f * jx + 0.5f * Fx) * ir;
        const float uy = (3.0f * jy + 0.5f * Fy) * ir;
        const float cs2 = L::cs2;
        const float rcs2 = rho * cs2;
        const float p = sf + 0.5f * (cs2 * (ux * grx + uy * gry) + rcs2 * qp * P.kappa);
        const float ug = ux * gx + uy * gy;
        const float X = (phd - phip) + ug + ph * qp * P.kappa;
        const float Lc = P.L_over_Cp, Cl = P.Cp_over_L;
        const float Td = ss - 0.5f * Lc * X;
        const float T = Td + P.s_ref;
        const float alpha = P.alpha_interp == 0 ? pc * P.alpha_g + (1.0f - pc) * P.alpha_l
                                                : P.alpha_l * P.alpha_g / (pc * P.alpha_l + (1.0f - pc) * P.alpha_g);
        const float theta = Cl * (T - P.T_sat);
        const float Th = P.theta_I - theta;
        const float P2 = ph * (1.0f - ph);
        const float q = P.source_on ? -(P.prod_coef * alpha) * Th * P2 : 0.0f;
        const float sq = gx * gx + gy * gy;
        const bool big = sq > P.eps2;
        const float idn = rsqrt_approx(big ? sq : P.eps2);      // 1 / max(|grad phi|, eps)
        const float n0 = gx * idn, n1 = gy * idn;
        const float om_g = P.om_g;
        const float Bv = pc * P.nu_l + (1.0f - pc) * P.nu_g;
        const float iBv = rcp_approx(Bv);
        const float nu = P.visc_interp == 0 ? P.nu_l * P.nu_g * iBv : (1.0f - pc) * P.nu_l + pc * P.nu_g;
        const float om_f = rcp_approx(3.0f * nu + 0.5f);
        const float om_s = rcp_approx(3.0f * alpha + 0.5f);
        const float D = (phd - phip) + ug + ph * q * P.kappa;
        const float usq15 = 1.5f * (ux * ux + uy * uy);
        const float iface = P.four_over_W * P2;
        const float gAx = cs2 * grx, gAy = cs2 * gry;
        const float uA = ux * gAx + uy * gAy, uB = ux * Fx + uy * Fy;
        const float pf = rcs2 * q * P.kappa;
        const float a_g = 1.0f - om_g, b_g = 1.0f - 0.5f * om_g;
        const float a_f = 1.0f - om_f, b_f = 1.0f - 0.5f * om_f;
        const float a_s = 1.0f - om_s, b_s = 1.0f - 0.5f * om_s;
        const float Tref = P.s_ref, gref = P.g_ref;

        // ---------------- reverse sweep
        float l_f[9], l_g[9], l_s[9];
        float l_om_g = 0.f, l_om_f = 0.f, l_om_s = 0.f, l_bsw = 0.f, l_Td = 0.f, l_p = 0.f;
        float l_rcs2 = 0.f, l_pf = 0.f, l_phd = 0.f, l_q = 0.f, l_iface = 0.f, l_usq15 = 0.f;
        float l_ux = 0.f, l_uy = 0.f, l_gAx = 0.f, l_gAy = 0.f, l_Fx = 0.f, l_Fy = 0.f;
        float l_uA = 0.f, l_uB = 0.f, l_n0 = 0.f, l_n1 = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = L::ex(i), ey = L::ey(i);
            const float w = L::w(i);
            const float cu = edot2(ex, ey, ux, uy);
            const float poly = cu * (3.0f + 4.5f * cu) - usq15;
            const float G = w + w * poly, Gw = w * poly;
            const float en = edot2(ex, ey, n0, n1);
            const float eA = edot2(ex, ey, gAx, gAy), eB = edot2(ex, ey, Fx, Fy);
            // s
            l_s[i] = a_s * ls[i];
            // the non-equilibrium parts below are small differences of
            // values of size w_i: their weight products are formed as the
            // forward step forms them (weighted(), no bias from the float
            // weights)
            l_om_s += (weighted<L>(i, fmaf(T, poly, Td)) - s[i]) * ls[i];
            const float l_seq = om_s * ls[i];
            l_bsw += w * ls[i];
            l_Td += G * l_seq;
            float l_G = Td * l_seq, l_Gw = Tref * l_seq;
            // f
            l_f[i] = a_f * lf[i];
            l_om_f += (weighted<L>(i, fmaf(rcs2, poly, p) - 0.5f * fmaf(poly, eA - uA,
                                                                     fmaf(1.0f + poly, eB - uB, pf)))
                       - f[i]) * lf[i];
            const float l_feq = om_f * lf[i], l_fS = b_f * lf[i];
            l_Gw += (eA - uA) * l_fS;
            l_G += (eB - uB) * l_fS;
            const float l_eA = Gw * l_fS, l_eB = G * l_fS;
            l_uA -= Gw * l_fS;
            l_uB -= G * l_fS;
            l_pf += w * l_fS;
            l_gAx += (float)ex * l_eA; l_gAy += (float)ey * l_eA;
            l_Fx += (float)ex * l_eB;  l_Fy += (float)ey * l_eB;
            l_p += w * l_feq;
            l_rcs2 += w * poly * l_feq;
            float l_poly = w * rcs2 * l_feq;
            // g
            l_g[i] = a_g * lg[i];
            l_om_g += (weighted<L>(i, fmaf(ph, poly, phd) - 0.5f * (i == 0 ? q : fmaf(iface, en, q)))
                       - g[i]) * lg[i];
            l_phd += om_g * G * lg[i];
            l_G += om_g * phd * lg[i];
            l_Gw += om_g * gref * lg[i];
            const float l_Sg = b_g * lg[i];
            l_q += w * l_Sg;
            if (i != 0) {
                l_iface += w * en * l_Sg;
                const float l_en = w * iface * l_Sg;
                l_n0 += (float)ex * l_en; l_n1 += (float)ey * l_en;
            }
            // Gamma
            l_poly += w * l_G + w * l_Gw;
            const float l_cu = (3.0f + 9.0f * cu) * l_poly;
            l_usq15 -= l_poly;
            l_ux += (float)ex * l_cu; l_uy += (float)ey * l_cu;
        }
        // bsw = b_s * (-Lc D) enters as w * bsw0 * b_s
        l_om_s += 0.5f * Lc * D * l_bsw;            // b_s = 1 - om_s / 2
        float l_Lc = -b_s * D * l_bsw;
        float l_D = -b_s * Lc * l_bsw;
        // pf = rcs2 q kappa
        l_rcs2 += q * P.kappa * l_pf;
        l_q += rcs2 * P.kappa * l_pf;
        // uA, uB
        l_ux += gAx * l_uA + Fx * l_uB;
        l_uy += gAy * l_uA + Fy * l_uB;
        l_gAx += ux * l_uA; l_gAy += uy * l_uA;
        l_Fx += ux * l_uB; l_Fy += uy * l_uB;
        float l_grx = cs2 * l_gAx, l_gry = cs2 * l_gAy;
        // iface, usq15
        float l_ph = P.four_over_W * (1.0f - 2.0f * ph) * l_iface;
        l_ux += 3.0f * ux * l_usq15;
        l_uy += 3.0f * uy * l_usq15;
        // outputs phi^{n-1} <- phi^n, q^{n-1} <- q^n
        l_phd += l_phip_new;
        l_q += l_q_new;
        // D = (phd - phip) + ug + ph q kappa
        l_phd += l_D;
        float l_phip = -l_D;
        float l_ug = l_D;
        l_ph += q * P.kappa * l_D;
        l_q += ph * P.kappa * l_D;
        // relaxation rates
        float l_alpha = -3.0f * om_s * om_s * l_om_s;
        const float l_nu = -3.0f * om_f * om_f * l_om_f;
        float l_pc = P.visc_interp == 0 ? -P.nu_l * P.nu_g * (P.nu_l - P.nu_g) * (iBv * iBv) * l_nu
                                        : (P.nu_g - P.nu_l) * l_nu;
        // M_phi enters om_g = 1 / (M_phi / cs2_g + 1/2): d om_g / d M_phi = -om_g^2 / cs2_g
        dM += (-om_g * om_g * L::inv_cs2) * l_om_g;
        // normal
        float l_gx = 0.0f, l_gy = 0.0f;
        if (big) {
            const float ndot = n0 * l_n0 + n1 * l_n1;
            l_gx += (l_n0 - n0 * ndot) * idn;
            l_gy += (l_n1 - n1 * ndot) * idn;
        } else {
            l_gx += l_n0 * idn;
            l_gy += l_n1 * idn;
        }
        // production rate
        float l_T = 0.0f, l_Cl = 0.0f;
        if (P.source_on) {
            l_alpha += -P.prod_coef * Th * P2 * l_q;
            const float l_Th = -P.prod_coef * alpha * P2 * l_q;
            const float l_theta = -l_Th;
            l_T += Cl * l_theta;
            l_Cl += (T - P.T_sat) * l_theta;
            l_ph += -P.prod_coef * alpha * Th * (1.0f - 2.0f * ph) * l_q;
        }
        // alpha(pc)
        if (P.alpha_interp == 0) l_pc += (P.alpha_g - P.alpha_l) * l_alpha;
        else {
            const float Ba = pc * P.alpha_l + (1.0f - pc) * P.alpha_g;
            l_pc += -P.alpha_l * P.alpha_g * (P.alpha_l - P.alpha_g) / (Ba * Ba) * l_alpha;
        }
        // T = Td + Tref; Td = ss - Lc X / 2
        l_Td += l_T;
        l_Lc += -0.5f * X * l_Td;
        const float l_X = -0.5f * Lc * l_Td;
        l_phd += l_X;
        l_phip -= l_X;
        l_ug += l_X;
        l_ph += qp * P.kappa * l_X;
        float l_qp = ph * P.kappa * l_X;
        // ug
        l_ux += gx * l_ug; l_uy += gy * l_ug;
        l_gx += ux * l_ug; l_gy += uy * l_ug;
        // p
        l_ux += 0.5f * cs2 * grx * l_p; l_uy += 0.5f * cs2 * gry * l_p;
        l_grx += 0.5f * cs2 * ux * l_p; l_gry += 0.5f * cs2 * uy * l_p;
        l_rcs2 += 0.5f * qp * P.kappa * l_p;
        l_qp += 0.5f * rcs2 * P.kappa * l_p;
        float l_rho = cs2 * l_rcs2;
        // u = (3 j + F / 2) / rho
        const float l_jx = 3.0f * ir * l_ux, l_jy = 3.0f * ir * l_uy;
        l_Fx += 0.5f * ir * l_ux; l_Fy += 0.5f * ir * l_uy;
        const float l_ir = (3.0f * jx + 0.5f * Fx) * l_ux + (3.0f * jy + 0.5f * Fy) * l_uy;
        l_rho += -ir * ir * l_ir;
        // F = mu grad + (rho - rho_l) gravity + body
        const float l_mu = gx * l_Fx + gy * l_Fy;
        l_gx += mu * l_Fx; l_gy += mu * l_Fy;
        l_rho += P.gravity[0] * l_Fx + P.gravity[1] * l_Fy;
        // mu = 4 H m3(ph) - K lap ; K = 1.5 W sigma, H = 12 sigma / W
        l_ph += 4.0f * P.H * (3.0f * ph * ph - 3.0f * ph + 0.5f) * l_mu;
        const float l_lap = -P.K * l_mu;
        // K = 1.5 W sigma, H = 12 sigma / W; 12 / W = 3 (4 / W)
        dS += l_mu * (4.0f * m3 * (3.0f * P.four_over_W) - lap * (1.5f * P.W));
        // gradients of rho
        l_gx += P.drho * l_grx; l_gy += P.drho * l_gry;
        // rho = rho_l + pc drho ; pc = clip(ph)
        l_pc += P.drho * l_rho;
        if (inside) l_ph += l_pc;
        l_phd += l_ph;
        // stencil transpose: the own-cell contribution to phi^n and the
        // adjoints of grad phi and lap phi, from which kernel B forms the
        // contribution 3 w_j e_j.(l_gx, l_gy) + 6 w_j l_lap to phi^n(x + e_j)
        cst[c] = l_phd - 24.0f * (w1 + w5) * l_lap;
        cst[N + c] = l_gx;
        cst[2 * N + c] = l_gy;
        cst[3 * N + c] = l_lap;
        // sums and moments into own populations
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            l_f[i] += l_p + (float)L::ex(i) * l_jx + (float)L::ey(i) * l_jy;
            l_s[i] += l_Td;
            reinterpret_cast<float2 *>(lam)[(size_t)i * N + c] = make_float2(l_f[i], l_s[i]);
            lam[st_idx(9 + i, c, N)] = l_g[i];
        }
        lam[st_idx(27, c, N)] = l_phip;
        lam[st_idx(28, c, N)] = l_qp;
        // latent heat: Lc = L / Cp (d/dL = 1/Cp), Cl = Cp / L (d/dL = -Cp/L^2)
        dL += l_Lc * P.inv_Cp - l_Cl * P.Cp_over_L2;
    }
}

template <bool BIASED>
__global__ void __launch_bounds__(32 * ADJ_TY, 16 / ADJ_TY)
adj_step2d_a_kernel(const float *__restrict__ st, const float *__restrict__ lam_next,
                    float *__restrict__ lam, float *__restrict__ cst, double *dparams,
                    const DevParams P) {
    __shared__ float sphi[ADJ_WMAX];
    pdl_wait();
    constexpr int R = BIASED ? 2 : 1;
    const int nx = P.n[0], ny = P.n[1];
    const int tiles_x = (nx + 31) / 32;
    const int x0 = (int)(blockIdx.x % tiles_x) * 32, y0 = (int)(blockIdx.x / tiles_x) * ADJ_TY;
    const bool fast = x0 >= R && x0 + 32 + R <= nx && y0 >= R && y0 + ADJ_TY + R <= ny;
    float dL = 0.0f, dM = 0.0f, dS = 0.0f;        // this cell's terms (FP32)
    if (fast) adj_a_tile<true, BIASED>(st, lam_next, lam, cst, P, sphi, x0, y0, dL, dM, dS);
    else adj_a_tile<false, BIASED>(st, lam_next, lam, cst, P, sphi, x0, y0, dL, dM, dS);
    block_sum3f_atomic(dL, dM, dS, dparams);
}

// ------------------------------------------------------------------ step B
// One row segment of 256 cells per block (grid: x segments, rows).  Cells
// whose eight neighbours all lie inside the grid take fixed offsets; the
// others wrap periodic axes and skip neighbours beyond a wall.
__global__ void __launch_bounds__(256)
adj_step2d_b_kernel(const float *__restrict__ cst, float *__restrict__ lam, const DevParams P) {
    pdl_wait();
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const size_t c = (size_t)y * nx + x;
    // lambda_phi(y) = c_0(y) + sum_{j >= 1} c_j(y - e_j) over the cells
    // y - e_j that exist (none beyond a wall; periodic axes wrap), with
    // c_j = 3 w_j e_j.(l_gx, l_gy) + 6 w_j l_lap from the four planes of A
    const float *lgx = cst + N, *lgy = cst + 2 * N, *llap = cst + 3 * N;
    float lphi = cst[c];
    if (P.opts & OPT_BIASED) {
        // biased gradient: a cell's gradient adjoint reaches the cells one
        // (6 w_j e_j.l_grad) and two (-3/2 w_j e_j.l_grad) links away; the
        // Laplacian's share stays 6 w_j l_lap on the near ones
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            const float w = L::w(j);
#pragma unroll
            for (int k = 1; k <= 2; ++k) {
                int sx = x - k * L::ex(j), sy = y - k * L::ey(j);
                const int kx = wrap_coord_far(sx, nx, P.periodic[0]);
                const int ky = wrap_coord_far(sy, ny, P.periodic[1]);
                if (kx >= 2 || ky >= 2) continue;        // no such cell
                const size_t sc = (size_t)sy * nx + sx;
                const float eg = edot2(L::ex(j), L::ey(j), __ldg(lgx + sc), __ldg(lgy + sc));
                lphi += k == 1 ? fmaf(6.0f * w, eg, 6.0f * w * __ldg(llap + sc)) : (-1.5f * w) * eg;
            }
        }
    } else if (x >= 1 && x + 1 < nx && y >= 1 && y + 1 < ny) {
        // all eight sources exist: c_j(y - e_j) with fixed offsets; the axis
        // and diagonal weights factored out
        const size_t up = c + nx, dn = c - nx;
        // sources y - e_j: e = +x -> c - 1, -x -> c + 1, +y -> dn, -y -> up
        const float ax = __ldg(lgx + c - 1) - __ldg(lgx + c + 1);
        const float ay = __ldg(lgy + dn) - __ldg(lgy + up);
        const float al = (__ldg(llap + c - 1) + __ldg(llap + c + 1)) + (__ldg(llap + dn) + __ldg(llap + up));
        // diagonals: (1,1) from dn - 1, (-1,1) from dn + 1, (-1,-1) from up + 1, (1,-1) from up - 1
        const float dx = (__ldg(lgx + dn - 1) - __ldg(lgx + up + 1)) + (__ldg(lgx + up - 1) - __ldg(lgx + dn + 1));
        const float dy = (__ldg(lgy + dn - 1) - __ldg(lgy + up + 1)) + (__ldg(lgy + dn + 1) - __ldg(lgy + up - 1));
        const float dl = (__ldg(llap + dn - 1) + __ldg(llap + up + 1)) + (__ldg(llap + dn + 1) + __ldg(llap + up - 1));
        lphi += fmaf(3.0f / 9.0f, ax + ay, fmaf(6.0f / 9.0f, al, fmaf(3.0f / 36.0f, dx + dy, (6.0f / 36.0f) * dl)));
    } else {
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            int sx = x - L::ex(j), sy = y - L::ey(j);
            const int kx = wrap_coord(sx, nx, P.periodic[0]);
            const int ky = wrap_coord(sy, ny, P.periodic[1]);
            if (kx >= 2 || ky >= 2) continue;        // no such cell
            const size_t sc = (size_t)sy * nx + sx;
            const float w = L::w(j);
            lphi += fmaf(3.0f * w, edot2(L::ex(j), L::ey(j), __ldg(lgx + sc), __ldg(lgy + sc)),
                         6.0f * w * __ldg(llap + sc));
        }
    }
    lam[(size_t)LPHI * N + c] = lphi;
}

// ------------------------------------------------------------------ init
// dJ/dT_0(x) and the initialisation's share of dJ/dL, dJ/dsigma from
// Lambda^0, through the barred equilibria of lbm_init (u_0, p_0 and phi_0
// are inputs, not differentiated).
__global__ void __launch_bounds__(256)
adj_init2d_kernel(const float *__restrict__ phi0, const float *__restrict__ T0,
                  const float *__restrict__ ux0, const float *__restrict__ uy0,
                  const float *__restrict__ lam, float *__restrict__ dT0, double *dparams,
                  const DevParams P) {
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double dL = 0.0, dS = 0.0;
    if (c < N) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        float nb[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            int cx = x + L::ex(j), cy = y + L::ey(j);
            const int kx = wrap_coord(cx, nx, P.periodic[0]);
            const int ky = wrap_coord(cy, ny, P.periodic[1]);
            nb[j] = kx >= 2 ? P.phi_wall[kx - 2] : (ky >= 2 ? P.phi_wall[ky - 2] : phi0[(size_t)cy * nx + cx]);
        }
        const float ph = nb[0];
        const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
        const float dA = nb[5] - nb[7], dB = nb[8] - nb[6];
        float gx, gy;
        if (P.opts & OPT_BIASED) {
            // the initialisation's biased gradient (two ghost layers)
            float q2[9];
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                int cx = x + 2 * L::ex(j), cy = y + 2 * L::ey(j);
                const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
                const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
                q2[j] = kx >= 2 ? P.phi_wall[kx - 2] : (ky >= 2 ? P.phi_wall[ky - 2] : phi0[(size_t)cy * nx + cx]);
            }
            const float bx = 0.5f * fmaf(4.0f, nb[1] - nb[3], -(q2[1] - q2[3]));
            const float by = 0.5f * fmaf(4.0f, nb[2] - nb[4], -(q2[2] - q2[4]));
            const float bA = 0.5f * fmaf(4.0f, dA, -(q2[5] - q2[7]));
            const float bB = 0.5f * fmaf(4.0f, dB, -(q2[8] - q2[6]));
            gx = 3.0f * fmaf(w1, bx, w5 * (bA + bB));
            gy = 3.0f * fmaf(w1, by, w5 * (bA - bB));
        } else {
            gx = 3.0f * (w1 * (nb[1] - nb[3]) + w5 * (dA + dB));
            gy = 3.0f * (w1 * (nb[2] - nb[4]) + w5 * (dA - dB));
        }
        const float lap = 6.0f * (w1 * ((nb[1] + nb[3]) + (nb[2] + nb[4]) - 4.0f * ph)
                                + w5 * ((nb[5] + nb[7]) + (nb[6] + nb[8]) - 4.0f * ph));
        const float pc = unit_phi(ph);
        const float rho = pc * P.rho_g + (1.0f - pc) * P.rho_l;
        const float m3 = ph * (ph - 1.0f) * (ph - 0.5f);
        const float ux = ux0 ? ux0[c] : 0.0f, uy = uy0 ? uy0[c] : 0.0f;
        const float T = T0[c];
        const float alpha = P.alpha_interp == 0 ? pc * P.alpha_g + (1.0f - pc) * P.alpha_l
                                                : P.alpha_l * P.alpha_g / (pc * P.alpha_l + (1.0f - pc) * P.alpha_g);
        const float P2 = ph * (1.0f - ph);
        const float Cl = P.Cp_over_L, Lc = P.L_over_Cp;
        const float theta = Cl * (T - P.T_sat);
        const float q = P.source_on ? -(P.prod_coef * alpha) * (P.theta_I - theta) * P2 : 0.0f;
        const float D = (ux * gx + uy * gy) + ph * q * P.kappa;
        const float rcs2 = rho * L::cs2;
        const float usq15 = 1.5f * (ux * ux + uy * uy);
        // the adjoint of g_i adds lambda_phi, that of the lagged source half of it
        const float lphi = lam[(size_t)LPHI * N + c];
        float l_q = fmaf(0.5f, lphi, lam[st_idx(28, c, N)]), l_Td = 0.0f, l_Lc = 0.0f, l_Fx = 0.0f, l_Fy = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float w = L::w(i);
            const float cu = edot2(L::ex(i), L::ey(i), ux, uy);
            const float poly = cu * (3.0f + 4.5f * cu) - usq15;
            const float G = w + w * poly;
            const float lf = lam[st_idx(i, c, N)], lg = lam[st_idx(9 + i, c, N)] + lphi;
            const float ls = lam[st_idx(18 + i, c, N)];
            // f_i = feq - fS/2, fS contains G (e - u).F + w rcs2 q kappa
            l_Fx += -0.5f * G * ((float)L::ex(i) - ux) * lf;
            l_Fy += -0.5f * G * ((float)L::ey(i) - uy) * lf;
            l_q += -0.5f * w * rcs2 * P.kappa * lf;
            // g_i = phi G - (w (iface e.n + q)) / 2 - w phi_ref
            l_q += -0.5f * w * lg;
            // s_i = Td G + Tref (G - w) + w Lc D / 2
            l_Td += G * ls;
            l_Lc += 0.5f * w * D * ls;
            l_q += 0.5f * w * Lc * ph * P.kappa * ls;
        }
        float l_T = l_Td, l_Cl = 0.0f;
        if (P.source_on) {
            l_T += P.prod_coef * alpha * P2 * Cl * l_q;
            l_Cl += P.prod_coef * alpha * P2 * (T - P.T_sat) * l_q;
        }
        dT0[c] = l_T;
        dL = (double)l_Lc * (double)P.inv_Cp - (double)l_Cl * (double)P.Cp_over_L2;
        const float l_mu = gx * l_Fx + gy * l_Fy;
        const double W = 4.0 / (double)P.four_over_W;
        dS = (double)l_mu * (4.0 * (double)m3 * (12.0 / W) - (double)lap * 1.5 * W);
    }
    block_sum3_atomic(dL, 0.0, dS, dparams);
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_adj_terminal2d(const float *st, const float *target, float *adj, double *J,
                                  const DevParams &P, cudaStream_t stream) {
    const int nb = (int)((P.N + 255) / 256);
    adj_terminal2d_kernel<<<nb, 256, 0, stream>>>(st, target, adj, J, P);
    return cudaGetLastError();
}

cudaError_t launch_adj_step2d(const float *st, const float *lam_next, float *lam, float *cst,
                              double *dparams, const DevParams &P, cudaStream_t stream) {
    const int tiles = ((P.n[0] + 31) / 32) * ((P.n[1] + ADJ_TY - 1) / ADJ_TY);
    cudaError_t e;
    if (P.opts & OPT_BIASED)
        e = pdl_launch(adj_step2d_a_kernel<true>, dim3(tiles), dim3(32 * ADJ_TY), 0, stream, st, lam_next, lam,
                       cst, dparams, P);
    else
        e = pdl_launch(adj_step2d_a_kernel<false>, dim3(tiles), dim3(32 * ADJ_TY), 0, stream, st, lam_next, lam,
                       cst, dparams, P);
    if (e != cudaSuccess) return e;
    e = pdl_launch(adj_step2d_b_kernel, dim3((P.n[0] + 255) / 256, P.n[1]), dim3(256), 0, stream,
                   (const float *)cst, lam, P);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adj_init2d(const float *phi0, const float *T0, const float *ux0,
                              const float *uy0, const float *lam, float *dT0, double *dparams,
                              const DevParams &P, cudaStream_t stream) {
    const int nb = (int)((P.N + 255) / 256);
    adj_init2d_kernel<<<nb, 256, 0, stream>>>(phi0, T0, ux0, uy0, lam, dT0, dparams, P);
    return cudaGetLastError();
}

}  // namespace lbm
