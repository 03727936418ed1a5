// Per-cell pieces of the 3D step (D3Q19 for f and s, D3Q7 for g), shared by
// the z-marching kernel that loads with plain loads (lbm3d.cu) and the one
// that stages each layer with bulk tensor copies (lbm3d_tma.cu).
#pragma once

#include "lbm_common.cuh"

namespace lbm {

using LF = D3Q19L;   // f and s
using LG = D3Q7L;    // g
constexpr int TX = 32, TY = 4, SX = TX + 2, SY = TY + 2, PLANE = SX * SY;
constexpr int ZB = 32;                       // z planes per block
// window of the biased gradient: two rings around the tile, five planes
constexpr int SXB = TX + 4, SYB = TY + 4, PLANEB = SXB * SYB;
// Slots of the biased gradient's five-plane window (plane p in slot
// (p + 2) % NWB): with six, the plane formed for layer z + 2 never
// overwrites one that the slowest threads still read for layer z - 1, so one
// barrier per layer suffices.
constexpr int NWB = 6;
constexpr int QF = 19, QG = 7;
constexpr int G0 = QF, S0 = QF + QG;         // flat plane number of g_0 and of s_0

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
    const float mu = fmaf(-P.K, m.lap, 4.0f * P.H * phi * (phi - 1.0f) * (phi - 0.5f));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.gr[a] = P.drho * m.g[a];
        m.F[a] = fmaf(mu, m.g[a], fmaf(m.rho - P.rho_l, P.gravity[a], P.body[a]));
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
// The step works on the working representation of the stored values (the
// raw number widened to float, see IsNarrow): FP32 deviations theta - w ref,
// or 16-bit (theta / w - ref) * scale.  theta = w ref + mu v with mu = 1 or
// w / scale.

// sum_i mu_i v_i over D3Q7 (g) and D3Q19 (f, s) sets
template <typename S>
__device__ __forceinline__ float set_sum7(const float v[QG], float inv_sc) {
    const float ax = ((v[1] + v[4]) + (v[2] + v[5])) + (v[3] + v[6]);
    if (!IsNarrow<S>::value) return v[0] + ax;
    return fmaf(0.25f, v[0], 0.125f * ax) * inv_sc;
}

template <typename S>
__device__ __forceinline__ float set_sum19(const float v[QF], float inv_sc) {
    const float ax = ((v[1] + v[4]) + (v[2] + v[5])) + (v[3] + v[6]);
    const float dg = (((v[7] + v[10]) + (v[8] + v[9])) + ((v[11] + v[14]) + (v[12] + v[13])))
                   + ((v[15] + v[18]) + (v[16] + v[17]));
    if (!IsNarrow<S>::value) return v[0] + (ax + dg);
    return fmaf(1.0f / 3.0f, v[0], fmaf(1.0f / 18.0f, ax, (1.0f / 36.0f) * dg)) * inv_sc;
}

// set_sum19 of the flow (x) and temperature (y) sets at once, with the
// same sum tree, so each lane equals set_sum19 of its set
template <typename S>
__device__ __forceinline__ float2 set_sum19x2(const float f[QF], const float s[QF], float2 inv_sc) {
    float2 v[QF];
#pragma unroll
    for (int i = 0; i < QF; ++i) v[i] = make_float2(f[i], s[i]);
    const float2 ax = fadd2(fadd2(fadd2(v[1], v[4]), fadd2(v[2], v[5])), fadd2(v[3], v[6]));
    const float2 dg = fadd2(fadd2(fadd2(fadd2(v[7], v[10]), fadd2(v[8], v[9])),
                                  fadd2(fadd2(v[11], v[14]), fadd2(v[12], v[13]))),
                            fadd2(fadd2(v[15], v[18]), fadd2(v[16], v[17])));
    if (!IsNarrow<S>::value) return fadd2(v[0], fadd2(ax, dg));
    return fmul2(ffma2(splat2(1.0f / 3.0f), v[0],
                       ffma2(splat2(1.0f / 18.0f), ax, fmul2(splat2(1.0f / 36.0f), dg))),
                 inv_sc);
}

__device__ __forceinline__ float sgnv(int e, float v) { return e > 0 ? v : -v; }
// e.(a, b, c) for e in {-1, 0, 1}^3 without multiplications; __fadd_rn keeps
// a product among a, b, c from being fused into the sum
__device__ __forceinline__ float edot3(int ex, int ey, int ez, float a, float b, float c) {
    float r = 0.0f;
    bool any = false;
    if (ex != 0) { r = sgnv(ex, a); any = true; }
    if (ey != 0) { r = any ? __fadd_rn(r, sgnv(ey, b)) : sgnv(ey, b); any = true; }
    if (ez != 0) { r = any ? __fadd_rn(r, sgnv(ez, c)) : sgnv(ez, c); }
    return r;
}

// positive half of the D3Q19 directions: each pair (i, opposite) once
__device__ __forceinline__ constexpr int half19(int k) {
    return k < 3 ? k + 1 : (k < 5 ? k + 4 : (k < 7 ? k + 6 : k + 8));   // 1,2,3,7,8,11,12,15,16
}

// sum_i mu_i e_i v_i over a D3Q19 set
template <typename S>
__device__ __forceinline__ void set_flux19(const float v[QF], float inv_sc, float j[3]) {
    float ja[3] = {0.0f, 0.0f, 0.0f}, jd[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k), o = LF::opp(i);
        const float d = v[i] - v[o];
        float *acc = i <= 6 ? ja : jd;
        if (LF::ex(i) != 0) acc[0] += sgnv(LF::ex(i), d);
        if (LF::ey(i) != 0) acc[1] += sgnv(LF::ey(i), d);
        if (LF::ez(i) != 0) acc[2] += sgnv(LF::ez(i), d);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
        j[a] = IsNarrow<S>::value ? fmaf(1.0f / 18.0f, ja[a], (1.0f / 36.0f) * jd[a]) * inv_sc
                                  : ja[a] + jd[a];
}

// phi - phi_ref at one cell
template <typename S>
__device__ __forceinline__ float phid_at(const S *__restrict__ pin, const float *__restrict__ q_in,
                                         size_t cc, size_t N, const DevParams &P) {
    float v[QG];
#pragma unroll
    for (int i = 0; i < QG; ++i) v[i] = load_raw(pin + off_g(QF, i, cc, N));
    (void)in_bounds((long long)cc, (long long)N, P);
    return fmaf(0.5f, q_in[cc], set_sum7<S>(v, P.set_isc[1]));
}

template <typename S>
__device__ __forceinline__ float phi_at(const S *__restrict__ pin, const float *__restrict__ q_in,
                                        size_t cc, size_t N, const DevParams &P) {
    return phid_at<S>(pin, q_in, cc, N, P) + P.g_ref;
}

// Classes of a 32 x TYv column tile (TYv = 4 unless a kernel picks another).  XY_IN: the tile and its halo ring lie
// inside the grid in x and y.  XY_WRAP: the tile lies inside the grid and its
// ring crosses only periodic x / y boundaries (so every x / y link of its
// cells lands on a grid cell after the periodic wrap).  XY_GEN: anything
// else (a ragged tile, or a wall next to the tile), handled generically.
constexpr int XY_GEN = 0, XY_IN = 1, XY_WRAP = 2;

template <int TYv = TY>
__device__ __forceinline__ int tile_class3d(int x0, int y0, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1];
    if (x0 + TX > nx || y0 + TYv > ny) return XY_GEN;
    const bool xin = x0 >= 1 && x0 + TX + 1 <= nx, yin = y0 >= 1 && y0 + TYv + 1 <= ny;
    if (xin && yin) return XY_IN;
    if ((xin || P.periodic[0]) && (yin || P.periodic[1])) return XY_WRAP;
    return XY_GEN;
}

// Fill window slot `slot` with phi of plane z (tile + halo ring).  When
// owners_write is set, each thread whose column is inside the grid has
// already stored its own cell of an in-range plane (own_ok, own_phi); every
// other slot is computed here: phi of the wrapped cell, or the wall's
// Dirichlet value beyond a wall.  XY (a tile class): for XY_IN / XY_WRAP an
// in-range plane needs no wall test, one thread per ring cell.
template <typename S, int XY, int TYv = TY>
__device__ __forceinline__ void fill_plane(float *sphi, int slot, int z, bool owners_write,
                                           bool own_ok, float own_phi, const S *__restrict__ pin,
                                           const float *__restrict__ q_in, int x0, int y0, int tid,
                                           int tx, int ty, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    constexpr int SYv = TYv + 2, PLANEv = SX * SYv;
    float *plane = sphi + slot * PLANEv;
    const bool z_in = z >= 0 && z < nz;
    if (owners_write && own_ok) plane[(ty + 1) * SX + tx + 1] = own_phi;
    if (XY != XY_GEN && z_in && owners_write) {
        constexpr int RING = 2 * SX + 2 * TYv;
        if (tid < RING) {
            int sx, sy;
            if (tid < SX) { sx = tid; sy = 0; }
            else if (tid < 2 * SX) { sx = tid - SX; sy = SYv - 1; }
            else if (tid < 2 * SX + TYv) { sx = 0; sy = 1 + tid - 2 * SX; }
            else { sx = SX - 1; sy = 1 + tid - 2 * SX - TYv; }
            int cx = x0 + sx - 1, cy = y0 + sy - 1;
            if (XY == XY_WRAP) {
                cx = cx < 0 ? cx + nx : (cx >= nx ? cx - nx : cx);
                cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
            }
            const size_t cc = ((size_t)z * ny + cy) * nx + cx;
            plane[sy * SX + sx] = phid_at<S>(pin, q_in, cc, N, P);
        }
        return;
    }
    for (int sidx = tid; sidx < PLANEv; sidx += TX * TYv) {
        const int sx = sidx % SX, sy = sidx / SX;
        int cx = x0 + sx - 1, cy = y0 + sy - 1, cz = z;
        const bool inner = sx >= 1 && sx <= TX && sy >= 1 && sy <= TYv;
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

// Base pointers of the population planes of the buffer read and of the
// buffer written, passed to the kernels as a parameter, so that a load or a
// fast-path store addresses its plane as base + cell: entries 0..18 are the
// (f_i, s_i) pair planes, G0 + i the g planes.
template <typename S> struct Planes3d {
    const S *in[QF + QG];
    S *out[QF + QG];
};

template <typename S>
inline Planes3d<S> planes3d(const void *pin, void *pout, const DevParams &P) {
    Planes3d<S> PL;
    const size_t N = (size_t)P.N;
    for (int i = 0; i < QF; ++i) {
        PL.in[i] = (const S *)pin + off_f(i, 0, N);
        PL.out[i] = (S *)pout + off_f(i, 0, N);
    }
    for (int i = 0; i < QG; ++i) {
        PL.in[G0 + i] = (const S *)pin + off_g(QF, i, 0, N);
        PL.out[G0 + i] = (S *)pout + off_g(QF, i, 0, N);
    }
    return PL;
}

// Multiplier of a wall's Dirichlet term in the working representation: the
// lattice weight for FP32 deviations, the set's scale for 16-bit values.
template <typename S, class Lt>
__device__ __forceinline__ float wall_mul3(int i, int set, const DevParams &P) {
    return IsNarrow<S>::value ? P.set_sc[set] : Lt::w(i);
}

// Multiplier taking a per-weight increment to the working representation:
// the lattice weight for FP32 deviations; 1 for 16-bit values, whose set
// scale is folded into the per-cell collision coefficients instead.
template <typename S, class Lt>
__device__ __forceinline__ float rep_mul3(int i) {
    return IsNarrow<S>::value ? 1.0f : Lt::w(i);
}

// The per-weight increment x in the working representation: w_i x as the
// split-weight product of weighted() for FP32, x itself for 16-bit values.
template <typename S, class Lt>
__device__ __forceinline__ float rep3(int i, float x) {
    return IsNarrow<S>::value ? x : weighted<Lt>(i, x);
}
template <typename S, class Lt>
__device__ __forceinline__ float2 rep3x2(int i, float2 x) {
    return IsNarrow<S>::value ? x : weighted2<Lt>(i, x);
}

// ---- MRT collisions in 3D (an extension outside the paper)
// With d_i = theta_i - theta_eq_bar_i (population units) and an orthogonal
// moment basis M (rows m_k with squared norms N_k), the MRT update is the
// BGK update plus -(M^T diag((s_k - om) / N_k) M d)_i.
//
// D3Q19, flow set, d'Humieres basis: rho and the stress moments p_xx, p_ww,
// p_xy, p_yz, p_xz keep om; e (N = 2394) takes s_e; eps (252), pi_xx (72)
// and pi_ww (24) take s_eps; the nine odd moments j, q, m take s_q.  Those
// nine span every function odd in e, so their share of the correction is
// -(s_q - om) (d_i - d_o) / 2 (o = opposite).  The even share depends only
// on the link's class (rest; x, y, z axis; xy, xz, yz edge) through
//   e     = -30 d_0 - 11 sum_a A_a + 8 sum_ab E_ab
//   eps   =  12 d_0 -  4 sum_a A_a +   sum_ab E_ab
//   pi_xx = -4 A_x + 2 (A_y + A_z) + E_xy + E_xz - 2 E_yz
//   pi_ww = -2 A_y + 2 A_z + E_xy - E_xz
// with A_a the sum of d over the two a-axis links and E_ab over the four
// ab-edge links.  Every product is rounded on its own (__fmul_rn, explicit
// fmaf), so each kernel that runs the correction produces the same bits.
struct Mrt19Even { float r0, ax, ay, az, exy, exz, eyz; };

__device__ __forceinline__ Mrt19Even mrt19_even(float d0, float Ax, float Ay, float Az, float Exy,
                                                float Exz, float Eyz, float de, float dp) {
    const float sA = (Ax + Ay) + Az, sE = (Exy + Exz) + Eyz;
    const float me = fmaf(-30.0f, d0, fmaf(-11.0f, sA, __fmul_rn(8.0f, sE)));
    const float meps = fmaf(12.0f, d0, fmaf(-4.0f, sA, sE));
    const float mxx = fmaf(-4.0f, Ax, fmaf(2.0f, Ay + Az, fmaf(-2.0f, Eyz, Exy + Exz)));
    const float mww = fmaf(2.0f, Az - Ay, Exy - Exz);
    const float Te = __fmul_rn(__fmul_rn(de, 1.0f / 2394.0f), me);
    const float Tp = __fmul_rn(__fmul_rn(dp, 1.0f / 252.0f), meps);
    const float Tx = __fmul_rn(__fmul_rn(dp, 1.0f / 72.0f), mxx);
    const float Tw = __fmul_rn(__fmul_rn(dp, 1.0f / 24.0f), mww);
    Mrt19Even r;
    r.r0 = fmaf(30.0f, Te, __fmul_rn(-12.0f, Tp));
    const float axb = fmaf(11.0f, Te, __fmul_rn(4.0f, Tp));    // common to the axis links
    r.ax = fmaf(4.0f, Tx, axb);
    const float ayz = fmaf(-2.0f, Tx, axb);
    r.ay = fmaf(2.0f, Tw, ayz);
    r.az = fmaf(-2.0f, Tw, ayz);
    const float eb = -fmaf(8.0f, Te, Tp);                      // common to the edge links
    r.exy = eb - (Tx + Tw);
    r.exz = eb - (Tx - Tw);
    r.eyz = fmaf(2.0f, Tx, eb);
    return r;
}

// the even share of the link pair half19(k) (k = 0..8)
__device__ __forceinline__ float mrt19_class(const Mrt19Even &r, int k) {
    return k == 0 ? r.ax : k == 1 ? r.ay : k == 2 ? r.az : k <= 4 ? r.exy : k <= 6 ? r.exz : r.eyz;
}

// D3Q7, phase-field set: rho and j keep om_g (the mobility); e = 7|c|^2 - 6
// (N = 42) takes s_e, the stress moments p_xx = 3c_x^2 - |c|^2 (12) and
// p_ww = c_y^2 - c_z^2 (4) take s_p.  The correction is even: r0 for the
// rest link, r[a] for both links of axis a (A_a as above).
__device__ __forceinline__ void mrt7_even(float d0, float Ax, float Ay, float Az, float de,
                                          float dp, float &r0, float r[3]) {
    const float me = fmaf(-6.0f, d0, (Ax + Ay) + Az);
    const float mxx = fmaf(2.0f, Ax, -(Ay + Az));
    const float mww = Ay - Az;
    const float Te = __fmul_rn(__fmul_rn(de, 1.0f / 42.0f), me);
    const float Tx = __fmul_rn(__fmul_rn(dp, 1.0f / 12.0f), mxx);
    const float Tw = __fmul_rn(__fmul_rn(dp, 0.25f), mww);
    r0 = __fmul_rn(6.0f, Te);
    r[0] = -fmaf(2.0f, Tx, Te);
    const float yz = Tx - Te;
    r[1] = yz - Tw;
    r[2] = yz + Tw;
}

// d_i from the working value v and eqw = theta_eq_bar_i / w_i - ref
template <typename S, class Lt>
__device__ __forceinline__ float mrt_dev3(int i, float v, float eqw, float inv_sc) {
    return IsNarrow<S>::value ? __fmul_rn(Lt::w(i), fmaf(v, inv_sc, -eqw)) : fmaf(-Lt::w(i), eqw, v);
}

// a correction c in population units, in the working representation: c for
// FP32 deviations, c scale / w_i for 16-bit values
template <typename S, class Lt>
__device__ __forceinline__ float mrt_rep3(int i, float c, float sc) {
    const float iw = Lt::Q == 19 ? (i == 0 ? 3.0f : (i <= 6 ? 18.0f : 36.0f)) : (i == 0 ? 4.0f : 8.0f);
    return IsNarrow<S>::value ? __fmul_rn(__fmul_rn(sc, iw), c) : c;
}

// Push from cell c = (x, y, z).  MODE XY_IN: the link stays inside the grid;
// XY_WRAP: it may cross a periodic x / y boundary but not a z edge or a wall;
// XY_GEN: anything.  Through a wall a value comes back to c in the opposite
// direction: unchanged for f (bounce-back), -v + 2 w (value - ref) for g and
// s (anti-bounce-back), in the working representation.  Fast-path stores
// address their plane through PL (base + cell).

// Offset of the cell that link e = (ex, ey, ez) of cell (x, y) reaches, on
// the fast paths: in the grid (XY_IN), or across a periodic x / y edge
// (wrap); the grid holds fewer than 2^31 cells, so it fits an int.
__device__ __forceinline__ int push_off3(int ex, int ey, int ez, int x, int y, bool wrap,
                                         const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1];
    if (!wrap) return (ez * ny + ey) * nx + ex;
    int oxy = 0;
    if (ex > 0) oxy = x == nx - 1 ? 1 - nx : 1;
    if (ex < 0) oxy = x == 0 ? nx - 1 : -1;
    if (ey > 0) oxy += y == ny - 1 ? (1 - ny) * nx : nx;
    if (ey < 0) oxy += y == 0 ? (ny - 1) * nx : -nx;
    return ez * (ny * nx) + oxy;
}

// Push of direction i's g value (D3Q7).
template <typename S, int MODE>
__device__ __forceinline__ void push3d_g(int i, float v, int x, int y, int z, size_t c,
                                         S *__restrict__ pout, const DevParams &P,
                                         const Planes3d<S> &PL) {
    const int ex = LG::ex(i), ey = LG::ey(i), ez = LG::ez(i);
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    if (MODE == XY_IN || MODE == XY_WRAP) {
        const int off = push_off3(ex, ey, ez, x, y, MODE == XY_WRAP, P);
        if (!in_bounds((long long)c + off, (long long)N, P)) return;
        PL.out[G0 + i][(cidx)c + (cidx)off] = narrow<S>(v);
        return;
    }
    int dx = x + ex, dy = y + ey, dz = z + ez;
    const int kx = wrap_coord(dx, nx, P.periodic[0]);
    const int ky = wrap_coord(dy, ny, P.periodic[1]);
    const int kz = wrap_coord(dz, nz, P.periodic[2]);
    if (kx >= 2 || ky >= 2 || kz >= 2) {
        const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
        v = fmaf(2.0f * wall_mul3<S, LG>(i, 1, P), P.phi_wall[side] - P.g_ref, -v);
        if (in_bounds((long long)c, (long long)N, P)) pout[off_g(QF, LG::opp(i), c, N)] = narrow<S>(v);
    } else {
        const size_t d = ((size_t)dz * ny + dy) * nx + dx;
        if (in_bounds((long long)d, (long long)N, P)) pout[off_g(QF, i, d, N)] = narrow<S>(v);
    }
}

// Push of direction i's f and s values (D3Q19) as one (f_i, s_i) pair.
template <typename S, int MODE>
__device__ __forceinline__ void push3d_fs(int i, float vf, float vs, int x, int y, int z, size_t c,
                                          S *__restrict__ pout, const DevParams &P,
                                          const Planes3d<S> &PL) {
    const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const size_t N = (size_t)P.N;
    if (MODE == XY_IN || MODE == XY_WRAP) {
        const int off = push_off3(ex, ey, ez, x, y, MODE == XY_WRAP, P);
        if (!in_bounds((long long)c + off, (long long)N, P)) return;
        store_pair<S>(PL.out[i], (cidx)c + (cidx)off, vf, vs);
        return;
    }
    int dx = x + ex, dy = y + ey, dz = z + ez;
    const int kx = wrap_coord(dx, nx, P.periodic[0]);
    const int ky = wrap_coord(dy, ny, P.periodic[1]);
    const int kz = wrap_coord(dz, nz, P.periodic[2]);
    if (kx >= 2 || ky >= 2 || kz >= 2) {
        const int side = (kx >= 2 ? kx : (ky >= 2 ? ky : kz)) - 2;
        vs = fmaf(2.0f * wall_mul3<S, LF>(i, 2, P), P.T_wall[side] - P.s_ref, -vs);
        if (in_bounds((long long)c, (long long)N, P))
            store_pair<S>(pout + off_f(LF::opp(i), 0, N), (long long)c, vf, vs);
    } else {
        const size_t d = ((size_t)dz * ny + dy) * nx + dx;
        if (in_bounds((long long)d, (long long)N, P)) store_pair<S>(pout + off_f(i, 0, N), (long long)d, vf, vs);
    }
}

// Update of one cell of layer z: stencils from the three window planes,
// moments, closures, production, the three collisions, then the push.  The
// collisions use the even / odd split of the 2D step: with
// poly_i = Gamma_i / w_i - 1 = e.u / cs2 + P_e (P_e even in e),
//   theta*_i - w_i ref = (1 - om)(theta_i - w_i ref) + w_i [E(e_i) + O(e_i)]
//   g (D3Q7, cs2 = 1/4): E = Ag + Bg P_e,                 O = e.Vg
//   f (D3Q19):           E = K0 + K1 P_e + 3 (e.u)(e.Hf),  O = e.Vf + P_e (e.Hf)
//   s (D3Q19):           E = As + Bs P_e,                 O = e.Ws
// (algebraically Eq. LBE with theta_eq_bar = theta_eq - S/2 and the sources of
// Eqs. Forcing, MicroProduction, SourceTerm_AllenCahn, Def_SourceTerms_Temp).
// MODE (see push3d): how the links of this cell are pushed.
// COLL_TRT: see cell_update2d; the rest direction relaxes with the symmetric
// rate, every other output is a1 v_i + a2 v_o + ... (o = opposite).
// COLL_MRT: the BGK update of f and g plus the moment-space correction of
// mrt19_even / mrt7_even (rates mrt_rates, mrt_rates_g; s keeps BGK).
// BIASED: sphi holds the two-ring window planes (plane p in slot
// (p + 2) % NW, the five planes z - 2 .. z + 2 read) and the gradient of
// Eq. Grad uses the second-order biased difference
// [-phi(x + 2e) + 4 phi(x + e) - 3 phi(x)] / 2 (Sec. 3.4).  Otherwise plane
// p of the one-ring window is in slot (p + 1) % NW.
template <typename S, int MODE, int COLL = COLL_BGK, bool BIASED = false, int NW = BIASED ? NWB : 3>
__device__ __forceinline__ void layer_update3d(const float *sphi, int z, int x, int y, size_t c,
                                               const float f[QF], const float s[QF],
                                               const float g[QG], float qp, float phip,
                                               S *__restrict__ pout, float *__restrict__ phi_prev,
                                               float *__restrict__ q_out, const DevParams &P,
                                               const Planes3d<S> &PL) {
    constexpr bool TRT = COLL == COLL_TRT, MRT = COLL == COLL_MRT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    Macro3 m;
    float phd, gx = 0.0f, gy = 0.0f, gz = 0.0f, la = 0.0f, ld = 0.0f;
    if constexpr (!BIASED) {
        const int centre = (ty + 1) * SX + tx + 1;
        // planes z-1, z, z+1 (plane p in window slot (p + 1) % NW)
        const float *pl[3] = {sphi + (z % NW) * PLANE + centre, sphi + ((z + 1) % NW) * PLANE + centre,
                              sphi + ((z + 2) % NW) * PLANE + centre};
        phd = pl[1][0];                      // the window holds phi - phi_ref
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
    } else {
        const int centre = (ty + 2) * SXB + tx + 2;
        const float *pl[5];                  // planes z-2 .. z+2
#pragma unroll
        for (int k = 0; k < 5; ++k) pl[k] = sphi + ((z + k) % NW) * PLANEB + centre;
        phd = pl[2][0];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = half19(k);
            const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
            const int o1 = ey * SXB + ex;
            const float a = pl[2 + ez][o1], b = pl[2 - ez][-o1];
            const float a2 = pl[2 + 2 * ez][2 * o1], b2 = pl[2 - 2 * ez][-2 * o1];
            // a direction and its opposite: w e (4 (a - b) - (a2 - b2)) / 2
            const float d = 0.5f * fmaf(4.0f, a - b, -(a2 - b2)), sm = a + b;
            if (ex != 0) gx += sgnv(ex, d) * LF::w(i);
            if (ey != 0) gy += sgnv(ey, d) * LF::w(i);
            if (ez != 0) gz += sgnv(ez, d) * LF::w(i);
            if (i <= 6) la += sm; else ld += sm;
        }
    }
    const float ph = phd + P.g_ref;
    m.phi = ph;
    m.g[0] = 3.0f * gx; m.g[1] = 3.0f * gy; m.g[2] = 3.0f * gz;
    m.lap = 6.0f * fmaf(1.0f / 18.0f, fmaf(-6.0f, phd, la), (1.0f / 36.0f) * fmaf(-12.0f, phd, ld));
    closures3d(m, P);
    float j[3];
    set_flux19<S>(f, P.set_isc[0], j);
    const float2 sfs = set_sum19x2<S>(f, s, make_float2(P.set_isc[0], P.set_isc[2]));
    const float sf = sfs.x + P.set_ref[0];
    const float ss = sfs.y;                                          // T - T_ref
    const float inv_rho = rcp_approx(m.rho);
#pragma unroll
    for (int a = 0; a < 3; ++a) m.u[a] = fmaf(0.5f, m.F[a], 3.0f * j[a]) * inv_rho;
    const float ux = m.u[0], uy = m.u[1], uz = m.u[2];
    const float rcs2 = m.rho * LF::cs2;
    const float ugr = fmaf(uz, m.gr[2], fmaf(uy, m.gr[1], ux * m.gr[0]));
    const float ug = fmaf(uz, m.g[2], fmaf(uy, m.g[1], ux * m.g[0]));
    m.p = fmaf(0.5f, fmaf(LF::cs2, ugr, (rcs2 * qp) * P.kappa), sf);
    m.Td = fmaf(-0.5f * P.L_over_Cp, fmaf(ph * qp, P.kappa, (phd - phip) + ug), ss);
    m.T = m.Td + P.s_ref;
    const float q = production(ph, m.T, P);
    const float inv_d = rsqrt_approx(fmaxf(fmaf(m.g[2], m.g[2], fmaf(m.g[1], m.g[1], m.g[0] * m.g[0])), P.eps2));
    const float n0 = m.g[0] * inv_d, n1 = m.g[1] * inv_d, n2 = m.g[2] * inv_d;
    const float phu = unit_phi(ph);
    float om_f;
    if (P.visc_interp == 0) {
        const float den = fmaf(phu, P.nu_l - P.nu_g, P.nu_g);
        om_f = den * rcp_approx(fmaf(0.5f, den, 3.0f * P.nu_l * P.nu_g));
    } else {
        om_f = rcp_approx(fmaf(LF::inv_cs2, fmaf(phu, P.nu_g - P.nu_l, P.nu_l), 0.5f));
    }
    const float om_s = rcp_approx(fmaf(LF::inv_cs2, diffusivity(ph, P), 0.5f));
    const float om_g = P.om_g;
    const float D = fmaf(ph * q, P.kappa, (phd - phip) + ug);
    if (in_bounds((long long)c, P.N, P)) {
        phi_prev[c] = phd;       // stored as phi - phi_ref
        q_out[c] = q;
    }

    const float usq = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
    // symmetric (p) and antisymmetric (m) rates: BGK, or TRT with the BGK rate
    // on the part that carries the transport coefficient
    const float omp_f = om_f, omm_g = om_g, omm_s = om_s;
    const float omm_f = TRT ? trt_other_rate(om_f, P.trt_magic[0]) : om_f;
    const float omp_g = TRT ? trt_other_rate(om_g, P.trt_magic[1]) : om_g;
    const float omp_s = TRT ? trt_other_rate(om_s, P.trt_magic[2]) : om_s;
    const float b_g = fmaf(-0.5f, omp_g, 1.0f), b_f = fmaf(-0.5f, omp_f, 1.0f);
    const float b_s = fmaf(-0.5f, omp_s, 1.0f);
    const float bm_g = TRT ? fmaf(-0.5f, omm_g, 1.0f) : b_g;
    const float bm_f = TRT ? fmaf(-0.5f, omm_f, 1.0f) : b_f;
    const float a_g = 1.0f - omp_g, a_f = 1.0f - omp_f, a_s = 1.0f - omp_s;
    const float a1_f = 1.0f - 0.5f * (omp_f + omm_f), a2_f = 0.5f * (omm_f - omp_f);
    const float a1_g = 1.0f - 0.5f * (omp_g + omm_g), a2_g = 0.5f * (omm_g - omp_g);
    const float a1_s = 1.0f - 0.5f * (omp_s + omm_s), a2_s = 0.5f * (omm_s - omp_s);

    // an output plus its MRT correction (the correction is never formed for
    // BGK and TRT)
    auto plus = [&](float v, float cm) { return MRT ? __fadd_rn(v, cm) : v; };

    // phase field on D3Q7: poly = 4 e.u + 8 (e.u)^2 - 2 u^2
    {
        const float iface = P.four_over_W * ph * (1.0f - ph);
        // 16-bit storage: the set's scale folded into the coefficients
        const float sg = IsNarrow<S>::value ? P.set_sc[1] : 1.0f;
        const float Ag = sg * fmaf(omp_g, phd, b_g * q), Bg = sg * (omp_g * ph);
        const float Bgo = TRT ? sg * (omm_g * ph) : Bg;
        const float bgi = sg * (bm_g * iface);
        const float Vg[3] = {fmaf(4.0f * Bgo, ux, bgi * n0), fmaf(4.0f * Bgo, uy, bgi * n1),
                             fmaf(4.0f * Bgo, uz, bgi * n2)};
        const float usq2 = 2.0f * usq;
        // MRT: the correction of the rest link and of each axis pair
        float cg0 = 0.0f, cgA[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (MRT) {
            // g_eq_bar / w - phi_ref: the coefficients above at om = 1, b = -1/2
            const float Agb = fmaf(-0.5f, q, phd);
            const float hif = __fmul_rn(-0.5f, iface);
            const float nn[3] = {n0, n1, n2};
            const float isc = P.set_isc[1];
            const float d0 = mrt_dev3<S, LG>(0, g[0], fmaf(ph, -usq2, Agb), isc);
            float A[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float ua = m.u[a];
                const float Eb = fmaf(ph, fmaf(8.0f * ua, ua, -usq2), Agb);
                const float Vb = fmaf(4.0f * ph, ua, __fmul_rn(hif, nn[a]));
                A[a] = mrt_dev3<S, LG>(a + 1, g[a + 1], Eb + Vb, isc) +
                       mrt_dev3<S, LG>(a + 4, g[a + 4], Eb - Vb, isc);
            }
            float r0, r[3];
            mrt7_even(d0, A[0], A[1], A[2], P.mrt_rates_g[0] - om_g, P.mrt_rates_g[3] - om_g, r0, r);
            cg0 = mrt_rep3<S, LG>(0, r0, P.set_sc[1]);
#pragma unroll
            for (int a = 0; a < 3; ++a) cgA[a] = mrt_rep3<S, LG>(a + 1, r[a], P.set_sc[1]);
        }
        push3d_g<S, MODE>(0, plus(fmaf(a_g, g[0], rep3<S, LG>(0, fmaf(Bg, -usq2, Ag))), cg0),
                            x, y, z, c, pout, P, PL);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ua = m.u[a];
            const float Eg = fmaf(Bg, fmaf(8.0f * ua, ua, -usq2), Ag);
            auto rg = [&](float v) { return rep3<S, LG>(a + 1, v); };
            if (!TRT) {
                push3d_g<S, MODE>(a + 1, plus(fmaf(a_g, g[a + 1], rg(Eg + Vg[a])), cgA[a]), x, y, z, c,
                                  pout, P, PL);
                push3d_g<S, MODE>(a + 4, plus(fmaf(a_g, g[a + 4], rg(Eg - Vg[a])), cgA[a]), x, y, z, c,
                                  pout, P, PL);
            } else {
                push3d_g<S, MODE>(a + 1, fmaf(a1_g, g[a + 1], fmaf(a2_g, g[a + 4], rg(Eg + Vg[a]))),
                                  x, y, z, c, pout, P, PL);
                push3d_g<S, MODE>(a + 4, fmaf(a1_g, g[a + 4], fmaf(a2_g, g[a + 1], rg(Eg - Vg[a]))),
                                  x, y, z, c, pout, P, PL);
            }
        }
    }

    // flow and temperature on D3Q19: poly = 3 e.u + 4.5 (e.u)^2 - 1.5 u^2
    const float usq15 = 1.5f * usq;
    const float hx = fmaf(LF::cs2, m.gr[0], m.F[0]);
    const float hy = fmaf(LF::cs2, m.gr[1], m.F[1]);
    const float hz = fmaf(LF::cs2, m.gr[2], m.F[2]);
    const float hU = fmaf(uz, hz, fmaf(uy, hy, ux * hx));
    const float uB = fmaf(uz, m.F[2], fmaf(uy, m.F[1], ux * m.F[0]));
    // P^f_i / w_i = rho cs2 q kappa, here minus u.F
    const float scf = IsNarrow<S>::value ? P.set_sc[0] : 1.0f;
    const float scs = IsNarrow<S>::value ? P.set_sc[2] : 1.0f;
    const float K0 = scf * fmaf(omp_f, m.p - P.set_ref[0], b_f * fmaf(rcs2 * q, P.kappa, -uB));
    const float K1 = scf * fmaf(omp_f, rcs2, -b_f * hU);
    const float bf = scf * b_f;
    const float Hx = bf * hx, Hy = bf * hy, Hz = bf * hz;
    // the odd part: K1 and H with the antisymmetric rate
    const float K1o = TRT ? scf * fmaf(omm_f, rcs2, -bm_f * hU) : K1;
    const float bfo = TRT ? scf * bm_f : bf;
    const float Hox = TRT ? bfo * hx : Hx, Hoy = TRT ? bfo * hy : Hy, Hoz = TRT ? bfo * hz : Hz;
    const float Vfx = fmaf(3.0f * K1o, ux, bfo * m.F[0]);
    const float Vfy = fmaf(3.0f * K1o, uy, bfo * m.F[1]);
    const float Vfz = fmaf(3.0f * K1o, uz, bfo * m.F[2]);
    const float As = scs * fmaf(omp_s, m.Td, -b_s * P.L_over_Cp * D), Bs = scs * (omp_s * m.T);
    const float Bso = TRT ? scs * (omm_s * m.T) : Bs;
    // __fmul_rn: W enters E +- e.W as a finished product, never fused into the sum
    const float Wx = __fmul_rn(3.0f * Bso, ux), Wy = __fmul_rn(3.0f * Bso, uy), Wz = __fmul_rn(3.0f * Bso, uz);
    // MRT: the even share of f's correction by link class and the odd parts
    // d_i - d_o of the pairs
    Mrt19Even cfe{};
    float fdif[9], hq = 0.0f;
    if constexpr (MRT) {
        // f_eq_bar / w - ref: the coefficients above at om = 1, b = -1/2
        const float K0b = fmaf(-0.5f, fmaf(rcs2 * q, P.kappa, -uB), m.p - P.set_ref[0]);
        const float K1b = fmaf(0.5f, hU, rcs2);
        const float Hbx = __fmul_rn(-0.5f, hx), Hby = __fmul_rn(-0.5f, hy), Hbz = __fmul_rn(-0.5f, hz);
        const float Vbx = fmaf(3.0f * K1b, ux, __fmul_rn(-0.5f, m.F[0]));
        const float Vby = fmaf(3.0f * K1b, uy, __fmul_rn(-0.5f, m.F[1]));
        const float Vbz = fmaf(3.0f * K1b, uz, __fmul_rn(-0.5f, m.F[2]));
        const float isc = P.set_isc[0];
        const float d0 = mrt_dev3<S, LF>(0, f[0], fmaf(K1b, -usq15, K0b), isc);
        float cls[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = half19(k), o = LF::opp(i);
            const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
            const float cu = edot3(ex, ey, ez, ux, uy, uz);
            const float Pe = fmaf(4.5f * cu, cu, -usq15);
            const float eHb = edot3(ex, ey, ez, Hbx, Hby, Hbz);
            const float Eb = fmaf(3.0f * cu, eHb, fmaf(K1b, Pe, K0b));
            const float Ob = fmaf(Pe, eHb, edot3(ex, ey, ez, Vbx, Vby, Vbz));
            const float di = mrt_dev3<S, LF>(i, f[i], Eb + Ob, isc);
            const float dO = mrt_dev3<S, LF>(o, f[o], Eb - Ob, isc);
            cls[k] = di + dO;
            fdif[k] = di - dO;
        }
        cfe = mrt19_even(d0, cls[0], cls[1], cls[2], cls[3] + cls[4], cls[5] + cls[6], cls[7] + cls[8],
                         P.mrt_rates[0] - om_f, P.mrt_rates[1] - om_f);
        hq = -0.5f * (P.mrt_rates[2] - om_f);
    }
    // f and s of a direction as one FP32x2 pair (x: f, y: s), as stored
    const float2 a_fs = make_float2(a_f, a_s);
    {
        float2 v0 = ffma2(a_fs, make_float2(f[0], s[0]),
                          rep3x2<S, LF>(0, make_float2(fmaf(K1, -usq15, K0), fmaf(Bs, -usq15, As))));
        v0.x = plus(v0.x, mrt_rep3<S, LF>(0, cfe.r0, P.set_sc[0]));
        push3d_fs<S, MODE>(0, v0.x, v0.y, x, y, z, c, pout, P, PL);
    }
    const float2 a1_fs = make_float2(a1_f, a1_s), a2_fs = make_float2(a2_f, a2_s);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = half19(k), o = LF::opp(i);
        const int ex = LF::ex(i), ey = LF::ey(i), ez = LF::ez(i);
        const float cu = edot3(ex, ey, ez, ux, uy, uz);
        const float Pe = fmaf(4.5f * cu, cu, -usq15);
        const float eH = edot3(ex, ey, ez, Hx, Hy, Hz);
        const float eHo = TRT ? edot3(ex, ey, ez, Hox, Hoy, Hoz) : eH;
        const float Ef = fmaf(3.0f * cu, eH, fmaf(K1, Pe, K0));
        const float Of = fmaf(Pe, eHo, edot3(ex, ey, ez, Vfx, Vfy, Vfz));
        const float Es = fmaf(Bs, Pe, As);
        const float Os = edot3(ex, ey, ez, Wx, Wy, Wz);
        // (E + O, E - O) of both sets; w_i = w_o: i and o share the weight of i
        const float2 E = make_float2(Ef, Es), O = make_float2(Of, Os);
        const float2 ri = rep3x2<S, LF>(i, fadd2(E, O));
        const float2 ro = rep3x2<S, LF>(i, fadd2(E, make_float2(-Of, -Os)));
        const float2 fsi = make_float2(f[i], s[i]), fso = make_float2(f[o], s[o]);
        float2 vi, vo;
        if (!TRT) {
            vi = ffma2(a_fs, fsi, ri);
            vo = ffma2(a_fs, fso, ro);
            if constexpr (MRT) {
                const float ck = mrt19_class(cfe, k), od = __fmul_rn(hq, fdif[k]);
                vi.x = __fadd_rn(vi.x, mrt_rep3<S, LF>(i, ck + od, P.set_sc[0]));
                vo.x = __fadd_rn(vo.x, mrt_rep3<S, LF>(o, ck - od, P.set_sc[0]));
            }
        } else {
            vi = ffma2(a1_fs, fsi, ffma2(a2_fs, fso, ri));
            vo = ffma2(a1_fs, fso, ffma2(a2_fs, fsi, ro));
        }
        push3d_fs<S, MODE>(i, vi.x, vi.y, x, y, z, c, pout, P, PL);
        push3d_fs<S, MODE>(o, vo.x, vo.y, x, y, z, c, pout, P, PL);
    }
}

// Slots of the phi window of step3d_column: plane p in slot (p + 1) % NW3.
// With four, the plane formed for layer z + 1 never overwrites one that the
// slowest threads still read for layer z - 1, so one barrier per layer
// suffices.
constexpr int NW3 = 4;

// One z-column of a 32x4 tile over layers [blockIdx.z * ZBLK, +ZBLK), every
// value read with plain loads (see lbm3d.cu).
template <typename S, int XY, int COLL = COLL_BGK, int ZBLK = ZB>
__device__ __forceinline__ void step3d_column(const S *__restrict__ pin, S *__restrict__ pout,
                                              float *__restrict__ phi_prev,
                                              const float *__restrict__ q_in,
                                              float *__restrict__ q_out, const DevParams &P,
                                              float *sphi, const Planes3d<S> &PL) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZBLK;
    const int zend = min(zbeg + ZBLK, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = XY != XY_GEN || ((x < nx) && (y < ny));
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;

    float g[QG], qcur = 0.0f;
    // prologue: plane zbeg (own cells kept in registers) and plane zbeg-1;
    // plane p lives in window slot (p + 1) % NW3
    {
        float ph = 0.0f;
        if (col) {
            const size_t c = zbeg * plane_cells + cxy;
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = load_raw(PL.in[G0 + i] + c);
            qcur = q_in[c];
            ph = fmaf(0.5f, qcur, set_sum7<S>(g, P.set_isc[1]));
        }
        fill_plane<S, XY>(sphi, (zbeg + 1) % NW3, zbeg, true, col, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        fill_plane<S, XY_GEN>(sphi, zbeg % NW3, zbeg - 1, false, false, 0.0f, pin, q_in, x0, y0, tid, tx, ty, P);
    }

    for (int z = zbeg; z < zend; ++z) {
        float gn[QG], qnext = 0.0f;
        {
            float ph = 0.0f;
            const bool ok = col && (z + 1 < nz);
            if (ok) {
                const size_t c = (size_t)(z + 1) * plane_cells + cxy;
#pragma unroll
                for (int i = 0; i < QG; ++i) gn[i] = load_raw(PL.in[G0 + i] + (cidx)c);
                qnext = q_in[c];
                ph = fmaf(0.5f, qnext, set_sum7<S>(gn, P.set_isc[1]));
            }
            fill_plane<S, XY>(sphi, (z + 2) % NW3, z + 1, true, ok, ph, pin, q_in, x0, y0, tid, tx, ty, P);
        }
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            float f[QF], s[QF];
#pragma unroll
            for (int i = 0; i < QF; ++i) load_pair<S>(PL.in[i], (cidx)c, f[i], s[i]);
            const float phip = phi_prev[c];
            if (XY != XY_GEN && z >= 1 && z + 1 < nz)
                layer_update3d<S, XY, COLL, false, NW3>(sphi, z, x, y, c, f, s, g, qcur, phip, pout, phi_prev, q_out, P, PL);
            else
                layer_update3d<S, XY_GEN, COLL, false, NW3>(sphi, z, x, y, c, f, s, g, qcur, phip, pout, phi_prev, q_out, P, PL);
        }
#pragma unroll
        for (int i = 0; i < QG; ++i) g[i] = gn[i];
        qcur = qnext;
    }
}

// phi - phi_ref of window slot (sx, sy) of plane z of the two-ring window:
// the wall's Dirichlet value beyond a wall, wrapped on periodic axes (to any
// distance, for axes shorter than the ring)
template <typename S>
__device__ __forceinline__ float window_phid_b(int cx, int cy, int cz, const S *__restrict__ pin,
                                               const float *__restrict__ q_in, const DevParams &P) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int kx = wrap_coord_far(cx, nx, P.periodic[0]);
    const int ky = wrap_coord_far(cy, ny, P.periodic[1]);
    const int kz = wrap_coord_far(cz, nz, P.periodic[2]);
    if (kx >= 2) return P.phi_wall[kx - 2] - P.g_ref;
    if (ky >= 2) return P.phi_wall[ky - 2] - P.g_ref;
    if (kz >= 2) return P.phi_wall[kz - 2] - P.g_ref;
    return phid_at<S>(pin, q_in, ((size_t)cz * ny + cy) * nx + cx, (size_t)P.N, P);
}

// One z-column with the biased gradient: a rolling window of five planes,
// each of the tile and two rings, every value formed from plain loads.
// XY: the tile class, used for the push of interior layers as in
// step3d_column.
template <typename S, int XY, int COLL>
__device__ __forceinline__ void step3d_column_biased(const S *__restrict__ pin, S *__restrict__ pout,
                                                     float *__restrict__ phi_prev,
                                                     const float *__restrict__ q_in,
                                                     float *__restrict__ q_out, const DevParams &P,
                                                     float *sphi, const Planes3d<S> &PL) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * ZB;
    const int zend = min(zbeg + ZB, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool col = (x < nx) && (y < ny);
    const size_t cxy = col ? (size_t)y * nx + x : 0;
    const size_t plane_cells = (size_t)nx * ny;
    auto fill = [&](int p) {                 // plane p into slot (p + 2) % NWB
        float *pl = sphi + ((p + 2 + NWB * 4) % NWB) * PLANEB;
        for (int sidx = tid; sidx < PLANEB; sidx += TX * TY)
            pl[sidx] = window_phid_b<S>(x0 + sidx % SXB - 2, y0 + sidx / SXB - 2, p, pin, q_in, P);
    };
    for (int p = zbeg - 2; p <= zbeg + 1; ++p) fill(p);
    for (int z = zbeg; z < zend; ++z) {
        fill(z + 2);
        __syncthreads();
        if (col) {
            const size_t c = (size_t)z * plane_cells + cxy;
            float f[QF], s[QF], g[QG];
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = load_raw(PL.in[G0 + i] + c);
#pragma unroll
            for (int i = 0; i < QF; ++i) load_pair<S>(PL.in[i], (cidx)c, f[i], s[i]);
            const float qp = q_in[c], phip = phi_prev[c];
            if (XY != XY_GEN && z >= 1 && z + 1 < nz)
                layer_update3d<S, XY, COLL, true>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P, PL);
            else
                layer_update3d<S, XY_GEN, COLL, true>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P, PL);
        }
    }
}

}  // namespace lbm
