// 2D phase field alone in an imposed velocity field (LBM_MODEL_PHASE_FIELD).
//
// The conservative Allen-Cahn scheme of Sec. 3.2 without phase change (q = 0)
// and with the velocity u(x) c(n) prescribed instead of computed from f --
// the setting of the paper's CAC validations (Sec. 4.1).  One launch per step
// over tiles of 64 x 4 (FP32) or 32 x 4 cells (16-bit), the same organisation
// as step2d_kernel for the g set only:
// the tile's 9 g planes are loaded (the halo ring's first, so their L2
// latency overlaps the own loads), phi - phi_ref of the tile and its ring
// goes to shared memory, then each cell forms grad(phi) (Eqs. DerivDirec_Grad,
// Grad), the normal, Gamma(u) (Eq. FunctionGamma) and the collision of Eq. LBE
// with the source F^g of Eq. SourceTerm_AllenCahn, written in the even / odd
// form of the coupled step (E = Ag + Bg P_e, O = e.Vg with Ag = om (phi -
// phi_ref), Bg = om phi, Vg = 3 Bg u + (1 - om/2)(4/W) phi (1 - phi) n), and
// pushes its 9 values.  Algorithmic bytes per cell: the g planes read and
// written and the two velocity components, 9 x 2 x (4 or 2) + 8.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm2d_cell.cuh"

namespace lbm {

template <typename S, bool FAST>
__device__ __forceinline__ void cac_push2d(int i, float v, int x, int y, size_t c,
                                           S *__restrict__ pout, const DevParams &P,
                                           const Planes2d<S> &PL) {
    const int ex = L::ex(i), ey = L::ey(i);
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    if (FAST) {
        // 32-bit cell offsets (fewer than 2^31 cells)
        const int off = ey * nx + ex;
        if (in_bounds((long long)c + off, (long long)N, P)) PL.out[9 + i][(cidx)c + (cidx)off] = narrow<S>(v);
        return;
    }
    int dx = x + ex, dy = y + ey;
    const int kx = wrap_coord(dx, nx, P.periodic[0]);
    const int ky = wrap_coord(dy, ny, P.periodic[1]);
    if (kx >= 2 || ky >= 2) {      // anti bounce-back with the wall's phi
        const int side = (kx >= 2 ? kx : ky) - 2;
        const int o = L::opp(i);
        const float m2 = 2.0f * (IsNarrow<S>::value ? P.set_sc[1] : L::w(i));
        if (in_bounds((long long)c, (long long)N, P))
            pout[off_g(9, o, c, N)] = narrow<S>(fmaf(m2, P.phi_wall[side] - P.g_ref, -v));
    } else {
        const size_t d = (size_t)dy * nx + dx;
        if (in_bounds((long long)d, (long long)N, P)) pout[off_g(9, i, d, N)] = narrow<S>(v);
    }
}

template <typename S, bool FAST, class T>
__device__ __forceinline__ void cac_tile2d(const S *__restrict__ pin, S *__restrict__ pout,
                                           const float *__restrict__ vel, float factor,
                                           const DevParams &P, float *sphi, int x0, int y0,
                                           const Planes2d<S> &PL) {
    constexpr int TX = T::TX, TY = T::TY, SX = T::SX, SY = T::SY;
    static_assert(T::RING <= T::NT, "one halo-ring cell per thread");
    const int nx = P.n[0], ny = P.n[1];
    const size_t N = (size_t)P.N;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = FAST || ((x < nx) && (y < ny));
    const size_t c = active ? (size_t)y * nx + x : 0;
    const float isc = P.set_isc[1];

    // the ring's g values come from L2: requested before the tile's own for
    // FP32, after them for the 16-bit formats (measured +1.6% / +2.6%)
    constexpr int RING = 2 * SX + 2 * TY;
    constexpr bool RING_FIRST = !IsNarrow<S>::value;
    float rv[9];
    int rslot = 0;
    auto load_ring = [&]() {
        if (FAST && tid < RING) {
            int sx, sy;
            if (tid < SX) { sx = tid; sy = 0; }
            else if (tid < 2 * SX) { sx = tid - SX; sy = SY - 1; }
            else if (tid < 2 * SX + TY) { sx = 0; sy = 1 + tid - 2 * SX; }
            else { sx = SX - 1; sy = 1 + tid - 2 * SX - TY; }
            rslot = sy * SX + sx;
            const cidx cc = (cidx)((y0 + sy - 1) * nx + (x0 + sx - 1));
#pragma unroll
            for (int i = 0; i < 9; ++i) rv[i] = load_raw(PL.in[9 + i] + cc);
            (void)in_bounds((long long)cc, (long long)N, P);
        }
    };
    if (RING_FIRST) load_ring();
    float g[9];
    if (active) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = load_raw(PL.in[9 + i] + (cidx)c);
        sphi[(ty + 1) * SX + tx + 1] = set_sum2d<S>(g, isc);          // phi - phi_ref
    }
    if (!RING_FIRST) load_ring();
    if (FAST) {
        if (tid < RING) sphi[rslot] = set_sum2d<S>(rv, isc);
    } else {
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
                float w9[9];
                const size_t cc = (size_t)cy * nx + cx;
#pragma unroll
                for (int i = 0; i < 9; ++i) w9[i] = load_raw(pin + off_g(9, i, cc, N));
                v = set_sum2d<S>(w9, isc);
            }
            sphi[sidx] = v;
        }
    }
    __syncthreads();
    if (!active) return;

    // gradient (Eqs. DerivDirec_Grad, Grad) and the normal
    const float *sp = sphi + (ty + 1) * SX + tx + 1;
    const float phd = sp[0];
    const float ph = phd + P.g_ref;
    const float dA = sp[SX + 1] - sp[-SX - 1], dB = sp[-SX + 1] - sp[SX - 1];
    const float gx = 3.0f * fmaf(1.0f / 9.0f, sp[1] - sp[-1], (1.0f / 36.0f) * (dA + dB));
    const float gy = 3.0f * fmaf(1.0f / 9.0f, sp[SX] - sp[-SX], (1.0f / 36.0f) * (dA - dB));
    const float inv_d = rsqrt_approx(fmaxf(fmaf(gx, gx, gy * gy), P.eps2));
    const float nx_ = gx * inv_d, ny_ = gy * inv_d;
    // imposed velocity
    const float ux = vel[(cidx)c] * factor, uy = (vel + N)[(cidx)c] * factor;

    const float om = P.om_g, a_g = 1.0f - om, b_g = fmaf(-0.5f, om, 1.0f);
    const float Ag = om * phd, Bg = om * ph;
    const float bgi = b_g * (P.four_over_W * ph * (1.0f - ph));
    const float Vgx = fmaf(3.0f * Bg, ux, bgi * nx_), Vgy = fmaf(3.0f * Bg, uy, bgi * ny_);
    const float uxx = ux * ux, uyy = uy * uy, uxy = ux * uy;
    const float usq = fmaf(ux, ux, uyy);
    const float P0 = -1.5f * usq;
    const float Pxa = fmaf(3.0f, uxx, -1.5f * uyy), Pya = fmaf(3.0f, uyy, -1.5f * uxx);
    const float Pd0 = 3.0f * usq;
    // increments in the working representation (split-weight product for FP32)
    auto rep = [&](int i, float v) { return IsNarrow<S>::value ? P.set_sc[1] * v : weighted<L>(i, v); };

    cac_push2d<S, FAST>(0, fmaf(a_g, g[0], rep(0, fmaf(Bg, P0, Ag))), x, y, c, pout, P, PL);
    auto pair = [&](int i, int o, float Pe, float eV) {
        const float E = fmaf(Bg, Pe, Ag);
        cac_push2d<S, FAST>(i, fmaf(a_g, g[i], rep(i, E + eV)), x, y, c, pout, P, PL);
        cac_push2d<S, FAST>(o, fmaf(a_g, g[o], rep(i, E - eV)), x, y, c, pout, P, PL);
    };
    pair(1, 3, Pxa, Vgx);
    pair(2, 4, Pya, Vgy);
    pair(5, 7, fmaf(9.0f, uxy, Pd0), __fadd_rn(Vgx, Vgy));
    pair(6, 8, fmaf(-9.0f, uxy, Pd0), __fsub_rn(Vgy, Vgx));
}

// Tile per storage, chosen by measurement on the 4096^2 vortex (one thread
// per cell, 2048 threads per SM, 32 registers): FP32 64 x 4 (67.1k MLUPS
// against 65.2k for 32 x 8), 16-bit 32 x 4 (82.6k against 80.6k).
template <typename S> struct CacTile { using T = Tile2<32, 4>; };
template <> struct CacTile<float> { using T = Tile2<64, 4>; };

template <typename S>
__global__ void __launch_bounds__(CacTile<S>::T::NT, 2048 / CacTile<S>::T::NT)
cac2d_kernel(const S *__restrict__ pin, S *__restrict__ pout, const float *__restrict__ vel,
             float factor, const DevParams P, const __grid_constant__ Planes2d<S> PL) {
    using T = typename CacTile<S>::T;
    __shared__ float sphi[T::SY * T::SX];
    pdl_wait();
    const int x0 = blockIdx.x * T::TX, y0 = blockIdx.y * T::TY;
    const bool fast = x0 >= 1 && x0 + T::TX + 1 <= P.n[0] && y0 >= 1 && y0 + T::TY + 1 <= P.n[1];
    if (fast) cac_tile2d<S, true, T>(pin, pout, vel, factor, P, sphi, x0, y0, PL);
    else cac_tile2d<S, false, T>(pin, pout, vel, factor, P, sphi, x0, y0, PL);
}

template <typename S>
cudaError_t launch_cac2d(const void *pin, void *pout, const float *vel, float factor,
                         const DevParams &P, cudaStream_t st) {
    using T = typename CacTile<S>::T;
    dim3 block(T::TX, T::TY);
    dim3 grid((P.n[0] + T::TX - 1) / T::TX, (P.n[1] + T::TY - 1) / T::TY);
    pdl_launch(cac2d_kernel<S>, grid, block, 0, st, (const S *)pin, (S *)pout, vel, factor, P,
               planes2d<S>(pin, pout, P));
    return cudaGetLastError();
}

template cudaError_t launch_cac2d<float>(const void *, void *, const float *, float, const DevParams &,
                                         cudaStream_t);
template cudaError_t launch_cac2d<__half>(const void *, void *, const float *, float, const DevParams &,
                                          cudaStream_t);
template cudaError_t launch_cac2d<__nv_bfloat16>(const void *, void *, const float *, float,
                                                 const DevParams &, cudaStream_t);

}  // namespace lbm
