// Shared device-side definitions of the B300 phase-field LB kernels.
//
// Lattices (Sec. 3): D2Q9 e0=(0,0), e1..4 = +x,+y,-x,-y, e5..8 = (1,1),
// (-1,1), (-1,-1), (1,-1); D3Q7 = rest + six axis vectors in the order
// +x,+y,+z,-x,-y,-z; D3Q19 = D3Q7's vectors + face diagonals (+-1,1,0),
// (+-1,-1,0), (+-1,0,1), (+-1,0,-1), (0,+-1,1), (0,+-1,-1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------- lattices
struct D2Q9L {
    static constexpr int Q = 9;
    static __host__ __device__ constexpr int ex(int i) {
        return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
    }
    static __host__ __device__ constexpr int ey(int i) {
        return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
    }
    static __host__ __device__ constexpr int ez(int) { return 0; }
    static __host__ __device__ constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
    static __host__ __device__ constexpr float w(int i) {
        return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
    // w(i) + wlo(i) = the exact weight to about 1e-16 (see weighted())
    static __host__ __device__ constexpr float wlo(int i) {
        return i == 0 ? -3.3113692e-09f : (i <= 4 ? -8.278423e-10f : -2.0696057e-10f);
    }
    static constexpr float cs2 = 1.0f / 3.0f;
    static constexpr float inv_cs2 = 3.0f;
};

// axis part shared by D3Q7 and D3Q19: 1..6 = +x,+y,+z,-x,-y,-z
__host__ __device__ constexpr int axis_e(int i, int a) {
    return (i >= 1 && i <= 6) ? ((i - 1) % 3 == a ? (i <= 3 ? 1 : -1) : 0) : 0;
}

struct D3Q7L {
    static constexpr int Q = 7;
    static __host__ __device__ constexpr int ex(int i) { return axis_e(i, 0); }
    static __host__ __device__ constexpr int ey(int i) { return axis_e(i, 1); }
    static __host__ __device__ constexpr int ez(int i) { return axis_e(i, 2); }
    static __host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 3 ? i + 3 : i - 3); }
    static __host__ __device__ constexpr float w(int i) { return i == 0 ? 0.25f : 0.125f; }
    static __host__ __device__ constexpr float wlo(int) { return 0.0f; }    // weights exact in binary
    static constexpr float cs2 = 0.25f;
    static constexpr float inv_cs2 = 4.0f;
};

struct D3Q19L {
    static constexpr int Q = 19;
    // diagonals 7..18 as (a, b) sign pairs on an axis pair
    static __host__ __device__ constexpr int ex(int i) {
        return i <= 6 ? axis_e(i, 0) : (i <= 14 ? ((i % 2) ? 1 : -1) : 0);
    }
    static __host__ __device__ constexpr int ey(int i) {
        return i <= 6 ? axis_e(i, 1)
             : (i <= 8 ? 1 : (i <= 10 ? -1 : (i <= 14 ? 0 : ((i % 2) ? 1 : -1))));
    }
    static __host__ __device__ constexpr int ez(int i) {
        return i <= 6 ? axis_e(i, 2)
             : (i <= 10 ? 0 : (i <= 12 ? 1 : (i <= 14 ? -1 : (i <= 16 ? 1 : -1))));
    }
    static __host__ __device__ constexpr int opp(int i) {
        // pairs (7,10) (8,9) (11,14) (12,13) (15,18) (16,17)
        return i == 0 ? 0 : (i <= 6 ? (i <= 3 ? i + 3 : i - 3)
             : (i == 7 ? 10 : i == 8 ? 9 : i == 9 ? 8 : i == 10 ? 7
             : i == 11 ? 14 : i == 12 ? 13 : i == 13 ? 12 : i == 14 ? 11
             : i == 15 ? 18 : i == 16 ? 17 : i == 17 ? 16 : 15));
    }
    static __host__ __device__ constexpr float w(int i) {
        return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
    static __host__ __device__ constexpr float wlo(int i) {
        return i == 0 ? -9.934108e-09f : (i <= 6 ? -4.1392115e-10f : -2.0696057e-10f);
    }
    static constexpr float cs2 = 1.0f / 3.0f;
    static constexpr float inv_cs2 = 3.0f;
};

// ---------------------------------------------------------------- parameters
constexpr int MAXQ_TOTAL = 45;   // 19 + 7 + 19

// Everything a kernel needs, precomputed on the host in float.
struct DevParams {
    int n[3];            // nx, ny, nz
    int periodic[3];
    int wall_axis;       // -1 when every axis is periodic
    long long N;         // cells
    float rho_l, rho_g, drho;          // drho = rho_g - rho_l
    float nu_l, nu_g, alpha_l, alpha_g;
    float K, H;                        // Eq. Def_K-H
    float W;                           // interface width
    float four_over_W;                 // 4/W
    float prod_coef;                   // 4 / (A W^2)
    float theta_I, L_over_Cp, Cp_over_L, T_sat;
    float tau_g;                       // M_phi / cs^2 of the phase-field lattice
    float om_g;                        // 1 / (tau_g + 1/2)
    float kappa;                       // 1 - rho_g/rho_l
    float eps2;                        // normal_eps^2
    float gravity[3], body[3];
    float phi_wall[2], T_wall[2];
    int source_on, visc_interp, alpha_interp, storage;
    float s_ref;                       // temperature storage reference T_ref
    float g_ref;                       // phase-field storage reference phi_ref
    float inv_Cp, Cp_over_L2;          // 1/Cp and Cp/L^2 (adjoint of L)
    // storage codec per population plane k (f planes, then g, then s):
    // FP32: theta = d + enc_c[k];  16-bit: theta = enc_c[k] + x * dec_s[k],
    // x = (theta - enc_c[k]) * enc_s[k]
    float enc_c[MAXQ_TOTAL], enc_s[MAXQ_TOTAL], dec_s[MAXQ_TOTAL];
    // per set (f, g, s): storage reference, 16-bit scale and its inverse
    float set_ref[3], set_sc[3], set_isc[3];
    // two-relaxation-time collision: magic parameter of the f, g, s sets
    // (read by the TRT instantiations of the step kernels only)
    float trt_magic[3];
    // multiple-relaxation-time collision of the flow set: rates s_e, s_eps
    // and s_q (read by the MRT instantiations of the step kernels only)
    float mrt_rates[3];
    // and of the phase-field set: s_e, s_eps, s_q, s_p (om_g stored for a 0)
    float mrt_rates_g[4];
    int opts;                          // OPT_TRT | OPT_MRT | OPT_BIASED
#ifdef LBM_CHECK_BOUNDS
    int *dbg;                          // device status word of the bounds checks
#endif
};

// Index check of the bounds-checking build (compiled with LBM_CHECK_BOUNDS):
// an index outside [0, lim) sets bit 2 of the handle's status word and the
// caller skips the access; lbm_sync reports it as LBM_EBOUNDS.  The normal
// build compiles every check away and its kernel parameters keep no status
// pointer (a larger parameter block measurably slowed the 16-bit 2D
// kernels).  Callers never return early on a failed check, so no thread
// leaves a block barrier behind.
__device__ __forceinline__ bool in_bounds(long long idx, long long lim, const DevParams &P) {
#ifdef LBM_CHECK_BOUNDS
    if (idx < 0 || idx >= lim) {
        if (P.dbg) atomicOr(P.dbg, 2);
        return false;
    }
#endif
    (void)idx; (void)lim; (void)P;
    return true;
}

// DevParams::opts: two-relaxation-time collision, biased gradient (Sec. 3.4),
// multiple-relaxation-time collision of the flow set (2D)
constexpr int OPT_TRT = 1, OPT_BIASED = 2, OPT_MRT = 4;
// collision instantiation of the step kernels
constexpr int COLL_BGK = 0, COLL_TRT = 1, COLL_MRT = 2;

// ---------------------------------------------------------------- layout
// Memory layout of a population buffer (and of the saved and the adjoint
// state).  f and s share their lattice (D2Q9 in 2D, D3Q19 in 3D) and the
// values of direction i of both sets travel to the same cell, so they are
// stored as a pair: pair plane i holds (f_i, s_i) of cell c at elements
// 2 (i N + c) and 2 (i N + c) + 1.  The Qg phase-field planes follow the Qf
// pair planes: g_i of cell c at (2 Qf + i) N + c.  A thread moves the f and s
// values of a direction with one 8-byte (FP32) or 4-byte (16-bit) access.
// The flat plane number k that indexes the per-plane codec tables is
// unchanged by the layout: f_i = i, g_i = Qf + i, s_i = Qf + Qg + i.
__host__ __device__ __forceinline__ size_t off_f(int i, size_t c, size_t N) {
    return 2 * ((size_t)i * N + c);
}
__host__ __device__ __forceinline__ size_t off_s(int i, size_t c, size_t N) {
    return 2 * ((size_t)i * N + c) + 1;
}
__host__ __device__ __forceinline__ size_t off_g(int Qf, int i, size_t c, size_t N) {
    return (size_t)(2 * Qf + i) * N + c;
}

template <typename S> struct PairOf;
template <> struct PairOf<float> { using T = float2; };
template <> struct PairOf<__half> { using T = __half2; };
template <> struct PairOf<__nv_bfloat16> { using T = __nv_bfloat162; };

__device__ __forceinline__ void unpack_pair(float2 v, float &a, float &b) { a = v.x; b = v.y; }
__device__ __forceinline__ void unpack_pair(__half2 v, float &a, float &b) {
    a = __low2float(v); b = __high2float(v);
}
__device__ __forceinline__ void unpack_pair(__nv_bfloat162 v, float &a, float &b) {
    a = __low2float(v); b = __high2float(v);
}
template <typename S> __device__ __forceinline__ typename PairOf<S>::T pack_pair(float a, float b);
template <> __device__ __forceinline__ float2 pack_pair<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ __half2 pack_pair<__half>(float a, float b) {
    return __floats2half2_rn(a, b);
}
template <> __device__ __forceinline__ __nv_bfloat162 pack_pair<__nv_bfloat16>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

// The (f_i, s_i) pair of cell c from / to pair plane `plane` (its first
// element), as raw stored values widened to float / narrowed from float.
template <typename S>
__device__ __forceinline__ void load_pair(const S *plane, long long c, float &f, float &s) {
    unpack_pair(__ldg(reinterpret_cast<const typename PairOf<S>::T *>(plane) + c), f, s);
}
// Fast-path cell index: the grid holds fewer than 2^31 cells (checked when
// the handle is created), so a cell index fits 32 bits and a plane element's
// address is one wide multiply-add from the plane base.
using cidx = uint32_t;
template <typename S>
__device__ __forceinline__ void load_pair(const S *plane, cidx c, float &f, float &s) {
    unpack_pair(__ldg(reinterpret_cast<const typename PairOf<S>::T *>(plane) + c), f, s);
}
template <typename S>
__device__ __forceinline__ void store_pair(S *plane, cidx c, float f, float s) {
    reinterpret_cast<typename PairOf<S>::T *>(plane)[c] = pack_pair<S>(f, s);
}
template <typename S>
__device__ __forceinline__ void store_pair(S *plane, long long c, float f, float s) {
    reinterpret_cast<typename PairOf<S>::T *>(plane)[c] = pack_pair<S>(f, s);
}

// ---------------------------------------------------------------- storage
template <typename S> struct Codec;

// load / store convert between the stored value and the full population;
// load_dev / store_dev work on the deviation theta_i - enc_c[k] directly (the
// temperature set is advanced in deviation form, see the step kernels).
template <> struct Codec<float> {
    static __device__ __forceinline__ float load(const float *p, int k, const DevParams &P) {
        return __ldg(p) + P.enc_c[k];
    }
    static __device__ __forceinline__ void store(float *p, float v, int k, const DevParams &P) {
        *p = v - P.enc_c[k];
    }
    static __device__ __forceinline__ float load_dev(const float *p, int, const DevParams &) {
        return __ldg(p);
    }
    static __device__ __forceinline__ void store_dev(float *p, float d, int, const DevParams &) {
        *p = d;
    }
    static __device__ __forceinline__ float dec(float raw, int k, const DevParams &P) {
        return raw + P.enc_c[k];
    }
    static __device__ __forceinline__ float dec_dev(float raw, int, const DevParams &) { return raw; }
};

template <> struct Codec<__half> {
    static __device__ __forceinline__ float load(const __half *p, int k, const DevParams &P) {
        return fmaf(__half2float(__ldg(p)), P.dec_s[k], P.enc_c[k]);
    }
    static __device__ __forceinline__ void store(__half *p, float v, int k, const DevParams &P) {
        *p = __float2half_rn((v - P.enc_c[k]) * P.enc_s[k]);
    }
    // __fmul_rn: the decoded value is rounded here, never folded into a
    // later addition, so every kernel that decodes a value gets the same float
    static __device__ __forceinline__ float load_dev(const __half *p, int k, const DevParams &P) {
        return __fmul_rn(__half2float(__ldg(p)), P.dec_s[k]);
    }
    static __device__ __forceinline__ void store_dev(__half *p, float d, int k, const DevParams &P) {
        *p = __float2half_rn(d * P.enc_s[k]);
    }
    static __device__ __forceinline__ float dec(__half raw, int k, const DevParams &P) {
        return fmaf(__half2float(raw), P.dec_s[k], P.enc_c[k]);
    }
    static __device__ __forceinline__ float dec_dev(__half raw, int k, const DevParams &P) {
        return __fmul_rn(__half2float(raw), P.dec_s[k]);
    }
};

template <> struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p, int k, const DevParams &P) {
        return fmaf(__bfloat162float(__ldg(p)), P.dec_s[k], P.enc_c[k]);
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v, int k, const DevParams &P) {
        *p = __float2bfloat16_rn((v - P.enc_c[k]) * P.enc_s[k]);
    }
    static __device__ __forceinline__ float load_dev(const __nv_bfloat16 *p, int k, const DevParams &P) {
        return __fmul_rn(__bfloat162float(__ldg(p)), P.dec_s[k]);
    }
    static __device__ __forceinline__ void store_dev(__nv_bfloat16 *p, float d, int k, const DevParams &P) {
        *p = __float2bfloat16_rn(d * P.enc_s[k]);
    }
    static __device__ __forceinline__ float dec(__nv_bfloat16 raw, int k, const DevParams &P) {
        return fmaf(__bfloat162float(raw), P.dec_s[k], P.enc_c[k]);
    }
    static __device__ __forceinline__ float dec_dev(__nv_bfloat16 raw, int k, const DevParams &P) {
        return __fmul_rn(__bfloat162float(raw), P.dec_s[k]);
    }
};

// Working representation of a stored value (the fused 2D step): the raw
// stored number widened to float.  FP32 stores the deviation theta - w ref of
// its set; the 16-bit formats store (theta / w - ref) * scale, so the step
// works on that normalised value directly and spends no multiplication on
// decoding or encoding.
template <typename S> struct IsNarrow { static constexpr bool value = true; };
template <> struct IsNarrow<float> { static constexpr bool value = false; };

__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(__half v) { return __half2float(v); }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename S> __device__ __forceinline__ S narrow(float v);
template <> __device__ __forceinline__ float narrow<float>(float v) { return v; }
template <> __device__ __forceinline__ __half narrow<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <typename S> __device__ __forceinline__ float load_raw(const S *p) { return widen(__ldg(p)); }

// w_i x for a lattice weight that binary floating point cannot hold exactly
// (4/9, 1/9, 1/36, 1/3, 1/18): the weight is split into its float value w and
// the remainder wlo, so the product is the correctly rounded w_i x up to a
// rare last-bit tie.  Multiplying by the rounded float weight alone scales
// every post-collision value by the same factor (1 + 3e-8 for 4/9), and the
// weights then no longer sum to one: on a 1000-step film-boiling run that
// systematic bias displaced the interface enough to put phi 3e-5 away from
// the exact (FP64) update, against 7e-6 with the split product.
template <class Lat>
__device__ __forceinline__ float weighted(int i, float x) {
    if (Lat::wlo(i) == 0.0f) return Lat::w(i) * x;
    return fmaf(x, Lat::w(i), __fmul_rn(x, Lat::wlo(i)));
}

// Packed FP32x2 arithmetic (sm_100 and later): one instruction works on two
// lanes, each rounded exactly as fmaf / __fadd_rn / __fmul_rn, so a paired
// expression gives the bits of the two scalar ones.  The step kernels pair
// the flow value of a direction with the temperature value stored beside it.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// weighted() on both lanes (one weight)
template <class Lat>
__device__ __forceinline__ float2 weighted2(int i, float2 x) {
    if (Lat::wlo(i) == 0.0f) return fmul2(splat2(Lat::w(i)), x);
    return ffma2(x, splat2(Lat::w(i)), fmul2(x, splat2(Lat::wlo(i))));
}

// Approximate reciprocal and reciprocal square root, one instruction each
// (PTX rcp.approx.ftz.f32, rsqrt.approx.ftz.f32: about one ulp); used where
// the argument is a density, a relaxation time or a squared norm, never
// subnormal.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The second rate of the two-relaxation-time collision: given the rate om of
// the part that carries the transport coefficient, the rate of the other part
// from the magic parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2), i.e.
// w_other = b / (Lambda om + b/2) with b = 1 - om/2.
__device__ __forceinline__ float trt_other_rate(float om, float magic) {
    const float b = fmaf(-0.5f, om, 1.0f);
    return b * rcp_approx(fmaf(magic, om, 0.5f * b));
}

// ---------------------------------------------------------------- closures
// Sums of two products are written with an explicit fmaf throughout the step
// code: left to the compiler, a*b + c*d may be fused either way round
// depending on the surrounding kernel, and the kernels that share a cell
// update must produce the same bits.
//
// Property closures take phi restricted to the model's range [0, 1]
// (Sec. 2.1): overshoot beyond it is numerical, and at large density ratios
// an unrestricted rho(phi) of Eq. Density would reach zero.
__device__ __forceinline__ float unit_phi(float phi) { return fminf(fmaxf(phi, 0.0f), 1.0f); }

__device__ __forceinline__ float density(float phi, const DevParams &P) {
    phi = unit_phi(phi);
    return fmaf(phi, P.rho_g, (1.0f - phi) * P.rho_l);
}

__device__ __forceinline__ float diffusivity(float phi, const DevParams &P) {
    phi = unit_phi(phi);
    return P.alpha_interp == 0 ? fmaf(phi, P.alpha_g, (1.0f - phi) * P.alpha_l)
                               : P.alpha_l * P.alpha_g / (phi * P.alpha_l + (1.0f - phi) * P.alpha_g);
}

// mdot'''/rho_g of Eq. ProductionRate
__device__ __forceinline__ float production(float phi, float T, const DevParams &P) {
    if (!P.source_on) return 0.0f;
    // theta_I - theta with theta = (Cp/L)(T - T_sat)
    const float dth = fmaf(-P.Cp_over_L, T - P.T_sat, P.theta_I);
    return -(P.prod_coef * diffusivity(phi, P)) * dth * phi * (1.0f - phi);
}

// Periodic wrap / wall test of one coordinate.  Returns 0 in range, 1 wrapped,
// 2 beyond the low wall, 3 beyond the high wall (c is wrapped in place).
__device__ __forceinline__ int wrap_coord(int &c, int n, int periodic) {
    if (c >= 0 && c < n) return 0;
    if (periodic) { c = c < 0 ? c + n : c - n; return 1; }
    return c < 0 ? 2 : 3;
}

// The same for a coordinate up to any distance outside [0, n) (the second
// ghost layer of the biased gradient on an axis of one cell).
__device__ __forceinline__ int wrap_coord_far(int &c, int n, int periodic) {
    if (c >= 0 && c < n) return 0;
    if (periodic) { c = ((c % n) + n) % n; return 1; }
    return c < 0 ? 2 : 3;
}

}  // namespace lbm
