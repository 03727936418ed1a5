// C ABI of the phase-field LB solver (declarations and contracts in
// include/lbm_pf.h).  Host-side validation, workspace carving, dispatch to the
// 2D / 3D kernels and host <-> device transfers.  No cudaMalloc anywhere: the
// caller provides the device workspace.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm_pf.h"
#include "lbm_kernels.h"
#include "lbm3d.h"
#include "adjoint.h"
#include "lbm2d_tma.h"
#include "lbm3d_tma.h"

using namespace lbm;

struct lbm_handle {
    lbm_grid grid;
    int32_t lattice;
    lbm_params params;
    DevParams dp;
    cudaStream_t stream;
    int dim, Qf, Qg, Qtot;
    size_t elem;             // bytes per stored population value
    size_t N;
    void *pops[2];
    float *phi_prev;
    float *q[2];
    float *scratch;          // 6 planes of N floats
    double *partial;         // 2 doubles per reduction block
    double *red_out;         // 2 doubles
    int red_blocks;
    int cur;
    int64_t steps;
    int32_t last_launches;
    int *err;                // device error word (bounded waits that expired)
    int kernel_choice;       // LBM_KERNEL_*
    int tma_state;           // 0 not set up, 1 ready, -1 not available
    int tma_blocks;
    lbm::TmaMaps2d maps;
    lbm::TmaMaps3d maps3;
    int err_ready;           // the status word has been cleared on the device
    float *vel;              // LBM_MODEL_PHASE_FIELD: imposed velocity, dim planes
    double vel_period;       // time factor cos(pi n / period) when > 0
    int vel_set;
    int32_t health_every;    // lbm_set_health_check: steps between checks (0 = off)
    float health_excess;     // allowed |phi - 1/2|
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t pops, phi, q, scratch, partial, red, err, vel, total;
    int red_blocks;
};

int lattice_dims(int32_t lattice, int *dim, int *Qf, int *Qg) {
    if (lattice == LBM_D2Q9) { *dim = 2; *Qf = 9; *Qg = 9; return LBM_OK; }
    if (lattice == LBM_D3Q19_D3Q7) { *dim = 3; *Qf = 19; *Qg = 7; return LBM_OK; }
    return LBM_EINVAL;
}

size_t elem_size(int32_t storage) { return storage == LBM_STORE_FP32 ? 4 : 2; }

int validate(const lbm_grid *g, int32_t lattice, const lbm_params *p) {
    if (!g || !p) return LBM_EINVAL;
    int dim, Qf, Qg;
    if (lattice_dims(lattice, &dim, &Qf, &Qg) != LBM_OK) return LBM_EINVAL;
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return LBM_EINVAL;
    if (dim == 2 && g->nz != 1) return LBM_EINVAL;
    const double N = (double)g->nx * g->ny * g->nz;
    if (N >= 2147483647.0) return LBM_EINVAL;          // int32 stream-map indices
    int walls = 0;
    for (int a = 0; a < dim; ++a) walls += g->periodic[a] ? 0 : 1;
    if (walls > 1) return LBM_EINVAL;
    if (!(p->rho_l > 0 && p->rho_g > 0 && p->nu_l > 0 && p->nu_g > 0 && p->alpha_l > 0 &&
          p->alpha_g > 0 && p->W > 0 && p->M_phi > 0 && p->A != 0 && p->L != 0 && p->Cp != 0 &&
          p->sigma >= 0 && p->normal_eps > 0))
        return LBM_EINVAL;
    if (p->storage < LBM_STORE_FP32 || p->storage > LBM_STORE_BF16) return LBM_EINVAL;
    if (p->model != LBM_MODEL_COUPLED && p->model != LBM_MODEL_PHASE_FIELD) return LBM_EINVAL;
    if (p->model == LBM_MODEL_PHASE_FIELD && p->source_on) return LBM_EINVAL;   // no phase change
    if (p->collision != LBM_COLLISION_BGK && p->collision != LBM_COLLISION_TRT &&
        p->collision != LBM_COLLISION_MRT)
        return LBM_EINVAL;
    if (p->grad_scheme != LBM_GRAD_CENTRAL && p->grad_scheme != LBM_GRAD_BIASED2) return LBM_EINVAL;
    if (p->grad_scheme == LBM_GRAD_BIASED2 && p->model != LBM_MODEL_COUPLED) return LBM_EUNSUPPORTED;
    if (p->collision == LBM_COLLISION_TRT) {
        for (int s = 0; s < 3; ++s)
            if (!(p->trt_magic[s] > 0.0 && std::isfinite(p->trt_magic[s]))) return LBM_EINVAL;
        if (p->model != LBM_MODEL_COUPLED) return LBM_EUNSUPPORTED;
    }
    if (p->collision == LBM_COLLISION_MRT) {
        for (int k = 0; k < 3; ++k)
            if (!(p->mrt_rates[k] > 0.0 && p->mrt_rates[k] < 2.0)) return LBM_EINVAL;
        for (int k = 0; k < 4; ++k)
            if (!(p->mrt_rates_g[k] == 0.0 || (p->mrt_rates_g[k] > 0.0 && p->mrt_rates_g[k] < 2.0)))
                return LBM_EINVAL;
        if (p->model != LBM_MODEL_COUPLED) return LBM_EUNSUPPORTED;
    }
    const double vals[] = {p->rho_l, p->rho_g, p->nu_l, p->nu_g, p->alpha_l, p->alpha_g, p->sigma,
                           p->W, p->M_phi, p->A, p->theta_I, p->L, p->Cp, p->T_sat,
                           p->gravity[0], p->gravity[1], p->gravity[2], p->body_force[0],
                           p->body_force[1], p->body_force[2], p->phi_wall[0], p->phi_wall[1],
                           p->T_wall[0], p->T_wall[1], p->normal_eps};
    for (double v : vals)
        if (!std::isfinite(v)) return LBM_EINVAL;
    return LBM_OK;
}

Layout layout(const lbm_grid *g, int32_t lattice, const lbm_params *p) {
    int dim, Qf, Qg;
    lattice_dims(lattice, &dim, &Qf, &Qg);
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    const size_t Qtot = (size_t)(2 * Qf + Qg);
    Layout L;
    L.pops = align_up(Qtot * N * elem_size(p->storage));
    L.phi = align_up(N * sizeof(float));
    L.q = align_up(N * sizeof(float));
    L.scratch = align_up(6 * N * sizeof(float));
    L.red_blocks = moment_blocks((long long)N);
    L.partial = align_up((size_t)L.red_blocks * 2 * sizeof(double));
    L.red = align_up(2 * sizeof(double));
    L.err = align_up(sizeof(int));
    L.vel = p->model == LBM_MODEL_PHASE_FIELD ? align_up((size_t)dim * N * sizeof(float)) : 0;
    L.total = 2 * L.pops + L.phi + 2 * L.q + L.scratch + L.partial + L.red + L.err + L.vel;
    return L;
}

// The 3D TMA-staged kernel runs the biased gradient only on grids without
// ragged tiles (nx a multiple of 32, ny of 4); the central gradient anywhere.
bool tma3_gradient_ok(const lbm_handle *h) {
    if (h->params.grad_scheme == LBM_GRAD_CENTRAL) return true;
    return h->dim == 3 && h->grid.nx % 32 == 0 && h->grid.ny % 4 == 0;
}

// What AUTO selects in 3D: the TMA kernel, except with the biased gradient
// and FP32 storage, where the tiled kernel measured faster on 256 x 256 x 512
// (13.3k against 12.9k MLUPS; FP16: TMA 20.6k against tiled 15.4k).
bool tma3_auto(const lbm_handle *h) {
    if (!tma3_gradient_ok(h)) return false;
    return h->params.grad_scheme == LBM_GRAD_CENTRAL || h->params.storage != LBM_STORE_FP32;
}

void fill_devparams(lbm_handle *h) {
    const lbm_params &p = h->params;
    DevParams &d = h->dp;
    std::memset(&d, 0, sizeof(d));
    d.n[0] = h->grid.nx; d.n[1] = h->grid.ny; d.n[2] = h->grid.nz;
    d.wall_axis = -1;
    for (int a = 0; a < 3; ++a) {
        d.periodic[a] = (a < h->dim) ? (h->grid.periodic[a] ? 1 : 0) : 1;
        if (!d.periodic[a]) d.wall_axis = a;
    }
    d.N = (long long)h->N;
    d.rho_l = (float)p.rho_l; d.rho_g = (float)p.rho_g; d.drho = (float)(p.rho_g - p.rho_l);
    d.nu_l = (float)p.nu_l; d.nu_g = (float)p.nu_g;
    d.alpha_l = (float)p.alpha_l; d.alpha_g = (float)p.alpha_g;
    d.K = (float)(1.5 * p.W * p.sigma);
    d.H = (float)(12.0 * p.sigma / p.W);
    d.four_over_W = (float)(4.0 / p.W);
    d.W = (float)p.W;
    d.prod_coef = (float)(4.0 / (p.A * p.W * p.W));
    d.theta_I = (float)p.theta_I;
    d.L_over_Cp = (float)(p.L / p.Cp);
    d.Cp_over_L = (float)(p.Cp / p.L);
    d.T_sat = (float)p.T_sat;
    const double cs2_g = h->dim == 2 ? 1.0 / 3.0 : 0.25;
    d.tau_g = (float)(p.M_phi / cs2_g);
    d.om_g = (float)(1.0 / (p.M_phi / cs2_g + 0.5));
    d.kappa = (float)(1.0 - p.rho_g / p.rho_l);
    d.eps2 = (float)(p.normal_eps * p.normal_eps);
    for (int a = 0; a < 3; ++a) { d.gravity[a] = (float)p.gravity[a]; d.body[a] = (float)p.body_force[a]; }
    for (int k = 0; k < 2; ++k) { d.phi_wall[k] = (float)p.phi_wall[k]; d.T_wall[k] = (float)p.T_wall[k]; }
    d.source_on = p.source_on ? 1 : 0;
    d.visc_interp = p.visc_interp;
    d.alpha_interp = p.alpha_interp;
    d.storage = p.storage;
    d.s_ref = (float)p.store_ref[2];
    d.g_ref = (float)p.store_ref[1];
    d.inv_Cp = (float)(1.0 / p.Cp);
#ifdef LBM_CHECK_BOUNDS
    d.dbg = h->err;
#endif
    d.Cp_over_L2 = (float)(p.Cp / (p.L * p.L));
    d.opts = (p.collision == LBM_COLLISION_TRT ? OPT_TRT : 0) |
             (p.collision == LBM_COLLISION_MRT ? OPT_MRT : 0) |
             (p.grad_scheme == LBM_GRAD_BIASED2 ? OPT_BIASED : 0);
    for (int s = 0; s < 3; ++s) d.trt_magic[s] = (float)p.trt_magic[s];
    for (int k = 0; k < 3; ++k) d.mrt_rates[k] = (float)p.mrt_rates[k];
    for (int k = 0; k < 4; ++k) d.mrt_rates_g[k] = p.mrt_rates_g[k] == 0.0 ? d.om_g : (float)p.mrt_rates_g[k];
    // codec constants, planes ordered f (Qf), g (Qg), s (Qf)
    int k = 0;
    for (int set = 0; set < 3; ++set) {
        const int Q = set == 1 ? h->Qg : h->Qf;
        const double scale = p.store_scale[set] != 0.0 ? p.store_scale[set] : 1.0;
        d.set_ref[set] = (float)p.store_ref[set];
        d.set_sc[set] = p.storage == LBM_STORE_FP32 ? 1.0f : (float)scale;
        d.set_isc[set] = p.storage == LBM_STORE_FP32 ? 1.0f : (float)(1.0 / scale);
        for (int i = 0; i < Q; ++i, ++k) {
            double w;   // exact lattice weights in double
            if (h->dim == 2) w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
            else if (set == 1) w = i == 0 ? 0.25 : 0.125;
            else w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            d.enc_c[k] = (float)(w * p.store_ref[set]);
            if (p.storage == LBM_STORE_FP32) { d.enc_s[k] = 1.0f; d.dec_s[k] = 1.0f; }
            else { d.enc_s[k] = (float)(scale / w); d.dec_s[k] = (float)(w / scale); }
        }
    }
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

// ---- dispatch on storage type and dimension
// Lazily prepare the TMA-staged kernel of the handle's dimension (needs a
// device): eligibility, tensor maps over this handle's buffers, shared-memory
// limit, grid size.
void setup_tma(lbm_handle *h) {
    h->tma_state = -1;
    const int es = (int)h->elem;
    if (h->dim == 2 ? !lbm::tma2d_eligible(h->dp, es) : !lbm::tma3d_eligible(h->dp, es)) return;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return;
    const int per_sm = h->dim == 2 ? lbm::tma2d_blocks_per_sm(es) : lbm::tma3d_blocks_per_sm(es);
    if (per_sm < 1) return;
    if (h->dim == 2) {
        if (lbm::make_tma_maps2d(&h->maps, h->dp, es, h->pops, h->q, h->phi_prev) != 0) return;
    } else {
        if (lbm::make_tma_maps3d(&h->maps3, h->dp, es, h->pops, h->q, h->phi_prev) != 0) return;
    }
    if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return;
    h->tma_blocks = sms * per_sm;
    h->tma_state = 1;
}

int do_step(lbm_handle *h) {
    const int nxt = h->cur ^ 1;
    cudaError_t e;
    if (h->params.model == LBM_MODEL_PHASE_FIELD) {
        const double n = (double)h->steps;
        const float factor = h->vel_period > 0.0 ? (float)std::cos(M_PI * n / h->vel_period) : 1.0f;
        if (h->dim == 2) {
            switch (h->params.storage) {
            case LBM_STORE_FP32: e = launch_cac2d<float>(h->pops[h->cur], h->pops[nxt], h->vel, factor, h->dp, h->stream); break;
            case LBM_STORE_FP16: e = launch_cac2d<__half>(h->pops[h->cur], h->pops[nxt], h->vel, factor, h->dp, h->stream); break;
            default: e = launch_cac2d<__nv_bfloat16>(h->pops[h->cur], h->pops[nxt], h->vel, factor, h->dp, h->stream); break;
            }
        } else {
            // the lagged-source buffers hold zeros in this model
            const float *qz = h->q[h->cur];
            switch (h->params.storage) {
            case LBM_STORE_FP32: e = launch_cac3d<float>(h->pops[h->cur], h->pops[nxt], qz, h->vel, factor, h->dp, h->stream); break;
            case LBM_STORE_FP16: e = launch_cac3d<__half>(h->pops[h->cur], h->pops[nxt], qz, h->vel, factor, h->dp, h->stream); break;
            default: e = launch_cac3d<__nv_bfloat16>(h->pops[h->cur], h->pops[nxt], qz, h->vel, factor, h->dp, h->stream); break;
            }
        }
        if (e != cudaSuccess) return LBM_ECUDA;
        h->cur = nxt;
        return LBM_OK;
    }
    if (h->dim == 2 && h->kernel_choice == LBM_KERNEL_TMA) {
        if (h->tma_state == 0) setup_tma(h);
        if (h->tma_state == 1) {
            switch (h->params.storage) {
            case LBM_STORE_FP32: e = launch_step2d_tma<float>(h->maps, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
            case LBM_STORE_FP16: e = launch_step2d_tma<__half>(h->maps, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
            default: e = launch_step2d_tma<__nv_bfloat16>(h->maps, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
            }
            if (e != cudaSuccess) return LBM_ECUDA;
            h->cur = nxt;
            return LBM_OK;
        }
        if (h->kernel_choice == LBM_KERNEL_TMA) return LBM_EUNSUPPORTED;
    }
    // 3D: AUTO resolves to the TMA-staged kernel whenever it is available
    const bool tma3 = h->dim == 3 && (h->kernel_choice == LBM_KERNEL_TMA ||
                                      (h->kernel_choice == LBM_KERNEL_AUTO && tma3_auto(h)));
    if (tma3 && h->tma_state == 0) setup_tma(h);
    if (h->dim == 3 && h->kernel_choice == LBM_KERNEL_TMA && h->tma_state != 1) return LBM_EUNSUPPORTED;
    if (tma3 && h->tma_state == 1) {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_step3d_tma<float>(h->maps3, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_step3d_tma<__half>(h->maps3, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
        default: e = launch_step3d_tma<__nv_bfloat16>(h->maps3, h->cur, h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->err, h->dp, h->stream); break;
        }
        if (e != cudaSuccess) return LBM_ECUDA;
        h->cur = nxt;
        return LBM_OK;
    }
    if (h->dim == 2) {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_step2d<float>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_step2d<__half>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        default: e = launch_step2d<__nv_bfloat16>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        }
    } else {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_step3d<float>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_step3d<__half>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        default: e = launch_step3d<__nv_bfloat16>(h->pops[h->cur], h->pops[nxt], h->phi_prev, h->q[h->cur], h->q[nxt], h->dp, h->stream); break;
        }
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    h->cur = nxt;
    return LBM_OK;
}

int do_macro(lbm_handle *h, float *o_phi, float *o_T, float *o_u[3], float *o_p, double *partial) {
    float *phi_tmp = h->scratch;   // plane 0 of the scratch
    const double Cp = h->params.Cp, Lh = h->params.L;
    cudaError_t e;
    if (h->dim == 2) {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_macro2d<float>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u[0], o_u[1], o_p, partial, Cp, Lh, h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_macro2d<__half>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u[0], o_u[1], o_p, partial, Cp, Lh, h->dp, h->stream); break;
        default: e = launch_macro2d<__nv_bfloat16>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u[0], o_u[1], o_p, partial, Cp, Lh, h->dp, h->stream); break;
        }
    } else {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_macro3d<float>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u, o_p, partial, Cp, Lh, h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_macro3d<__half>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u, o_p, partial, Cp, Lh, h->dp, h->stream); break;
        default: e = launch_macro3d<__nv_bfloat16>(h->pops[h->cur], phi_tmp, h->phi_prev, h->q[h->cur], o_phi, o_T, o_u, o_p, partial, Cp, Lh, h->dp, h->stream); break;
        }
    }
    return cuda_status(e);
}

int do_init(lbm_handle *h, const float *phi0, const float *T0, const float *u0[3], const float *p0) {
    cudaError_t e;
    if (h->dim == 2) {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_init2d<float>(phi0, T0, u0[0], u0[1], p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_init2d<__half>(phi0, T0, u0[0], u0[1], p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        default: e = launch_init2d<__nv_bfloat16>(phi0, T0, u0[0], u0[1], p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        }
    } else {
        switch (h->params.storage) {
        case LBM_STORE_FP32: e = launch_init3d<float>(phi0, T0, u0, p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        case LBM_STORE_FP16: e = launch_init3d<__half>(phi0, T0, u0, p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        default: e = launch_init3d<__nv_bfloat16>(phi0, T0, u0, p0, h->pops[h->cur], h->phi_prev, h->q[h->cur], h->dp, h->stream); break;
        }
    }
    return cuda_status(e);
}

// Stage one input field as float32 on the device (scratch plane `slot`).
int stage_in(lbm_handle *h, const void *src, int on_device, int dtype, int slot, const float **out) {
    *out = nullptr;
    if (!src) return LBM_OK;
    float *dst = h->scratch + (size_t)slot * h->N;
    const size_t N = h->N;
    if (on_device) {
        if (dtype == 0) { *out = (const float *)src; return LBM_OK; }
        if (dtype != 1) return LBM_EINVAL;
        if (launch_convert_f64_to_f32((const double *)src, dst, N, h->stream) != cudaSuccess) return LBM_ECUDA;
    } else {
        if (dtype == 0) {
            if (cudaMemcpyAsync(dst, src, N * sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return LBM_ECUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
        } else if (dtype == 1) {
            std::vector<float> tmp(N);
            const double *s = (const double *)src;
            for (size_t i = 0; i < N; ++i) tmp[i] = (float)s[i];
            if (cudaMemcpyAsync(dst, tmp.data(), N * sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return LBM_ECUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
        } else return LBM_EINVAL;
    }
    *out = dst;
    return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_strerror(int code) {
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "workspace or buffer too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENONFINITE: return "non-finite value in the fields";
    case LBM_ETIMEOUT: return "timeout";
    case LBM_EBOUNDS: return "an index check of the bounds-checking build failed";
    case LBM_EUNSUPPORTED: return "unsupported combination";
    default: return "unknown error";
    }
}

int lbm_workspace_bytes(const lbm_grid *grid, int32_t lattice, const lbm_params *params, size_t *bytes) {
    if (!bytes) return LBM_EINVAL;
    const int v = validate(grid, lattice, params);
    if (v != LBM_OK) return v;
    *bytes = layout(grid, lattice, params).total;
    return LBM_OK;
}

int lbm_create(const lbm_grid *grid, int32_t lattice, const lbm_params *params, void *workspace,
               size_t workspace_bytes, void *stream, lbm_handle **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    const int v = validate(grid, lattice, params);
    if (v != LBM_OK) return v;
    if (!workspace || ((uintptr_t)workspace % ALIGN) != 0) return LBM_EINVAL;
    const Layout L = layout(grid, lattice, params);
    if (workspace_bytes < L.total) return LBM_ENOMEM;
    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ENOMEM;
    h->grid = *grid;
    if (lattice == LBM_D2Q9) { h->grid.nz = 1; h->grid.periodic[2] = 1; }
    h->lattice = lattice;
    h->params = *params;
    lattice_dims(lattice, &h->dim, &h->Qf, &h->Qg);
    h->Qtot = 2 * h->Qf + h->Qg;
    h->elem = elem_size(params->storage);
    h->N = (size_t)grid->nx * grid->ny * grid->nz;
    h->stream = (cudaStream_t)stream;
    char *p = (char *)workspace;
    h->pops[0] = p; p += L.pops;
    h->pops[1] = p; p += L.pops;
    h->phi_prev = (float *)p; p += L.phi;
    h->q[0] = (float *)p; p += L.q;
    h->q[1] = (float *)p; p += L.q;
    h->scratch = (float *)p; p += L.scratch;
    h->partial = (double *)p; p += L.partial;
    h->red_out = (double *)p; p += L.red;
    h->err = (int *)p; p += L.err;
    h->vel = L.vel ? (float *)p : nullptr; p += L.vel;
    h->vel_period = 0.0;
    h->vel_set = 0;
    h->health_every = 0;
    h->health_excess = 0.0f;
    h->err_ready = 0;
    h->red_blocks = L.red_blocks;
    h->kernel_choice = LBM_KERNEL_AUTO;
    h->tma_state = 0;
    h->tma_blocks = 0;
    h->cur = 0;
    h->steps = 0;
    h->last_launches = 0;
    fill_devparams(h);
    *out = h;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle *h, void *stream) {
    if (!h) return LBM_EINVAL;
    h->stream = (cudaStream_t)stream;
    return LBM_OK;
}

// The phase-field-only kernels write the g planes alone: copy the current
// population buffer into the other one, so that the flow and temperature
// planes read after an odd number of steps hold the initial values (finite
// moments, reductions and state checks) instead of whatever the workspace
// held.
static int mirror_unstepped(lbm_handle *h) {
    const size_t bytes = (size_t)h->Qtot * h->N * h->elem;
    if (cudaMemcpyAsync(h->pops[h->cur ^ 1], h->pops[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int lbm_init(lbm_handle *h, const lbm_fields *in) {
    if (!h || !in || !in->phi || !in->T) return LBM_EINVAL;
    const float *phi0, *T0, *p0, *u0[3] = {nullptr, nullptr, nullptr};
    int r;
    if ((r = stage_in(h, in->phi, in->on_device, in->dtype, 0, &phi0)) != LBM_OK) return r;
    if ((r = stage_in(h, in->T, in->on_device, in->dtype, 1, &T0)) != LBM_OK) return r;
    if ((r = stage_in(h, in->ux, in->on_device, in->dtype, 2, &u0[0])) != LBM_OK) return r;
    if ((r = stage_in(h, in->uy, in->on_device, in->dtype, 3, &u0[1])) != LBM_OK) return r;
    if (h->dim == 3 && (r = stage_in(h, in->uz, in->on_device, in->dtype, 4, &u0[2])) != LBM_OK) return r;
    if ((r = stage_in(h, in->p, in->on_device, in->dtype, 5, &p0)) != LBM_OK) return r;
    if (h->params.model == LBM_MODEL_PHASE_FIELD) {
        // the populations start from the imposed velocity (factor 1 at n = 0)
        u0[0] = h->vel_set ? h->vel : nullptr;
        u0[1] = h->vel_set ? h->vel + h->N : nullptr;
        if (h->dim == 3) u0[2] = h->vel_set ? h->vel + 2 * h->N : nullptr;
    }
    h->cur = 0;
    h->steps = 0;
    if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return LBM_ECUDA;
    h->err_ready = 1;
    // the phase-field-only kernel leaves the lagged source alone (it is zero
    // without phase change): the buffer read after an odd step must hold zeros too
    if (h->params.model == LBM_MODEL_PHASE_FIELD &&
        cudaMemsetAsync(h->q[1], 0, h->N * sizeof(float), h->stream) != cudaSuccess)
        return LBM_ECUDA;
    const int r0 = do_init(h, phi0, T0, u0, p0);
    if (r0 != LBM_OK || h->params.model != LBM_MODEL_PHASE_FIELD) return r0;
    return mirror_unstepped(h);
}

// the periodic state check after a step, when one is due
static int maybe_health(lbm_handle *h) {
    if (h->health_every <= 0 || h->steps % h->health_every != 0) return LBM_OK;
    cudaError_t e;
    switch (h->params.storage) {
    case LBM_STORE_FP32: e = launch_health<float>(h->pops[h->cur], h->q[h->cur], h->health_excess, h->err, h->dp, h->dim, h->stream); break;
    case LBM_STORE_FP16: e = launch_health<__half>(h->pops[h->cur], h->q[h->cur], h->health_excess, h->err, h->dp, h->dim, h->stream); break;
    default: e = launch_health<__nv_bfloat16>(h->pops[h->cur], h->q[h->cur], h->health_excess, h->err, h->dp, h->dim, h->stream); break;
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    ++h->last_launches;
    return LBM_OK;
}

int lbm_step(lbm_handle *h, int32_t n) {
    if (!h || n < 0) return LBM_EINVAL;
    h->last_launches = 0;
    for (int32_t k = 0; k < n; ++k) {
        int r = do_step(h);
        if (r != LBM_OK) return r;
        ++h->steps;
        ++h->last_launches;
        r = maybe_health(h);
        if (r != LBM_OK) return r;
    }
    return LBM_OK;
}

int lbm_set_health_check(lbm_handle *h, int32_t every, float phi_excess) {
    if (!h || every < 0) return LBM_EINVAL;
    if (every > 0 && !(phi_excess > 0.0f && std::isfinite(phi_excess))) return LBM_EINVAL;
    h->health_every = every;
    h->health_excess = phi_excess;
    return LBM_OK;
}

static int copy_state(lbm_handle *h, void *buf, size_t bytes, int32_t on_device, bool save);

// One 2D step of the coupled model on the tiled kernel from the state (in
// populations, phi^{n-1}, lagged source) to another; phi^{n-1} is copied
// into the output first, since the kernel reads and rewrites it in place.
static int step2d_between(lbm_handle *h, const void *in_pops, const float *in_pp, const float *in_q,
                          void *out_pops, float *out_pp, float *out_q) {
    if (cudaMemcpyAsync(out_pp, in_pp, h->N * sizeof(float), cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    cudaError_t e;
    switch (h->params.storage) {
    case LBM_STORE_FP32: e = launch_step2d<float>(in_pops, out_pops, out_pp, in_q, out_q, h->dp, h->stream); break;
    case LBM_STORE_FP16: e = launch_step2d<__half>(in_pops, out_pops, out_pp, in_q, out_q, h->dp, h->stream); break;
    default: e = launch_step2d<__nv_bfloat16>(in_pops, out_pops, out_pp, in_q, out_q, h->dp, h->stream); break;
    }
    return cuda_status(e);
}

int lbm_step_record(lbm_handle *h, int32_t n, void *buf, size_t stride) {
    if (!h || n < 0 || (!buf && n > 0)) return LBM_EINVAL;
    size_t need;
    lbm_state_bytes(h, &need);
    if (stride < need) return LBM_ENOMEM;
    h->last_launches = 0;
    // 2D coupled model on the tiled kernel without the periodic check: step
    // k reads record slot k - 1 (the handle's state for k = 0) and writes
    // slot k directly, and only the last slot is copied back into the
    // handle, instead of a state copy after every step
    const size_t pb = (size_t)h->Qtot * h->N * h->elem, sb = h->N * sizeof(float);
    if (n > 0 && h->dim == 2 && h->params.model == LBM_MODEL_COUPLED &&
        h->kernel_choice != LBM_KERNEL_TMA && h->health_every <= 0 && (uintptr_t)buf % 16 == 0 &&
        stride % 16 == 0 && pb % 16 == 0) {
        char *b = (char *)buf;
        for (int32_t k = 0; k < n; ++k) {
            char *out = b + (size_t)k * stride;
            const char *in = b + (size_t)(k - 1) * stride;
            const int r = k == 0
                ? step2d_between(h, h->pops[h->cur], h->phi_prev, h->q[h->cur], out, (float *)(out + pb),
                                 (float *)(out + pb + sb))
                : step2d_between(h, in, (const float *)(in + pb), (const float *)(in + pb + sb), out,
                                 (float *)(out + pb), (float *)(out + pb + sb));
            if (r != LBM_OK) return r;
            ++h->steps;
            ++h->last_launches;
        }
        return copy_state(h, b + (size_t)(n - 1) * stride, stride, 1, false);
    }
    for (int32_t k = 0; k < n; ++k) {
        int r = do_step(h);
        if (r != LBM_OK) return r;
        ++h->steps;
        ++h->last_launches;
        r = maybe_health(h);
        if (r != LBM_OK) return r;
        r = copy_state(h, (char *)buf + (size_t)k * stride, stride, 1, true);
        if (r != LBM_OK) return r;
    }
    return LBM_OK;
}

int lbm_get_fields(lbm_handle *h, lbm_fields *out) {
    if (!h || !out) return LBM_EINVAL;
    if (out->dtype != 0 && out->dtype != 1) return LBM_EINVAL;
    void *dsts[6] = {out->phi, out->T, out->ux, out->uy, h->dim == 3 ? out->uz : nullptr, out->p};
    float *dev[6];
    const bool direct = out->on_device && out->dtype == 0;
    // scratch plane 0 holds phi_tmp; planes 1..5 stage outputs (phi shares plane 1
    // with T only when both requested, so phi staging uses the destination or plane 5)
    float *stage[6] = {nullptr, h->scratch + 1 * h->N, h->scratch + 2 * h->N, h->scratch + 3 * h->N,
                       h->scratch + 4 * h->N, h->scratch + 5 * h->N};
    for (int k = 0; k < 6; ++k) {
        if (!dsts[k]) { dev[k] = nullptr; continue; }
        dev[k] = direct ? (float *)dsts[k] : (k == 0 ? nullptr : stage[k]);
    }
    // phi output: staged through phi_tmp itself (plane 0 holds the moment phi)
    float *o_phi = (dsts[0] && direct) ? (float *)dsts[0] : nullptr;
    float *o_u[3] = {dev[2], dev[3], dev[4]};
    int r = do_macro(h, o_phi, dev[1], o_u, dev[5], nullptr);
    if (r != LBM_OK) return r;
    if (direct) return LBM_OK;
    dev[0] = dsts[0] ? h->scratch : nullptr;   // phi moment lives in plane 0
    const size_t N = h->N;
    for (int k = 0; k < 6; ++k) {
        if (!dsts[k]) continue;
        if (out->on_device) {   // float64 device output
            if (launch_convert_f32_to_f64(dev[k], (double *)dsts[k], N, h->stream) != cudaSuccess) return LBM_ECUDA;
        } else if (out->dtype == 0) {
            if (cudaMemcpyAsync(dsts[k], dev[k], N * sizeof(float), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return LBM_ECUDA;
        } else {
            std::vector<float> tmp(N);
            if (cudaMemcpyAsync(tmp.data(), dev[k], N * sizeof(float), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return LBM_ECUDA;
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
            double *d = (double *)dsts[k];
            for (size_t i = 0; i < N; ++i) d[i] = tmp[i];
        }
    }
    if (!out->on_device && cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}

int lbm_reduce_async(lbm_handle *h, double *d_out) {
    if (!h || !d_out) return LBM_EINVAL;
    float *none[3] = {nullptr, nullptr, nullptr};
    const int r = do_macro(h, nullptr, nullptr, none, nullptr, h->partial);
    if (r != LBM_OK) return r;
    return cuda_status(launch_final_sum2(h->partial, h->red_blocks, d_out, h->stream));
}

int lbm_reduce(lbm_handle *h, double *phi_mass, double *energy) {
    if (!h) return LBM_EINVAL;
    int r = lbm_reduce_async(h, h->red_out);
    if (r != LBM_OK) return r;
    double host[2];
    if (cudaMemcpyAsync(host, h->red_out, sizeof(host), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return LBM_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
    if (phi_mass) *phi_mass = host[0];
    if (energy) *energy = host[1];
    if (!std::isfinite(host[0]) || !std::isfinite(host[1])) return LBM_ENONFINITE;
    return LBM_OK;
}

int lbm_state_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_EINVAL;
    *bytes = (size_t)h->Qtot * h->N * h->elem + 2 * h->N * sizeof(float);
    return LBM_OK;
}

static int copy_state(lbm_handle *h, void *buf, size_t bytes, int32_t on_device, bool save) {
    size_t need;
    lbm_state_bytes(h, &need);
    if (!buf) return LBM_EINVAL;
    if (bytes < need) return LBM_ENOMEM;
    const size_t pb = (size_t)h->Qtot * h->N * h->elem, sb = h->N * sizeof(float);
    char *b = (char *)buf;
    void *dev[3] = {h->pops[h->cur], h->phi_prev, h->q[h->cur]};
    const size_t sz[3] = {pb, sb, sb};
    size_t off = 0;
    cudaMemcpyKind kind = save ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                               : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = save ? cudaMemcpyAsync(b + off, dev[k], sz[k], kind, h->stream)
                             : cudaMemcpyAsync(dev[k], b + off, sz[k], kind, h->stream);
        if (e != cudaSuccess) return LBM_ECUDA;
        off += sz[k];
    }
    if (!on_device && cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}

int lbm_get_state(lbm_handle *h, void *dst, size_t bytes, int32_t on_device) {
    if (!h) return LBM_EINVAL;
    return copy_state(h, dst, bytes, on_device, true);
}

int lbm_set_state(lbm_handle *h, const void *src, size_t bytes, int32_t on_device) {
    if (!h) return LBM_EINVAL;
    const int r = copy_state(h, const_cast<void *>(src), bytes, on_device, false);
    if (r != LBM_OK) return r;
    if (h->params.model == LBM_MODEL_PHASE_FIELD) {
        if (cudaMemsetAsync(h->q[h->cur ^ 1], 0, h->N * sizeof(float), h->stream) != cudaSuccess)
            return LBM_ECUDA;
        const int rm = mirror_unstepped(h);
        if (rm != LBM_OK) return rm;
    }
    h->steps = 0;
    if (cudaMemsetAsync(h->err, 0, sizeof(int), h->stream) != cudaSuccess) return LBM_ECUDA;
    h->err_ready = 1;
    return LBM_OK;
}

int lbm_stream_map(lbm_handle *h, int32_t set, int32_t *src_index, int8_t *kind) {
    if (!h || !src_index || !kind || set < 0 || set > 1) return LBM_EINVAL;
    cudaError_t e;
    if (h->dim == 2) e = launch_streammap2d(src_index, kind, h->dp, h->stream);
    else e = launch_streammap3d(set, src_index, kind, h->dp, h->stream);
    return cuda_status(e);
}

int lbm_steps_done(const lbm_handle *h, int64_t *steps) {
    if (!h || !steps) return LBM_EINVAL;
    *steps = h->steps;
    return LBM_OK;
}

int lbm_last_launches(const lbm_handle *h, int32_t *launches) {
    if (!h || !launches) return LBM_EINVAL;
    *launches = h->last_launches;
    return LBM_OK;
}

int lbm_sync(lbm_handle *h) {
    if (!h) return LBM_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_ECUDA;
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (!h->err_ready) return LBM_OK;          // no kernel has run yet
    // the status word: bit 1 a bounded wait expired, bit 2 an index check of
    // the bounds-checking build failed, bit 4 the periodic state check failed
    int flag = 0;
    if (cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ECUDA;
    if (flag) {
        cudaMemset(h->err, 0, sizeof(int));
        if (flag & 2) return LBM_EBOUNDS;
        if (flag & 1) return LBM_ETIMEOUT;
        return LBM_ENONFINITE;
    }
    return LBM_OK;
}

int lbm_set_kernel(lbm_handle *h, int32_t kernel) {
    if (!h || kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_TMA) return LBM_EINVAL;
    if (kernel == LBM_KERNEL_TMA) {
        // the biased gradient's two-ring window: the 3D TMA kernel on grids
        // without ragged tiles, otherwise the tiled kernels alone
        if (h->params.grad_scheme != LBM_GRAD_CENTRAL && (h->dim != 3 || !tma3_gradient_ok(h)))
            return LBM_EUNSUPPORTED;
        if (h->tma_state == 0) setup_tma(h);
        if (h->tma_state != 1) return LBM_EUNSUPPORTED;
    }
    h->kernel_choice = kernel;
    return LBM_OK;
}

int lbm_get_kernel(const lbm_handle *h, int32_t *kernel) {
    if (!h || !kernel) return LBM_EINVAL;
    if (h->dim == 3 && h->kernel_choice == LBM_KERNEL_AUTO && h->tma_state == 0)
        setup_tma(const_cast<lbm_handle *>(h));
    const bool tma = h->params.model == LBM_MODEL_COUPLED &&
                     (h->kernel_choice == LBM_KERNEL_TMA ||
                      (h->dim == 3 && h->kernel_choice == LBM_KERNEL_AUTO && tma3_auto(h)));
    if (tma && h->tma_state == 1) *kernel = LBM_KERNEL_TMA;
    else *kernel = LBM_KERNEL_TILED;
    return LBM_OK;
}

static int adjoint_supported(const lbm_handle *h) {
    if (!h) return LBM_EINVAL;
    if (h->dim != 2 || h->params.storage != LBM_STORE_FP32 ||
        h->params.model != LBM_MODEL_COUPLED || h->params.collision != LBM_COLLISION_BGK)
        return LBM_EUNSUPPORTED;
    return LBM_OK;
}

int lbm_adjoint_bytes(const lbm_handle *h, size_t *adj_state_bytes, size_t *scratch_bytes) {
    const int r = adjoint_supported(h);
    if (r != LBM_OK) return r;
    // the state's 29 planes and lambda_phi
    if (adj_state_bytes) *adj_state_bytes = (size_t)(h->Qtot + 3) * h->N * sizeof(float);
    if (scratch_bytes) *scratch_bytes = (size_t)4 * h->N * sizeof(float);   // four stencil planes
    return LBM_OK;
}

int lbm_adjoint_terminal(lbm_handle *h, const void *state, const float *phi_target, void *adj,
                         double *d_J) {
    const int r = adjoint_supported(h);
    if (r != LBM_OK) return r;
    if (!state || !phi_target || !adj || !d_J) return LBM_EINVAL;
    return cuda_status(launch_adj_terminal2d((const float *)state, phi_target, (float *)adj, d_J,
                                             h->dp, h->stream));
}

int lbm_adjoint_step(lbm_handle *h, const void *state, const void *adj_next, void *adj,
                     void *scratch, double *d_dparams) {
    const int r = adjoint_supported(h);
    if (r != LBM_OK) return r;
    if (!state || !adj_next || !adj || !scratch || !d_dparams || adj == adj_next) return LBM_EINVAL;
    return cuda_status(launch_adj_step2d((const float *)state, (const float *)adj_next, (float *)adj,
                                         (float *)scratch, d_dparams, h->dp, h->stream));
}

int lbm_set_velocity(lbm_handle *h, const lbm_fields *u, double period) {
    if (!h || !u || !u->ux || !u->uy || (h->dim == 3 && !u->uz)) return LBM_EINVAL;
    if (h->params.model != LBM_MODEL_PHASE_FIELD) return LBM_EUNSUPPORTED;
    if (!std::isfinite(period) || period < 0.0) return LBM_EINVAL;
    const void *src[3] = {u->ux, u->uy, u->uz};
    for (int a = 0; a < h->dim; ++a) {
        const float *dev;
        const int r = stage_in(h, src[a], u->on_device, u->dtype, a, &dev);
        if (r != LBM_OK) return r;
        if (cudaMemcpyAsync(h->vel + (size_t)a * h->N, dev, h->N * sizeof(float),
                            cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return LBM_ECUDA;
    }
    h->vel_period = period;
    h->vel_set = 1;
    return LBM_OK;
}

int lbm_adjoint_steps(lbm_handle *h, const void *states, size_t stride, int32_t count,
                      void *adj_next, void *adj, void *scratch, double *d_dparams) {
    const int r = adjoint_supported(h);
    if (r != LBM_OK) return r;
    if (count < 0 || !states || !adj_next || !adj || !scratch || !d_dparams || adj == adj_next)
        return LBM_EINVAL;
    size_t need;
    lbm_state_bytes(h, &need);
    if (stride < need || stride % 4 != 0) return LBM_ENOMEM;
    const char *base = (const char *)states;
    void *a = adj_next, *b = adj;
    for (int32_t j = count - 1; j >= 0; --j) {
        const cudaError_t e = launch_adj_step2d((const float *)(base + (size_t)j * stride),
                                                (const float *)a, (float *)b, (float *)scratch,
                                                d_dparams, h->dp, h->stream);
        if (e != cudaSuccess) return LBM_ECUDA;
        void *t = a; a = b; b = t;
    }
    return LBM_OK;
}

int lbm_adjoint_init(lbm_handle *h, const lbm_fields *init, const void *adj0, float *dT0,
                     double *d_dparams) {
    const int r = adjoint_supported(h);
    if (r != LBM_OK) return r;
    if (!init || !init->phi || !init->T || !adj0 || !dT0 || !d_dparams) return LBM_EINVAL;
    if (!init->on_device || init->dtype != 0) return LBM_EINVAL;
    return cuda_status(launch_adj_init2d((const float *)init->phi, (const float *)init->T,
                                         (const float *)init->ux, (const float *)init->uy,
                                         (const float *)adj0, dT0, d_dparams, h->dp, h->stream));
}

int lbm_set_first_wait_limit(int32_t polls) {
    if (set_first_wait_limit2d(polls) != cudaSuccess) return LBM_ECUDA;
    if (set_first_wait_limit3d(polls) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}

int lbm_columns_bytes(const lbm_handle *h, int32_t ncols, size_t *bytes) {
    if (!h || !bytes || ncols < 1 || ncols > h->grid.nx) return LBM_EINVAL;
    const long long cells = (long long)ncols * h->grid.ny * h->grid.nz;
    *bytes = columns_pop_bytes(cells, h->Qtot, h->elem) + 2 * (size_t)cells * sizeof(float);
    return LBM_OK;
}

static int columns(lbm_handle *h, int32_t x0, int32_t ncols, void *buf, bool pack) {
    if (!h || !buf || ncols < 1 || x0 < 0 || x0 > h->grid.nx - ncols) return LBM_EINVAL;
    if (h->params.model != LBM_MODEL_COUPLED) return LBM_EUNSUPPORTED;
    if ((uintptr_t)buf % 16 != 0) return LBM_EINVAL;
    const long long rows = (long long)h->grid.ny * h->grid.nz;
    cudaError_t e;
    switch (h->params.storage) {
    case LBM_STORE_FP32: e = launch_columns<float>(h->pops[h->cur], h->phi_prev, h->q[h->cur], buf, x0, ncols, h->grid.nx, rows, (long long)h->N, h->Qf, h->Qtot, pack, h->stream); break;
    case LBM_STORE_FP16: e = launch_columns<__half>(h->pops[h->cur], h->phi_prev, h->q[h->cur], buf, x0, ncols, h->grid.nx, rows, (long long)h->N, h->Qf, h->Qtot, pack, h->stream); break;
    default: e = launch_columns<__nv_bfloat16>(h->pops[h->cur], h->phi_prev, h->q[h->cur], buf, x0, ncols, h->grid.nx, rows, (long long)h->N, h->Qf, h->Qtot, pack, h->stream); break;
    }
    return cuda_status(e);
}

int lbm_pack_columns(lbm_handle *h, int32_t x0, int32_t ncols, void *dst) {
    return columns(h, x0, ncols, dst, true);
}

int lbm_unpack_columns(lbm_handle *h, int32_t x0, int32_t ncols, const void *src) {
    return columns(h, x0, ncols, const_cast<void *>(src), false);
}

void lbm_destroy(lbm_handle *h) { delete h; }

}  // extern "C"
