/*
 * lbm_pf.h -- C ABI of the B300 lattice Boltzmann phase-field solver for
 * two-phase flow with phase change (Verdier, Kestener & Cartalade,
 * arXiv:2003.06342).
 *
 * One handle owns one lattice: the three coupled distribution sets of the
 * paper (Sec. 3) -- f for incompressible Navier-Stokes (Sec. 3.1), g for the
 * conservative Allen-Cahn phase field with the interfacial production source
 * (Sec. 3.2), s for the temperature with the latent-heat source (Sec. 3.3) --
 * advanced by one fused CUDA kernel per time step that also evaluates the
 * finite-difference gradient, Laplacian and chemical-potential stencils
 * (Sec. 3.4).
 *
 * Conventions for every call:
 *  - Lattice units, dx = dt = 1.  Fields are dense arrays of nx*ny*nz values,
 *    x fastest, then y, then z: index (z*ny + y)*nx + x.  2D runs use nz = 1.
 *  - All calls return LBM_OK (0) or a negative LBM_E* code; none aborts,
 *    throws or exits.  lbm_strerror() names the code.
 *  - Device work is queued on the handle's CUDA stream and is asynchronous
 *    unless a call says it synchronises.  Errors raised by a kernel surface at
 *    the next synchronising call (lbm_sync, lbm_reduce, host-side
 *    lbm_get_fields / lbm_get_state) as LBM_ECUDA.
 *  - The caller owns all memory: the workspace passed to lbm_create (device
 *    memory, kept by the handle until lbm_destroy) and every field, state and
 *    map buffer.  The library itself never calls cudaMalloc.
 *  - A handle is not thread-safe; different handles are independent.
 */
#ifndef LBM_PF_H
#define LBM_PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBM_OK            0
#define LBM_EINVAL       -1   /* bad argument: size, pointer, parameter range   */
#define LBM_ENOMEM       -2   /* workspace or caller buffer too small            */
#define LBM_ECUDA        -3   /* a CUDA runtime call or kernel launch failed     */
#define LBM_ENONFINITE   -4   /* NaN or Inf in the fields (reduction, state check) */
#define LBM_ETIMEOUT     -5   /* a bounded in-kernel wait expired (see lbm_sync) */
#define LBM_EUNSUPPORTED -6   /* combination not built (e.g. lattice/storage)    */
#define LBM_EBOUNDS      -7   /* an index check failed (bounds-checking build)  */

/* ---- lattices (Sec. 3, lattice definitions) ----------------------------- */
#define LBM_D2Q9        0     /* 2D: D2Q9 for f, g and s                         */
#define LBM_D3Q19_D3Q7  1     /* 3D: D3Q19 for f and s, D3Q7 for g               */

/* ---- population storage -------------------------------------------------- */
#define LBM_STORE_FP32  0     /* 32-bit deviations  d_i = theta_i - w_i*ref      */
#define LBM_STORE_FP16  1     /* 16-bit deviations  d_i = (theta_i/w_i - ref)*scale */
#define LBM_STORE_BF16  2     /* bfloat16, same encoding as FP16                 */

typedef struct lbm_handle lbm_handle;

/* Grid.  nz = 1 selects 2D.  periodic[a] != 0 makes axis a periodic; at most
 * one axis may be non-periodic: it carries two half-way walls, at -1/2 and at
 * n_a - 1/2, with no-slip bounce-back for f and anti-bounce-back Dirichlet
 * values for g and s (Sec. 3.3, Sec. 4.1). */
typedef struct {
    int32_t nx, ny, nz;
    int32_t periodic[3];
} lbm_grid;

/* Model parameters, lattice units (Table tab:FilmBoiling_Parameters after
 * conversion).  Index 0/1 of phi_wall and T_wall is the low/high wall of the
 * non-periodic axis. */
typedef struct {
    double rho_l, rho_g;          /* phase densities, Eq. Density                */
    double nu_l, nu_g;            /* kinematic viscosities, Eq. Viscosity        */
    double alpha_l, alpha_g;      /* thermal diffusivities                       */
    double sigma, W;              /* surface tension, interface width, Eq. Def_K-H */
    double M_phi;                 /* mobility, tau_g = M_phi / cs^2              */
    double A;                     /* coefficient of Eq. ProductionRate (10/48)   */
    double theta_I;               /* dimensionless interface temperature         */
    double L, Cp, T_sat;          /* latent heat, specific heat, saturation T    */
    double gravity[3];            /* gravity vector; F_v = (rho - rho_l) gravity */
    double body_force[3];         /* constant force density added to F_tot       */
    double phi_wall[2];           /* Dirichlet phi at the low / high wall        */
    double T_wall[2];             /* Dirichlet T at the low / high wall          */
    double normal_eps;            /* n = grad phi / max(|grad phi|, normal_eps)  */
    double store_ref[3];          /* storage reference per set (f, g, s)         */
    double store_scale[3];        /* 16-bit storage scale per set (f, g, s)      */
    int32_t source_on;            /* 0: mdot''' = 0                              */
    int32_t visc_interp;          /* 0: harmonic Eq. Viscosity, 1: linear Eq. Visco_lin */
    int32_t alpha_interp;         /* 0: linear in phi, 1: harmonic               */
    int32_t storage;              /* LBM_STORE_*                                 */
    int32_t model;                /* LBM_MODEL_*                                 */
    int32_t collision;            /* LBM_COLLISION_*                             */
    int32_t grad_scheme;          /* LBM_GRAD_*                                  */
    double trt_magic[3];          /* TRT magic parameter of the f, g, s sets     */
    double mrt_rates[3];          /* MRT rates s_e, s_eps, s_q of the f set      */
    double mrt_rates_g[4];        /* MRT rates s_e, s_eps, s_q, s_p of the g set */
} lbm_params;

/* Collision operators.  BGK: Eq. LBE (the paper's scheme, the default).
 * TRT: two relaxation rates per set, w+ for the symmetric and w- for the
 * antisymmetric part of (population - barred equilibrium) and of the source
 * (not in the paper; the two-relaxation-time extension its outlook names).
 * The part that carries the set's transport coefficient keeps the BGK rate
 * 1/(tau + 1/2) (the symmetric part for f: viscosity; the antisymmetric part
 * for g and s: mobility and diffusivity); the other rate follows from the
 * magic parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2) > 0 of that set
 * (Lambda = 3/16 puts the half-way bounce-back wall exactly at the middle of
 * the link for Poiseuille flow).  TRT is implemented for LBM_MODEL_COUPLED
 * in 2D and 3D; the adjoint covers BGK only. */
#define LBM_COLLISION_BGK 0
#define LBM_COLLISION_TRT 1
/* MRT: multiple relaxation times for the flow set f and the phase-field set
 * g (not in the paper; the multiple-relaxation-time extension its outlook
 * names); s keeps BGK.  d = theta - theta_eq_bar is taken to an orthogonal
 * moment basis.  D2Q9: rho, e = 3|c|^2 - 4, eps = 4 - 21|c|^2/2 + 9|c|^4/2,
 * j_x, q_x = (3|c|^2 - 5) c_x, j_y, q_y, p_xx = c_x^2 - c_y^2, p_xy = c_x c_y.
 * D3Q19 (f): the d'Humieres basis rho, e = 19|c|^2 - 30, eps = (21|c|^4 -
 * 53|c|^2 + 24)/2, j, q = (5|c|^2 - 9) c, p_xx = 3c_x^2 - |c|^2, pi_xx =
 * (3|c|^2 - 5) p_xx, p_ww = c_y^2 - c_z^2, pi_ww = (3|c|^2 - 5) p_ww, p_xy,
 * p_yz, p_xz, m_x = (c_y^2 - c_z^2) c_x and its cyclic m_y, m_z.  D3Q7 (g):
 * rho, j, e = 7|c|^2 - 6, p_xx = 3c_x^2 - |c|^2, p_ww = c_y^2 - c_z^2.
 *   f: rho and the stress moments (p_*) relax at the BGK rate 1/(tau_f +
 *      1/2) (the viscosity); e at mrt_rates[0]; eps (in 3D also pi_xx,
 *      pi_ww) at mrt_rates[1]; j and q (in 3D also m) at mrt_rates[2]; each
 *      rate in (0, 2), else LBM_EINVAL.  Equal rates give BGK; s_e = s_eps =
 *      1/(tau_f + 1/2) gives the TRT collision of f with antisymmetric rate
 *      s_q; s_q = 8 (2 - s_nu)/(8 - s_nu) puts the half-way bounce-back wall
 *      at the middle of the link for Poiseuille flow.
 *   g: phi and j relax at the BGK rate 1/(tau_g + 1/2) (the mobility); e,
 *      eps, q and the stress moments at mrt_rates_g[0..3] (D3Q7 has no eps
 *      and no q: mrt_rates_g[1] and [2] are checked but unused there); each
 *      rate 0 (meaning the BGK rate, so all zeros keep g on BGK) or in (0, 2),
 *      else LBM_EINVAL.
 * MRT is implemented for LBM_MODEL_COUPLED in 2D and 3D (tiled and TMA
 * kernels); the phase-field model returns LBM_EUNSUPPORTED; the adjoint
 * covers BGK only. */
#define LBM_COLLISION_MRT 2

/* Directional derivative inside Eq. Grad (Sec. 3.4).  CENTRAL: Eq.
 * DerivDirec_Grad (the paper's choice).  BIASED2: the second-order biased
 * difference e_i.grad(phi) = [-phi(x + 2 e_i) + 4 phi(x + e_i) - 3 phi(x)]/2
 * the paper names as the remedy for velocity profiles in low-density
 * regions (the first-order one gives exactly the central gradient through
 * Eq. Grad); two ghost layers, the wall's Dirichlet value beyond a wall.
 * The Laplacian stays central.  BIASED2 is implemented for the coupled model
 * on the tiled kernels (2D and 3D) and on the 3D TMA kernel for grids without
 * ragged tiles (n_x a multiple of 32, n_y of 4; there AUTO selects it for
 * 16-bit storage and the tiled kernel for FP32, the faster of each pair) and
 * in the adjoint; the 2D TMA kernel takes CENTRAL only (LBM_EUNSUPPORTED). */
#define LBM_GRAD_CENTRAL 0
#define LBM_GRAD_BIASED2 1

/* Models.  COUPLED: the three coupled schemes of Sec. 3 (the default).
 * PHASE_FIELD: the phase-field scheme alone (Sec. 3.2, no phase change) in a
 * velocity field imposed with lbm_set_velocity -- the setting of the CAC
 * validations of Sec. 4.1; the flow and temperature populations are not
 * stepped, lbm_get_fields returns phi (u, p and T are not meaningful) and
 * source_on must be 0.  2D (D2Q9) and 3D (the D3Q7 phase-field lattice of
 * the coupled model, on the tiled kernel). */
#define LBM_MODEL_COUPLED      0
#define LBM_MODEL_PHASE_FIELD  1

/* Macroscopic fields.  Any pointer may be NULL (that field is skipped on
 * output; on input NULL means zero, except phi and T, which are required).
 * uz is ignored in 2D.  on_device: 1 for device pointers, 0 for host
 * pointers (host transfers are synchronous).  dtype: 0 float32, 1 float64. */
typedef struct {
    void *phi, *T, *ux, *uy, *uz, *p;
    int32_t on_device;
    int32_t dtype;
} lbm_fields;

/* Device workspace needed by lbm_create for this grid, lattice and storage:
 * two population buffers (read/write per step), phi^{n-1}, two lagged-source
 * buffers, moment and reduction scratch, and for LBM_MODEL_PHASE_FIELD the
 * imposed velocity.  Returns LBM_EINVAL on an invalid grid or parameter set,
 * LBM_EUNSUPPORTED for a model not built for the lattice. */
int lbm_workspace_bytes(const lbm_grid *grid, int32_t lattice, const lbm_params *params,
                        size_t *bytes);

/* Validate grid and parameters (tau_f, tau_g, tau_s > 0, W > 0, densities > 0,
 * at most one wall axis) and build a handle over the caller's device
 * workspace (256-byte aligned, at least lbm_workspace_bytes).  stream is a
 * cudaStream_t (NULL: the legacy default stream).  The state is undefined
 * until lbm_init or lbm_set_state.  Errors: LBM_EINVAL, LBM_ENOMEM,
 * LBM_EUNSUPPORTED, LBM_ECUDA. */
int lbm_create(const lbm_grid *grid, int32_t lattice, const lbm_params *params,
               void *workspace, size_t workspace_bytes, void *stream, lbm_handle **out);

/* Queue later work on another cudaStream_t. */
int lbm_set_stream(lbm_handle *h, void *stream);

/* Set the populations to the barred equilibria of the given fields,
 * theta_bar_i = theta_eq_i - S_i/2 (App. C, Eq. VariableChange_feq), with
 * phi^{n-1} = phi_0 and the lagged source evaluated from (phi_0, T_0), so that
 * lbm_get_fields returns the input fields.  Resets the step counter. */
int lbm_init(lbm_handle *h, const lbm_fields *in);

/* Advance n >= 0 time steps: per step one fused kernel computing the moments
 * (Eqs. Moment_Phi, Velocity, Pressure, Moment_Temp), the phi stencils (Eqs.
 * Grad, Laplacian, ChemicalPotential), the production rate (Eq.
 * ProductionRate), the three collisions with sources (Eq. LBE, or the TRT
 * option of lbm_params.collision) and the streaming with boundary links.
 * Asynchronous. */
int lbm_step(lbm_handle *h, int32_t n);

/* Write phi, u, p and T of the current state (the moments of the step
 * above).  Device outputs are asynchronous; host outputs synchronise. */
int lbm_get_fields(lbm_handle *h, lbm_fields *out);

/* Global phase-field mass sum(phi) and enthalpy sum(rho (Cp T + phi L))
 * (Eq. Conservation_Enthalpie with H = Cp T + phi L), accumulated in FP64.
 * Synchronises; returns LBM_ENONFINITE if either sum is not finite. */
int lbm_reduce(lbm_handle *h, double *phi_mass, double *energy);

/* Same reduction, asynchronous: two doubles written to device memory d_out. */
int lbm_reduce_async(lbm_handle *h, double *d_out);

/* Checkpoint / resume: the state is the populations in their storage format
 * -- the Qf (f_i, s_i) pair planes (2N values each, f_i of cell x at
 * 2(iN + x), s_i at 2(iN + x) + 1), then the Qg g planes -- followed by
 * phi^{n-1} and the lagged source as float32 (bytes from lbm_state_bytes).
 * on_device selects the buffer's side.
 * Restoring a saved state and stepping reproduces the uninterrupted run bit
 * for bit. */
int lbm_state_bytes(const lbm_handle *h, size_t *bytes);
int lbm_get_state(lbm_handle *h, void *dst, size_t bytes, int32_t on_device);
int lbm_set_state(lbm_handle *h, const void *src, size_t bytes, int32_t on_device);

/* Test hook: the streaming map of one step as executed by the step kernel,
 * in pull form.  set 0 = the f/s lattice, 1 = the g lattice.  For direction i
 * and destination cell x, src_index[i*N + x] = cell the value comes from and
 * kind[i*N + x] = 0 interior, 1 wrapped over a periodic axis, 2 bounced at the
 * low wall, 3 bounced at the high wall (a bounced value comes from x itself,
 * opposite direction).  Both buffers are device memory of Q*N entries. */
int lbm_stream_map(lbm_handle *h, int32_t set, int32_t *src_index, int8_t *kind);

/* Kernel variants of the step.  TILED reads populations with plain loads.
 * TMA stages them in shared memory with bulk tensor copies, available when the
 * grid allows 16-byte-aligned tensor boxes (n_x a multiple of 4 for FP32 or 8
 * for 16-bit storage, at least 32 x 8 cells per plane): in 2D a kernel that
 * marches 32-column strips in chunks of 8 rows, in 3D the z-marching kernel,
 * each staging the next chunk or layer while the current one is computed.
 * AUTO (default) is the faster of the two on B300: TILED in 2D, TMA in 3D when
 * available (else TILED).  Tiled and TMA variants compute the same update bit
 * for bit. */
#define LBM_KERNEL_AUTO   0
#define LBM_KERNEL_TILED  1
#define LBM_KERNEL_TMA    2

/* Select the step kernel; LBM_EUNSUPPORTED if TMA staging is not possible
 * for this grid, storage or device. */
int lbm_set_kernel(lbm_handle *h, int32_t kernel);

/* The kernel lbm_step launches (LBM_KERNEL_TILED or LBM_KERNEL_TMA; AUTO is
 * reported as what it resolves to). */
int lbm_get_kernel(const lbm_handle *h, int32_t *kernel);

/* n time steps, saving the state after each: after step k (k = 0..n-1) the
 * state (lbm_get_state layout) is in buf + k*stride, device memory, and the
 * handle holds the last one.  Used to recompute a checkpointed segment for
 * the adjoint in one call.  stride >= lbm_state_bytes; LBM_ENOMEM for a
 * short stride.  For the 2D coupled model on the tiled kernel without the
 * periodic state check, with buf and stride multiples of 16 bytes, each
 * step reads the previous slot and writes the next one directly (one state
 * copy per call instead of one per step); the states are the same. */
int lbm_step_record(lbm_handle *h, int32_t n, void *buf, size_t stride);

/* Number of time steps since lbm_init / lbm_set_state. */
int lbm_steps_done(const lbm_handle *h, int64_t *steps);

/* Kernel launches queued by the last lbm_step call. */
int lbm_last_launches(const lbm_handle *h, int32_t *launches);

/* Periodic state check: when every > 0, every `every`-th step of lbm_step /
 * lbm_step_record is followed by one extra launch that reads the state, forms
 * phi = sum_i gbar_i + q/2 (Eq. Moment_Phi) of every cell and flags the state
 * when phi leaves [1/2 - phi_excess, 1/2 + phi_excess] or a stored
 * population, phi or the lagged source is not finite; lbm_sync then returns
 * LBM_ENONFINITE.  The launch reads every population once (about half the
 * traffic of a step).  every = 0 (the default) turns the check off.  Errors: LBM_EINVAL for every < 0 or,
 * with every > 0, phi_excess not a positive finite number. */
int lbm_set_health_check(lbm_handle *h, int32_t every, float phi_excess);

/* Wait for the handle's stream; report any pending CUDA error, or
 * LBM_ETIMEOUT if a bounded wait inside a step kernel expired (the kernel then
 * stopped early and the state is not valid), or -- in the bounds-checking
 * build of the library (liblbmpf_debug.so, every computed population and
 * field index checked against its buffer, a failing access skipped) --
 * LBM_EBOUNDS if a check failed since lbm_init / lbm_set_state, or
 * LBM_ENONFINITE if the periodic state check (lbm_set_health_check) flagged
 * the state.  The status is cleared when reported. */
int lbm_sync(lbm_handle *h);

/* ---- discrete adjoint (2D, FP32 storage) ----------------------------------
 * Reverse-mode derivative of the step for gradients of a final-time loss
 * with respect to the latent heat L, the mobility M_phi, the surface tension
 * sigma and the initial temperature field (the step is Eq. LBE with the
 * sources of Sec. 3; the loss is J = 1/2 sum (phi^N - phi_target)^2).
 * States are device buffers in the lbm_get_state layout (float32: the nine
 * (f_i, s_i) pair planes, 2N values each with f_i at 2(iN + x) and s_i at
 * 2(iN + x) + 1, the nine g planes, phi^{n-1}, lagged source).  An adjoint
 * state has the same 29 planes followed by a 30th, lambda_phi = dJ/dphi^n:
 * the derivative of J with respect to a stored g_i(x) is plane 9 + i plus
 * lambda_phi(x), with respect to the lagged source(x) plane 28 plus
 * lambda_phi(x)/2, with respect to every other stored value its own plane
 * (phi^n = sum_i g_i + q^{n-1}/2 is kept as one term instead of being spread
 * over ten planes).  Other lattices and storages return LBM_EUNSUPPORTED. */

/* Bytes of one adjoint state (30 planes of N floats) and of the per-step
 * scratch (4 planes). */
int lbm_adjoint_bytes(const lbm_handle *h, size_t *adj_state_bytes, size_t *scratch_bytes);

/* Seed: adj = dJ/dX^N for the state X^N; adds J to *d_J (device double). */
int lbm_adjoint_terminal(lbm_handle *h, const void *state, const float *phi_target, void *adj,
                         double *d_J);

/* One step backwards: adj = (dX^{n+1}/dX^n)^T adj_next, with X^n = state;
 * adds dJ/dL, dJ/dM_phi, dJ/dsigma of this step to d_dparams[0..2] (device
 * doubles).  adj and adj_next must differ; scratch from lbm_adjoint_bytes. */
int lbm_adjoint_step(lbm_handle *h, const void *state, const void *adj_next, void *adj,
                     void *scratch, double *d_dparams);

/* A segment of the reverse sweep in one call: for j = count-1 down to 0,
 * one lbm_adjoint_step with state = states + j*stride (device), the two
 * adjoint buffers swapping roles after every step.  On return the adjoint of
 * the segment's first state is in adj_next when count is even and in adj
 * when count is odd.  stride >= lbm_state_bytes (a multiple of 4);
 * LBM_EINVAL for count < 0 or a bad pointer, LBM_ENOMEM for a short stride. */
int lbm_adjoint_steps(lbm_handle *h, const void *states, size_t stride, int32_t count,
                      void *adj_next, void *adj, void *scratch, double *d_dparams);

/* Through the initialisation (lbm_init): dT0 = dJ/dT_0 (device float32,
 * nx*ny) from adj0 = dJ/dX^0, and the initialisation's share of dJ/dL and
 * dJ/dsigma added to d_dparams[0] and [2].  init holds the same device
 * float32 phi, T (and optional ux, uy) given to lbm_init. */
int lbm_adjoint_init(lbm_handle *h, const lbm_fields *init, const void *adj0, float *dT0,
                     double *d_dparams);

/* LBM_MODEL_PHASE_FIELD: the imposed velocity u(x) (ux, uy and in 3D uz of
 * `u`, same layout and pointer rules as lbm_init) and its time factor: the velocity at
 * step n is u(x) cos(pi n / period) when period > 0 (the reversing vortex of
 * Sec. 4.1 uses period = 2 T_f), u(x) otherwise, with n counted from
 * lbm_init or lbm_set_state (the saved state holds no step count, so a
 * resumed time-dependent run restarts its factor at n = 0).  Call before
 * lbm_init, which then builds the populations with that velocity.
 * LBM_EUNSUPPORTED for the coupled model. */
int lbm_set_velocity(lbm_handle *h, const lbm_fields *u, double period);

/* Allocation-free global sums (no counterpart in the paper).  For callers
 * that must not allocate device memory at all -- for example code running
 * inside a host application whose memory pool owns every device buffer, or a
 * monitoring hook on a latency-critical path where the implicit
 * synchronisation of cudaMalloc/cudaFree is not acceptable -- and who
 * therefore cannot provide the workspace lbm_reduce needs.
 * Computes out[0] = sum(phi) and out[1] = sum(rho(phi) (Cp T + phi L)), with
 * rho(phi) = phi rho_g + (1 - phi) rho_l on phi clipped to [0, 1], in FP64,
 * over n_cells float32 values of phi and T (device pointers); d_out is device
 * memory for two doubles.  Queued on `stream` (a cudaStream_t, NULL = legacy
 * default stream).  The per-block partial sums use a 1 MiB array in static
 * device memory that every GPU loading the library holds until exit; hence
 * n_cells is limited to 16,777,216 and larger sizes return LBM_ENOMEM.  Every
 * call looks up that array's device address on the current device (no
 * allocation), so the entry point stays valid after a device reset
 * (cudaDeviceReset, or a primary context released and created again); the
 * first call on a device may load the library's device code, so make it
 * before any stream capture.  All calls share the array: calls whose kernels
 * overlap on the GPU race and must be ordered by the caller.  Errors:
 * LBM_EINVAL (NULL pointer, n_cells < 1, non-positive density), LBM_ENOMEM,
 * LBM_ECUDA. */
int lbm_field_sums_noalloc(const float *phi, const float *T, int64_t n_cells, double rho_l,
                           double rho_g, double Cp, double L, double *d_out, void *stream);

/* Test hook of the bounded waits (no counterpart in the paper).  Every
 * mbarrier wait of the TMA-staged step kernels polls at most 4,194,304 times
 * before the block gives up, waits for the bulk copies it has issued,
 * records the timeout in the handle's status word and returns; lbm_sync then
 * reports LBM_ETIMEOUT.  This call sets the poll limit of the first wait of
 * every block (the later waits keep the default) on the current device and
 * for the whole process: 0 makes every block give up at once, which is how
 * the timeout path is tested without a stalled copy; a negative value
 * restores the default.  Error: LBM_ECUDA. */
int lbm_set_first_wait_limit(int32_t polls);

/* Column blocks of the state, for a slab domain decomposition along x (the
 * paper's implementation section: one sub-domain per GPU, neighbouring
 * sub-domains trade ghost layers every time step).  A block is the complete
 * stored state of columns [x0, x0 + ncols) over every y (and z): the Qtot
 * population planes in the handle's storage precision (each plane rows x
 * ncols values, rows = ny nz, x fastest; f, s of a direction as two planes,
 * then the g planes), zero-padded to a multiple of 16 bytes, followed by phi^{n-1}
 * and the lagged source as two planes of rows x ncols floats.
 * lbm_columns_bytes gives the size of a block of ncols columns.
 * lbm_pack_columns copies the block into dst, lbm_unpack_columns overwrites
 * the handle's state with src; both are device buffers owned by the caller,
 * 16-byte aligned, and both calls are queued on the handle's stream (the
 * caller orders them against other streams).  A decomposition built on these
 * calls gives each sub-domain h ghost columns on both sides (h = 2 for the
 * central gradient, 3 for the biased one) and, after every step, unpacks the
 * neighbours' h outermost owned columns into them; the owned columns then
 * evolve exactly as in the undivided grid.  Errors: LBM_EINVAL (NULL, a
 * misaligned buffer, columns outside [0, nx)), LBM_EUNSUPPORTED
 * (LBM_MODEL_PHASE_FIELD), LBM_ECUDA. */
int lbm_columns_bytes(const lbm_handle *h, int32_t ncols, size_t *bytes);
int lbm_pack_columns(lbm_handle *h, int32_t x0, int32_t ncols, void *dst);
int lbm_unpack_columns(lbm_handle *h, int32_t x0, int32_t ncols, const void *src);

/* Release the handle (not the workspace, which the caller owns). */
void lbm_destroy(lbm_handle *h);

const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LBM_PF_H */
