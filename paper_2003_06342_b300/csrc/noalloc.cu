// Allocation-free global sums over caller-provided fields.
//
// The per-block partial sums, which the handle-based reduction keeps in the
// caller's workspace, live here in a file-scope device array instead, so
// this entry point needs no workspace and allocates nothing.  Host code only
// sees a host-side stand-in for that array under its name; the device
// address is looked up with cudaGetSymbolAddress (with the caller's device
// current) on every call, so it stays right after a device reset or a
// recreated primary context reloads the module.
#include <cmath>

#include "../../include/lbm_pf.h"
#include "lbm_kernels.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 65536;                       // 16,777,216 cells
constexpr long long NA_MAX_CELLS = (long long)NA_MAX_BLOCKS * NA_THREADS;

// two doubles per block: 1 MiB, held by every GPU that loads the library
static __device__ __align__(256) double na_scratch[2 * NA_MAX_BLOCKS];

// Same per-cell terms as the moment kernels' reduction: phi and rho(phi)
// (Cp T + phi L), rho on phi clipped to [0, 1]; one cell per thread (the
// moment kernels add several cells per thread), so the FP64 sums agree with
// lbm_reduce to rounding.
__global__ void __launch_bounds__(NA_THREADS)
field_sums_kernel(const float *__restrict__ phi, const float *__restrict__ T, long long n,
                  float rho_l, float rho_g, double Cp, double Lh, double *partial) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double mass = 0.0, energy = 0.0;
    if (c < n) {
        const float ph = phi[c];
        const float pc = fminf(fmaxf(ph, 0.0f), 1.0f);
        const float rho = pc * rho_g + (1.0f - pc) * rho_l;
        mass = (double)ph;
        energy = (double)rho * (Cp * (double)T[c] + (double)ph * Lh);
    }
    lbm::block_sum2(mass, energy, partial);
}

int device_scratch(double **out) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, na_scratch) != cudaSuccess || !p) return LBM_ECUDA;
    *out = p;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_field_sums_noalloc(const float *phi, const float *T, int64_t n_cells,
                                      double rho_l, double rho_g, double Cp, double L,
                                      double *d_out, void *stream) {
    if (!phi || !T || !d_out || n_cells < 1) return LBM_EINVAL;
    if (n_cells > NA_MAX_CELLS) return LBM_ENOMEM;
    if (!(rho_l > 0 && rho_g > 0) || !std::isfinite(Cp) || !std::isfinite(L)) return LBM_EINVAL;
    double *partial = nullptr;
    const int r = device_scratch(&partial);
    if (r != LBM_OK) return r;
    const int nblocks = (int)((n_cells + NA_THREADS - 1) / NA_THREADS);
    cudaStream_t st = (cudaStream_t)stream;
    // every block writes its own pair, so no clearing is needed before use
    field_sums_kernel<<<nblocks, NA_THREADS, 0, st>>>(phi, T, (long long)n_cells, (float)rho_l,
                                                       (float)rho_g, Cp, L, partial);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (lbm::launch_final_sum2(partial, nblocks, d_out, st) != cudaSuccess) return LBM_ECUDA;
    return LBM_OK;
}
