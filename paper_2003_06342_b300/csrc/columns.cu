// Column blocks of the stored state, the exchange unit of the slab domain
// decomposition (the paper's implementation section splits the domain into
// sub-domains along one axis, one per GPU, and trades ghost layers between
// neighbours every time step).
//
// A block is the whole state of columns [x0, x0 + ncols) over every y (and z):
// the population planes in storage precision, then phi^{n-1} and the lagged
// source in float.  Packing and unpacking are plain strided copies on the
// handle's stream; the buffer may be any device memory the caller owns (a
// local staging buffer, or the send / receive buffer of a collective).
#include "../../include/lbm_pf.h"
#include "lbm_kernels.h"

namespace lbm {

namespace {

// element of virtual plane v at cell c: the first 2 Qf planes are the f and s
// halves of the (f_i, s_i) pair planes, the rest the g planes
__device__ __forceinline__ size_t plane_elem(int v, size_t c, size_t N, int Qf) {
    return v < 2 * Qf ? 2 * ((size_t)(v >> 1) * N + c) + (size_t)(v & 1) : (size_t)v * N + c;
}

template <typename S, bool PACK>
__global__ void __launch_bounds__(256)
columns_kernel(S *__restrict__ pops, float *__restrict__ phi_prev, float *__restrict__ q,
               S *__restrict__ bpops, float *__restrict__ bscal, int x0, int ncols, int nx,
               long long rows, long long N, int Qf, int Qtot) {
    const long long M = rows * ncols;                  // cells in the block
    const long long total = M * (Qtot + 2);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / M, k = t - v * M;      // plane, cell of the block
        const long long r = k / ncols;
        const size_t c = (size_t)(r * nx + x0 + (k - r * ncols));
        if (v < Qtot) {
            const size_t e = plane_elem((int)v, c, (size_t)N, Qf);
            if (PACK) bpops[t] = pops[e];
            else pops[e] = bpops[t];
        } else {
            float *field = v == Qtot ? phi_prev : q;
            const long long b = (v - Qtot) * M + k;
            if (PACK) bscal[b] = field[c];
            else field[c] = bscal[b];
        }
    }
}

}  // namespace

size_t columns_pop_bytes(long long cells, int Qtot, size_t elem) {
    return ((size_t)cells * Qtot * elem + 15) / 16 * 16;
}

template <typename S>
cudaError_t launch_columns(void *pops, float *phi_prev, float *q, void *buf, int x0, int ncols,
                           int nx, long long rows, long long N, int Qf, int Qtot, bool pack,
                           cudaStream_t st) {
    const long long M = rows * ncols;
    S *bpops = (S *)buf;
    float *bscal = (float *)((char *)buf + columns_pop_bytes(M, Qtot, sizeof(S)));
    const long long total = M * (Qtot + 2);
    const long long want = (total + 255) / 256;
    const int blocks = (int)(want < 148LL * 16 ? want : 148LL * 16);
    if (pack) {
        // the padding between the population and scalar parts is zeroed, so
        // equal states pack to equal bytes
        const size_t used = (size_t)M * Qtot * sizeof(S);
        const size_t pad = columns_pop_bytes(M, Qtot, sizeof(S)) - used;
        if (pad && cudaMemsetAsync((char *)buf + used, 0, pad, st) != cudaSuccess) return cudaGetLastError();
    }
    if (pack)
        columns_kernel<S, true><<<blocks, 256, 0, st>>>((S *)pops, phi_prev, q, bpops, bscal, x0, ncols,
                                                        nx, rows, N, Qf, Qtot);
    else
        columns_kernel<S, false><<<blocks, 256, 0, st>>>((S *)pops, phi_prev, q, bpops, bscal, x0, ncols,
                                                         nx, rows, N, Qf, Qtot);
    return cudaGetLastError();
}

template cudaError_t launch_columns<float>(void *, float *, float *, void *, int, int, int, long long,
                                           long long, int, int, bool, cudaStream_t);
template cudaError_t launch_columns<__half>(void *, float *, float *, void *, int, int, int, long long,
                                            long long, int, int, bool, cudaStream_t);
template cudaError_t launch_columns<__nv_bfloat16>(void *, float *, float *, void *, int, int, int,
                                                   long long, long long, int, int, bool, cudaStream_t);

}  // namespace lbm
