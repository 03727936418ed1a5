// 3D step with every tile layer staged by bulk tensor copies.
//
// Same update as step3d_kernel (lbm3d.cu): each block marches a 32x4 column
// tile through ZBT layers.  One thread issues cp.async.bulk.tensor copies of
// the tile's layers into shared-memory stages:
//   f/s stage  (f_i, s_i) pair planes 32 x 4 x 1 x 19 from (x0, y0, L, 0)
//                                          4D map (x, y, z, pair plane)
//              phi^{n-1} 32 x 4 x 1    from (x0, y0, L)       3D map (x, y, z)
//   g stage    g planes 32 x 4 x 1 x 7  from (x0, y0, L, 0)   4D map (x, y, z, g plane)
//              q^{n-1}  32 x 4 x 1     from (x0, y0, L)
// each completing on its own mbarrier (a box row of pairs is two whole
// 128-byte lines of FP32, or one of 16-bit values).  Two f/s stages and three g stages
// rotate so that every copy is issued a whole layer before it is needed: while
// layer z is computed (it needs f/s of z and g of z and z + 1, the latter for
// the phi window), the copies of f/s(z + 1) and g(z + 2) are in flight.  The
// populations therefore never wait in registers.  The halo ring of the phi
// window is formed with plain loads, which find those cells in L2 (the
// neighbouring blocks staged them a layer earlier).  A tile that does not fit
// the grid whole takes the plain-load column of step3d_kernel.
//
// Waits on the mbarriers are bounded: on expiry the block records an error in
// a device word, waits (bounded) for its copies in flight and returns; the
// host reports LBM_ETIMEOUT at the next sync.
#include "lbm_common.cuh"
#include "lbm_kernels.h"
#include "lbm3d_cell.cuh"
#include "lbm3d_tma.h"
#include "tma_util.cuh"

namespace lbm {

template <typename S> struct Tma3Geom {
    static constexpr int ES = (int)sizeof(S);
    static constexpr int CELLS = TX * TY;
    static constexpr int al(int b) { return (b + 127) / 128 * 128; }
    static constexpr int F_BYTES = QF * CELLS * ES;
    static constexpr int G_BYTES = QG * CELLS * ES;
    static constexpr int Q_BYTES = CELLS * 4;
    // f/s stage: f, s and phi^{n-1} of one layer; g stage: g and q^{n-1}
    static constexpr int OFF_FS = 0;                       // pairs (f_i, s_i)
    static constexpr int OFF_PP = OFF_FS + al(2 * F_BYTES);
    static constexpr int FS_STAGE = OFF_PP + al(Q_BYTES);
    static constexpr int OFF_G = 0;
    static constexpr int OFF_Q = OFF_G + al(G_BYTES);
    static constexpr int G_STAGE = OFF_Q + al(Q_BYTES);
    static constexpr int NFS = 2, NG = 3;                  // stages of each kind
    static constexpr int G_BASE = NFS * FS_STAGE;
    static constexpr unsigned FS_TX = 2 * F_BYTES + Q_BYTES;
    static constexpr unsigned G_TX = G_BYTES + Q_BYTES;
    static constexpr int DYN = NFS * FS_STAGE + NG * G_STAGE + 128;   // + alignment slack
    // layers per block: 64 for the issue-bound 16-bit kernel (fewer column
    // prologues, +1.0%), 32 for FP32 (64 measured -2.4%)
    static constexpr int ZBT = IsNarrow<S>::value ? 64 : 32;
};

template <typename S>
__device__ __forceinline__ void issue_fs(unsigned char *stage, uint64_t *bar, const TmaMaps3d &M,
                                         int par, int x0, int y0, int z) {
    using Gm = Tma3Geom<S>;
    // order earlier generic-proxy reads of this stage before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::FS_TX);
    tma_load_4d(stage + Gm::OFF_FS, &M.fs[par], x0, y0, z, 0, bar);
    tma_load_3d(stage + Gm::OFF_PP, &M.pp, x0, y0, z, bar);
}

template <typename S>
__device__ __forceinline__ void issue_g(unsigned char *stage, uint64_t *bar, const TmaMaps3d &M,
                                        int par, int x0, int y0, int z) {
    using Gm = Tma3Geom<S>;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, Gm::G_TX);
    tma_load_4d(stage + Gm::OFF_G, &M.g[par], x0, y0, z, 0, bar);
    tma_load_3d(stage + Gm::OFF_Q, &M.q[par], x0, y0, z, bar);
}

// phi - phi_ref of the thread's own cell from a g stage (same arithmetic as
// phid_at, so the halo ring of a neighbouring block sees the same float)
template <typename S>
__device__ __forceinline__ float staged_phid(const unsigned char *gstage, int own, const DevParams &P) {
    using Gm = Tma3Geom<S>;
    const S *G = (const S *)(gstage + Gm::OFF_G);
    float v[QG];
#pragma unroll
    for (int i = 0; i < QG; ++i) v[i] = widen(G[i * Gm::CELLS + own]);
    return fmaf(0.5f, ((const float *)(gstage + Gm::OFF_Q))[own], set_sum7<S>(v, P.set_isc[1]));
}

// Polls allowed to the first mbarrier wait of every block (all later waits
// take WAIT_LIMIT).  The default is WAIT_LIMIT; the timeout test lowers it to
// zero through set_first_wait_limit3d, so that every block gives up at its
// first stage, waits for the copies it issued, records the timeout in the
// status word and returns (no copy is left in flight).
static __device__ int first_wait_limit = WAIT_LIMIT;

cudaError_t set_first_wait_limit3d(int polls) {
    const int v = polls < 0 ? WAIT_LIMIT : polls;
    return cudaMemcpyToSymbol(first_wait_limit, &v, sizeof(int));
}

// Stage bookkeeping: bit b of `par_*` = parity awaited next on barrier b,
// bit b of `pend_*` = copies issued on barrier b and not yet seen complete.
struct StageSet {
    uint32_t par = 0u, pend = 0u;
    __device__ __forceinline__ bool wait(uint64_t *bars, int b, int limit = WAIT_LIMIT) {
        const bool ok = mbar_wait_bounded(&bars[b], (par >> b) & 1u, limit);
        if (ok) { par ^= 1u << b; pend &= ~(1u << b); }
        return ok;
    }
    __device__ __forceinline__ void drain(uint64_t *bars, int n) {
        for (int b = 0; b < n; ++b)
            if ((pend >> b) & 1u) mbar_wait_bounded(&bars[b], (par >> b) & 1u);
    }
};

// Halo ring of the phi window, fetched a layer ahead with cp.async (4-byte
// copies straight into shared memory, no registers held): ring cell r of the
// tile (one per thread r < RING_CELLS) gets its 7 g values and q in words
// buf[k * RING_CELLS + r].  A 16-bit value is fetched as the aligned 32-bit
// word that holds it (the workspace is 256-byte aligned, so element e sits in
// the word at 2 (e / 2) and in half e % 2 of it).
constexpr int RING_CELLS = 2 * SX + 2 * TY;
constexpr int RING_WORDS = 8 * RING_CELLS;

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// grid cell (column index + plane offset) of ring cell r for plane z
template <int XY>
__device__ __forceinline__ size_t ring_cell(int r, int z, int x0, int y0, const DevParams &P, int &slot) {
    const int nx = P.n[0], ny = P.n[1];
    int sx, sy;
    if (r < SX) { sx = r; sy = 0; }
    else if (r < 2 * SX) { sx = r - SX; sy = SY - 1; }
    else if (r < 2 * SX + TY) { sx = 0; sy = 1 + r - 2 * SX; }
    else { sx = SX - 1; sy = 1 + r - 2 * SX - TY; }
    slot = sy * SX + sx;
    int cx = x0 + sx - 1, cy = y0 + sy - 1;
    if (XY == XY_WRAP) {
        cx = cx < 0 ? cx + nx : (cx >= nx ? cx - nx : cx);
        cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
    }
    return ((size_t)z * ny + cy) * nx + cx;
}

template <typename S, int XY>
__device__ __forceinline__ void ring_prefetch(uint32_t *buf, const S *__restrict__ pin,
                                              const float *__restrict__ q_in, int z, int x0, int y0,
                                              int tid, const DevParams &P) {
    if (tid >= RING_CELLS) return;
    int slot;
    const size_t cc = ring_cell<XY>(tid, z, x0, y0, P, slot);
    const size_t N = (size_t)P.N;
    if (!in_bounds((long long)cc, (long long)N, P)) return;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        const size_t e = off_g(QF, i, cc, N);
        const S *src = pin + (IsNarrow<S>::value ? (e & ~(size_t)1) : e);
        cp_async4(&buf[i * RING_CELLS + tid], src);
    }
    cp_async4(&buf[QG * RING_CELLS + tid], q_in + cc);
    cp_async_commit();
}

// phi - phi_ref of ring cell tid from its fetched words (same arithmetic as phid_at)
template <typename S, int XY>
__device__ __forceinline__ void ring_store(float *plane, const uint32_t *buf, int z, int x0, int y0,
                                           int tid, const DevParams &P) {
    if (tid >= RING_CELLS) return;
    int slot;
    const size_t cc = ring_cell<XY>(tid, z, x0, y0, P, slot);
    const size_t N = (size_t)P.N;
    float v[QG];
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        const uint32_t w = buf[i * RING_CELLS + tid];
        if (IsNarrow<S>::value) {
            const size_t e = off_g(QF, i, cc, N);
            const unsigned short h = (unsigned short)((e & 1) ? (w >> 16) : (w & 0xffffu));
            S val;
            memcpy(&val, &h, 2);
            v[i] = widen(val);
        } else {
            v[i] = __uint_as_float(w);
        }
    }
    plane[slot] = fmaf(0.5f, __uint_as_float(buf[QG * RING_CELLS + tid]), set_sum7<S>(v, P.set_isc[1]));
}

// ---- the biased gradient's window: five planes of the tile and two rings.
// A window plane is fetched whole a layer ahead with cp.async (its own cells
// too: the g stage of that layer is still in flight when the plane is needed).

// slot of the two-ring window at (cx, cy, cz): the grid cell (wrapped over
// periodic axes, up to two cells out), or -1 beyond a wall with the wall's
// value in wall_val (the cases of window_phid_b)
__device__ __forceinline__ long long bwin_cell(int cx, int cy, int cz, const DevParams &P, float &wall_val) {
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    // x and y: this kernel runs on n_x >= 32, n_y >= 4, so a slot is at most
    // one period out and one add or subtract wraps it
    const int kx = (cx >= 0 && cx < nx) ? 0 : (P.periodic[0] ? (cx += cx < 0 ? nx : -nx, 1) : (cx < 0 ? 2 : 3));
    const int ky = (cy >= 0 && cy < ny) ? 0 : (P.periodic[1] ? (cy += cy < 0 ? ny : -ny, 1) : (cy < 0 ? 2 : 3));
    const int kz = (cz >= 0 && cz < nz) ? 0 : wrap_coord_far(cz, nz, P.periodic[2]);
    wall_val = 0.0f;
    if (kx >= 2) { wall_val = P.phi_wall[kx - 2] - P.g_ref; return -1; }
    if (ky >= 2) { wall_val = P.phi_wall[ky - 2] - P.g_ref; return -1; }
    if (kz >= 2) { wall_val = P.phi_wall[kz - 2] - P.g_ref; return -1; }
    return ((long long)cz * ny + cy) * nx + cx;
}

// The window plane is fetched in quads of x-adjacent cells, columns x0 - 4
// .. x0 + 35 (ten quads a row, eight rows; the window's 36 columns are
// x0 - 2 .. x0 + 33): x0 is a multiple of 32 and the biased TMA path runs on
// n_x a multiple of 32, so the four cells of a quad are grid cells cc .. cc
// + 3 with cc a multiple of 4 (x wrapped by a whole period on a periodic
// axis), or all beyond the same wall.  N is a multiple of 4 too, so a quad's
// values of one g plane fill one aligned 16-byte (FP32) or 8-byte (16-bit)
// block and one cp.async fetches them.
constexpr int BWQ_COLS = 40, BWQ_QUADS = BWQ_COLS / 4 * SYB;        // 80 quads a plane
// words of one fetched plane: FP32 plane i in [i * BWQ_W, +BWQ_W), the
// lagged source after the 7 g planes; 16-bit: g quads take 2 words
constexpr int BWQ_W = BWQ_COLS * SYB;                                // 320
constexpr int BWIN_WORDS = (QG + 1) * BWQ_W;

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// word offset of quad q's plane-i block in a fetched plane (the 16-bit g
// planes pack a quad into 2 words)
template <typename S>
__device__ __forceinline__ int bwq_off(int i, int q) {
    return IsNarrow<S>::value && i < QG ? i * BWQ_W + 2 * q : i * BWQ_W + 4 * q;
}

// issue the copies of window plane p for the quads this thread handles (one
// commit group): quad q = row * 10 + k covers columns x0 - 4 + 4k .. + 3 of
// window row `row` (y0 - 2 + row)
template <typename S>
__device__ __forceinline__ void bwin_prefetch(uint32_t *buf, const S *__restrict__ pin,
                                              const float *__restrict__ q_in, int p, int x0, int y0,
                                              int tid, const DevParams &P) {
    const size_t N = (size_t)P.N;
    for (int q = tid; q < BWQ_QUADS; q += TX * TY) {
        float wv;
        const long long cc = bwin_cell(x0 - 4 + 4 * (q % 10), y0 + q / 10 - 2, p, P, wv);
        if (cc < 0 || !in_bounds(cc + 3, (long long)N, P)) continue;
        const S *g0 = pin + off_g(QF, 0, (size_t)cc, N);
#pragma unroll
        for (int i = 0; i < QG; ++i) {
            if (IsNarrow<S>::value) cp_async8(&buf[bwq_off<S>(i, q)], g0 + (size_t)i * N);
            else cp_async16(&buf[bwq_off<S>(i, q)], g0 + (size_t)i * N);
        }
        cp_async16(&buf[bwq_off<S>(QG, q)], q_in + cc);
    }
    cp_async_commit();
}

// phi - phi_ref of the window slots of the quads this thread fetched (same
// arithmetic as phid_at); a quad's cells are window columns 4k - 2 .. 4k + 1
template <typename S>
__device__ __forceinline__ void bwin_store(float *pl, const uint32_t *buf, int p, int x0, int y0, int tid,
                                           const DevParams &P) {
    for (int q = tid; q < BWQ_QUADS; q += TX * TY) {
        const int k = q % 10, row = q / 10;
        float wv;
        const long long cc = bwin_cell(x0 - 4 + 4 * k, y0 + row - 2, p, P, wv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sx = 4 * k - 2 + j;
            if (sx < 0 || sx >= SXB) continue;
            float v;
            if (cc < 0) {
                v = wv;
            } else {
                float g[QG];
#pragma unroll
                for (int i = 0; i < QG; ++i) {
                    if (IsNarrow<S>::value) {
                        const uint32_t w = buf[bwq_off<S>(i, q) + (j >> 1)];
                        const unsigned short h = (unsigned short)((j & 1) ? (w >> 16) : (w & 0xffffu));
                        S val;
                        memcpy(&val, &h, 2);
                        g[i] = widen(val);
                    } else {
                        g[i] = __uint_as_float(buf[bwq_off<S>(i, q) + j]);
                    }
                }
                v = fmaf(0.5f, __uint_as_float(buf[bwq_off<S>(QG, q) + j]), set_sum7<S>(g, P.set_isc[1]));
            }
            pl[row * SXB + sx] = v;
        }
    }
}

// Layer z uses f/s stage (z - zbeg) % 2 and g stage (z - zbeg) % 3.  In
// iteration z the block needs the f/s stage of z and the g stages of z and
// z + 1; the copies of f/s(z + 1) and g(z + 2) are in flight.  Once every
// thread has passed the barrier of iteration z + 1 (so is done with layer
// z), the stages of layer z receive f/s(z + 2) and g(z + 3): every copy is
// issued about one whole layer before it is awaited, and one barrier per
// layer orders both the stages and the window slots.
template <typename S, int XY, int COLL, bool BIASED>
__device__ __forceinline__ void tma_column(const TmaMaps3d &M, int par, const S *__restrict__ pin,
                                           S *__restrict__ pout, float *__restrict__ phi_prev,
                                           const float *__restrict__ q_in, float *__restrict__ q_out,
                                           int *err, const DevParams &P, unsigned char *smem,
                                           uint64_t *barF, uint64_t *barG, float *sphi,
                                           uint32_t *rbuf, const Planes3d<S> &PL) {
    using Gm = Tma3Geom<S>;
    // XY_IN / XY_WRAP tiles fetch their halo ring a layer ahead (cp.async)
    constexpr bool PRE = XY != XY_GEN;
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zbeg = blockIdx.z * Tma3Geom<S>::ZBT;
    const int zend = min(zbeg + Tma3Geom<S>::ZBT, nz);
    const int zlast = min(zend, nz - 1);          // last layer whose g is staged
    const int x = x0 + tx, y = y0 + ty;
    const size_t cxy = (size_t)y * nx + x;
    const size_t plane_cells = (size_t)nx * ny;
    unsigned char *fs_base = smem;
    unsigned char *g_base = smem + Gm::G_BASE;

    StageSet F, G;
    for (int k = 0; k < Gm::NFS; ++k)
        if (zbeg + k < zend) F.pend |= 1u << k;
    for (int k = 0; k < Gm::NG; ++k)
        if (zbeg + k <= zlast) G.pend |= 1u << k;
    if (tid == 0) {
        for (int k = 0; k < Gm::NG; ++k)
            if ((G.pend >> k) & 1u) issue_g<S>(g_base + k * Gm::G_STAGE, &barG[k], M, par, x0, y0, zbeg + k);
        for (int k = 0; k < Gm::NFS; ++k)
            if ((F.pend >> k) & 1u) issue_fs<S>(fs_base + k * Gm::FS_STAGE, &barF[k], M, par, x0, y0, zbeg + k);
    }

    // After the barrier of layer z every thread is done with layer z - 1:
    // its f/s stage takes layer z - 1 + NFS and its g stage layer z - 1 + NG
    // (the layers of a stage are NFS, NG apart).  fb and gb are the stages of
    // layer z ((z - zbeg) mod NFS and mod NG).
    static_assert(Gm::NFS == 2, "the f/s stages alternate");
    auto refill = [&](int z, int fb, int gb) {
        if (z == zbeg) return;
        const int fp = fb ^ 1, gp = gb == 0 ? Gm::NG - 1 : gb - 1;
        if (z - 1 + Gm::NFS < zend) {
            if (tid == 0) issue_fs<S>(fs_base + fp * Gm::FS_STAGE, &barF[fp], M, par, x0, y0, z - 1 + Gm::NFS);
            F.pend |= 1u << fp;
        }
        if (z - 1 + Gm::NG <= zlast) {
            if (tid == 0) issue_g<S>(g_base + gp * Gm::G_STAGE, &barG[gp], M, par, x0, y0, z - 1 + Gm::NG);
            G.pend |= 1u << gp;
        }
    };

    if (BIASED) {
        // the two-ring window: planes zbeg - 2 .. zbeg + 1 with plain loads
        // (slot of plane p: (p + 2) mod NWB), plane zbeg + 2 fetched
        for (int p = zbeg - 2; p <= zbeg + 1; ++p) {
            float *pl = sphi + ((p + 2 + NWB * 4) % NWB) * PLANEB;
            for (int sidx = tid; sidx < PLANEB; sidx += TX * TY)
                pl[sidx] = window_phid_b<S>(x0 + sidx % SXB - 2, y0 + sidx / SXB - 2, p, pin, q_in, P);
        }
        bwin_prefetch<S>(rbuf, pin, q_in, zbeg + 2, x0, y0, tid, P);
        bool ok = G.wait(barG, 0, first_wait_limit);
        int fb = 0, gb = 0;
        for (int z = zbeg; z < zend; ++z) {
            const int gn = gb == Gm::NG - 1 ? 0 : gb + 1;
            if (z > zbeg) ok = G.wait(barG, gb) && ok;        // g stage of layer z
            ok = F.wait(barF, fb) && ok;
            // window plane z + 2 (fetched a layer ago); plane z + 3 in flight
            if (z + 1 < zend) {
                bwin_prefetch<S>(rbuf + ((z - zbeg + 1) & 1) * BWIN_WORDS, pin, q_in, z + 3, x0, y0, tid, P);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                cp_async_wait_all();
            }
            bwin_store<S>(sphi + ((z + 4) % NWB) * PLANEB, rbuf + ((z - zbeg) & 1) * BWIN_WORDS, z + 2, x0, y0,
                          tid, P);
            // every thread is done with layer z - 1 and has stored its part of plane z + 2
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(err, 1);
                cp_async_wait_all();
                F.drain(barF, Gm::NFS);              // copies that may still land
                G.drain(barG, Gm::NG);
                return;
            }
            refill(z, fb, gb);
            {
                const unsigned char *b = fs_base + fb * Gm::FS_STAGE;
                const unsigned char *bg = g_base + gb * Gm::G_STAGE;
                const auto *FSp = (const typename PairOf<S>::T *)(b + Gm::OFF_FS);
                const S *Gp = (const S *)(bg + Gm::OFF_G);
                float f[QF], s[QF], g[QG];
#pragma unroll
                for (int i = 0; i < QF; ++i) unpack_pair(FSp[i * Gm::CELLS + tid], f[i], s[i]);
#pragma unroll
                for (int i = 0; i < QG; ++i) g[i] = widen(Gp[i * Gm::CELLS + tid]);
                const float qp = ((const float *)(bg + Gm::OFF_Q))[tid];
                const float phip = ((const float *)(b + Gm::OFF_PP))[tid];
                const size_t c = (size_t)z * plane_cells + cxy;
                if (XY != XY_GEN && z >= 1 && z + 1 < nz)
                    layer_update3d<S, XY, COLL, true>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out,
                                                     P, PL);
                else
                    layer_update3d<S, XY_GEN, COLL, true>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev,
                                                         q_out, P, PL);
            }
            fb ^= 1;
            gb = gn;
        }
        return;
    }

    // window of NWIN slots, plane p in slot (p + 1) % NWIN: with four, the
    // plane built while the slowest threads still update layer z - 1 never
    // overwrites one they read, so one barrier per layer suffices
    constexpr int NWIN = NW3;
    // window: plane zbeg - 1 with plain loads, plane zbeg from its g stage
    fill_plane<S, XY_GEN>(sphi, zbeg % NWIN, zbeg - 1, false, false, 0.0f, pin, q_in, x0, y0, tid, tx, ty, P);
    bool ok = G.wait(barG, 0, first_wait_limit);
    fill_plane<S, XY>(sphi, (zbeg + 1) % NWIN, zbeg, true, true, staged_phid<S>(g_base, tid, P), pin,
                       q_in, x0, y0, tid, tx, ty, P);
    if (PRE && zbeg + 1 < nz)
        ring_prefetch<S, XY>(rbuf + ((zbeg + 1) & 1) * RING_WORDS, pin, q_in, zbeg + 1, x0, y0, tid, P);

    int fb = 0, gb = 0;            // stages of layer z
    for (int z = zbeg; z < zend; ++z) {
        const int gn = gb == Gm::NG - 1 ? 0 : gb + 1;       // g stage of layer z + 1
        const bool has_next = z + 1 < nz;
        float phn = 0.0f;
        if (has_next) {
            ok = G.wait(barG, gn) && ok;
            phn = staged_phid<S>(g_base + gn * Gm::G_STAGE, tid, P);
        }
        if (PRE && has_next) {
            float *plane = sphi + ((z + 2) % NWIN) * PLANE;
            plane[(ty + 1) * SX + tx + 1] = phn;
            cp_async_wait_all();                     // this thread's ring words have landed
            ring_store<S, XY>(plane, rbuf + ((z + 1) & 1) * RING_WORDS, z + 1, x0, y0, tid, P);
        } else {
            fill_plane<S, XY>(sphi, (z + 2) % NWIN, z + 1, true, has_next, phn, pin, q_in, x0, y0, tid,
                               tx, ty, P);
        }
        ok = F.wait(barF, fb) && ok;
        // every thread is done with layer z - 1 and has built plane z + 1
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(err, 1);
            cp_async_wait_all();
            F.drain(barF, Gm::NFS);                  // copies that may still land
            G.drain(barG, Gm::NG);
            return;
        }
        refill(z, fb, gb);
        // the ring of plane z + 2 goes into the buffer plane z's ring used
        if (PRE && z + 2 < nz && z + 1 < zend)
            ring_prefetch<S, XY>(rbuf + (z & 1) * RING_WORDS, pin, q_in, z + 2, x0, y0, tid, P);
        {
            const unsigned char *b = fs_base + fb * Gm::FS_STAGE;
            const unsigned char *bg = g_base + gb * Gm::G_STAGE;
            const auto *FSp = (const typename PairOf<S>::T *)(b + Gm::OFF_FS);
            const S *Gp = (const S *)(bg + Gm::OFF_G);
            float f[QF], s[QF], g[QG];
#pragma unroll
            for (int i = 0; i < QF; ++i) unpack_pair(FSp[i * Gm::CELLS + tid], f[i], s[i]);
#pragma unroll
            for (int i = 0; i < QG; ++i) g[i] = widen(Gp[i * Gm::CELLS + tid]);
            const float qp = ((const float *)(bg + Gm::OFF_Q))[tid];
            const float phip = ((const float *)(b + Gm::OFF_PP))[tid];
            const size_t c = (size_t)z * plane_cells + cxy;
            if (XY != XY_GEN && z >= 1 && z + 1 < nz)
                layer_update3d<S, XY, COLL, false, NWIN>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P, PL);
            else
                layer_update3d<S, XY_GEN, COLL, false, NWIN>(sphi, z, x, y, c, f, s, g, qp, phip, pout, phi_prev, q_out, P, PL);
        }
        fb ^= 1;
        gb = gn;
    }
}

template <typename S, int COLL, bool BIASED>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY))
step3d_tma_kernel(const __grid_constant__ TmaMaps3d maps, const S *__restrict__ pin,
                  S *__restrict__ pout, float *__restrict__ phi_prev,
                  const float *__restrict__ q_in, float *__restrict__ q_out, int par, int *err,
                  const DevParams P, const __grid_constant__ Planes3d<S> PL) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // bulk tensor copies want 128-byte aligned destinations
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    __shared__ __align__(8) uint64_t barF[Tma3Geom<S>::NFS], barG[Tma3Geom<S>::NG];
    pdl_wait();
    // the biased gradient: a five-plane two-ring window, two fetched planes
    __shared__ float sphi[BIASED ? NWB * PLANEB : NW3 * PLANE];
    __shared__ __align__(16) uint32_t rbuf[BIASED ? 2 * BWIN_WORDS : 2 * RING_WORDS];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    if (x0 + TX > P.n[0] || y0 + TY > P.n[1]) {          // ragged tile: plain loads
        if (BIASED) {
            // the host runs this kernel with the biased gradient only on grids
            // without ragged tiles; record the broken precondition
            if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(err, 2);
            return;
        }
        step3d_column<S, XY_GEN, COLL, Tma3Geom<S>::ZBT>(pin, pout, phi_prev, q_in, q_out, P, sphi, PL);
        return;
    }
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        for (int k = 0; k < Tma3Geom<S>::NFS; ++k) mbar_init(&barF[k], 1);
        for (int k = 0; k < Tma3Geom<S>::NG; ++k) mbar_init(&barG[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // interior tiles run the wrap-aware code too (its selects never fire
    // there): one fast instantiation instead of two keeps the hot code small
    // enough for the instruction cache (measured: FP32 +1.9%, FP16 +3.9%)
    const int cls = tile_class3d(x0, y0, P);
    if (cls != XY_GEN)
        tma_column<S, XY_WRAP, COLL, BIASED>(maps, par, pin, pout, phi_prev, q_in, q_out, err, P, smem, barF, barG, sphi, rbuf, PL);
    else
        tma_column<S, XY_GEN, COLL, BIASED>(maps, par, pin, pout, phi_prev, q_in, q_out, err, P, smem, barF, barG, sphi, rbuf, PL);
}

// ------------------------------------------------------------------ host side
bool tma3d_eligible(const DevParams &P, int elem_bytes) {
    const long long nx = P.n[0], ny = P.n[1];
    if (nx < TX || ny < TY || P.n[2] < 1) return false;
    if ((nx * elem_bytes) % 16 != 0 || (nx * 4) % 16 != 0) return false;
    return true;
}

int make_tma_maps3d(TmaMaps3d *M, const DevParams &P, int elem_bytes, void *const pops[2],
                    float *const q[2], float *phi_prev) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return -1;
    const cuuint64_t nx = (cuuint64_t)P.n[0], ny = (cuuint64_t)P.n[1], nz = (cuuint64_t)P.n[2];
    const cuuint64_t N = (cuuint64_t)P.N, es = (cuuint64_t)elem_bytes;
    const cuuint32_t one[4] = {1, 1, 1, 1};
    // a single value, and a (f_i, s_i) pair copied as one element of twice the size
    const CUtensorMapDataType dt = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                   : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const CUtensorMapDataType dt2 = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    // `planes` planes of `e`-byte elements, population planes pstride bytes apart
    auto map4 = [&](CUtensorMap *m, void *base, CUtensorMapDataType t, cuuint64_t e, cuuint32_t planes,
                    cuuint64_t pstride) {
        const cuuint64_t dims[4] = {nx, ny, nz, (cuuint64_t)planes};
        const cuuint64_t str[3] = {nx * e, nx * ny * e, pstride};
        const cuuint32_t box[4] = {TX, TY, 1, planes};
        return enc(m, t, 4, base, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto map3 = [&](CUtensorMap *m, void *base) {
        const cuuint64_t dims[3] = {nx, ny, nz};
        const cuuint64_t str[2] = {nx * 4, nx * ny * 4};
        const cuuint32_t box[3] = {TX, TY, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, str, box, one,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b) {
        if (!map4(&M->fs[b], pops[b], dt2, 2 * es, QF, 2 * N * es)) return -2;
        if (!map4(&M->g[b], (char *)pops[b] + off_g(QF, 0, 0, N) * es, dt, es, QG, N * es)) return -3;
        if (!map3(&M->q[b], q[b])) return -4;
    }
    if (!map3(&M->pp, phi_prev)) return -5;
    return 0;
}

template <typename S, int COLL, bool BIASED>
static int blocks_per_sm_one() {
    int n = 0;
    const int dyn = Tma3Geom<S>::DYN;
    if (cudaFuncSetAttribute(step3d_tma_kernel<S, COLL, BIASED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dyn) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step3d_tma_kernel<S, COLL, BIASED>, TX * TY, dyn) !=
        cudaSuccess)
        return 0;
    return n;
}

// every collision and gradient instantiation gets the shared-memory limit;
// the BGK and TRT central-gradient ones set the occupancy, every other one
// must fit at least one block
template <typename S>
static int blocks_per_sm_for() {
    const int a = blocks_per_sm_one<S, COLL_BGK, false>(), b = blocks_per_sm_one<S, COLL_TRT, false>();
    if (blocks_per_sm_one<S, COLL_MRT, false>() < 1 || blocks_per_sm_one<S, COLL_BGK, true>() < 1 ||
        blocks_per_sm_one<S, COLL_TRT, true>() < 1 || blocks_per_sm_one<S, COLL_MRT, true>() < 1)
        return 0;
    return a < b ? a : b;
}

int tma3d_blocks_per_sm(int elem_bytes) {
    if (elem_bytes == 4) return blocks_per_sm_for<float>();
    const int a = blocks_per_sm_for<__half>(), b = blocks_per_sm_for<__nv_bfloat16>();
    return a < b ? a : b;
}

template <typename S>
cudaError_t launch_step3d_tma(const TmaMaps3d &M, int par, const void *pin, void *pout,
                              float *phi_prev, const float *q_in, float *q_out, int *err,
                              const DevParams &P, cudaStream_t st) {
    dim3 block(TX, TY);
    constexpr int zb = Tma3Geom<S>::ZBT;
    dim3 grid((P.n[0] + TX - 1) / TX, (P.n[1] + TY - 1) / TY, (P.n[2] + zb - 1) / zb);
    const Planes3d<S> PL = planes3d<S>(pin, pout, P);
    const S *in = (const S *)pin;
    S *out = (S *)pout;
#define LBM_TMA3_LAUNCH(C, B)                                                                   \
    pdl_launch(step3d_tma_kernel<S, C, B>, grid, block, Tma3Geom<S>::DYN, st, M, in, out, phi_prev, q_in, \
               q_out, par, err, P, PL)
    switch (P.opts & (OPT_TRT | OPT_MRT | OPT_BIASED)) {
    case 0: LBM_TMA3_LAUNCH(COLL_BGK, false); break;
    case OPT_TRT: LBM_TMA3_LAUNCH(COLL_TRT, false); break;
    case OPT_MRT: LBM_TMA3_LAUNCH(COLL_MRT, false); break;
    case OPT_BIASED: LBM_TMA3_LAUNCH(COLL_BGK, true); break;
    case OPT_TRT | OPT_BIASED: LBM_TMA3_LAUNCH(COLL_TRT, true); break;
    case OPT_MRT | OPT_BIASED: LBM_TMA3_LAUNCH(COLL_MRT, true); break;
    default: return cudaErrorInvalidValue;
    }
#undef LBM_TMA3_LAUNCH
    return cudaGetLastError();
}

#define LBM_INST3DTMA(S)                                                                        \
    template cudaError_t launch_step3d_tma<S>(const TmaMaps3d &, int, const void *, void *,     \
                                              float *, const float *, float *, int *,           \
                                              const DevParams &, cudaStream_t);
LBM_INST3DTMA(float)
LBM_INST3DTMA(__half)
LBM_INST3DTMA(__nv_bfloat16)

}  // namespace lbm
