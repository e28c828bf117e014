// fpd_lattice.cu -- the fused lattice sweep of the FPD-MRT step and the
// lattice-wide helper kernels (initialisation, fields, population I/O,
// diagnostics).
//
// The sweep (Sec. 2.3, item (2), with the item-(1) fields of Eqs. 1, 2, 4):
// one thread per cell, 32 x 8 cells per CTA.  The bead phase has marked, in
// a bit mask per tile, every bead whose support (|r - R_i| < a + phi_cut xi)
// can reach the tile; a tile whose mask is empty ("cold") uses the fluid
// rates and the uniform body force, a "hot" tile evaluates phi_i, the
// viscosity of Eq. 1 and the spread force of Eq. 4 per cell, visiting the
// marked beads in bead order.  Every cell gathers its 9 populations (AA
// pattern, bounce-back at the walls), collides (MRT + Guo) and scatters them
// back in place.  No block-wide barrier: each thread reads the tile's mask.
#include <cuda_fp16.h>

#include <type_traits>

#include "fpd_kernels.h"

namespace fpd {

namespace {

template <class S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Relaxation rates and force density of one cell (Eqs. 1, 2, 4) from the
// beads marked in its tile's mask (m, W words; any = OR of the words).
template <class R>
__device__ __forceinline__ void cell_overlay(const Inst &I, const BeadTab &tab, const unsigned *__restrict__ m,
                                             const int W, const unsigned any, const int x, const int y, R &Fx,
                                             R &Fy, R &s_nu, R &s_e, R &s_eps, R &s_q) {
    if constexpr (std::is_same<R, double>::value) {
        Fx = I.gx;
        Fy = I.gy;
        if (any == 0u && !I.sandwich) {
            s_nu = I.fluid_rates_d[0];
            s_e = I.fluid_rates_d[1];
            s_eps = I.fluid_rates_d[2];
            s_q = I.fluid_rates_d[3];
            return;
        }
        const double xc = x + 0.5, yc = y + 0.5;
        double Phi = I.sandwich ? sandwich_phi_f64(I, yc) : 0.0;
        for (int w = 0; w < W; ++w) {
            unsigned bits = m[w];
            while (bits) {
                const int q = I.bead_off + 32 * w + __ffs(bits) - 1;
                bits &= bits - 1u;
                const double ph = phi_f64(I, xc, yc, tab.Rx[q], tab.Ry[q]);
                if (ph != 0.0) {
                    Phi += ph;
                    Fx += ph * tab.Gx[q];
                    Fy += ph * tab.Gy[q];
                }
            }
        }
        const double nu = I.nu_f * (1.0 + (I.visc_ratio - 1.0) * Phi);
        rates<double>(I.collision, nu, I.s_e, I.s_eps, I.s_q, s_nu, s_e, s_eps, s_q);
    } else {
        Fx = I.f_gx;
        Fy = I.f_gy;
        if (any == 0u && !I.sandwich) {
            s_nu = I.fluid_rates_f[0];
            s_e = I.fluid_rates_f[1];
            s_eps = I.fluid_rates_f[2];
            s_q = I.fluid_rates_f[3];
            return;
        }
        const float hnx = 0.5f * I.nx, fnx = (float)I.nx;
        const float xc = (float)x + 0.5f, yc = (float)y + 0.5f;
        float Phi = I.sandwich ? sandwich_phi_f32(I, yc) : 0.f;
        for (int w = 0; w < W; ++w) {
            unsigned bits = m[w];
            while (bits) {
                const int q = I.bead_off + 32 * w + __ffs(bits) - 1;
                bits &= bits - 1u;
                // (x_c - R_x) with R_x = hi + lo; the periodic shift is
                // applied to the cell centre first so that xc - hi is exact
                const float bx = tab.xh[q];
                float xcl = xc;
                const float d0 = xcl - bx;
                xcl = (d0 > hnx) ? xcl - fnx : ((d0 < -hnx) ? xcl + fnx : xcl);
                const float dx = (xcl - bx) - tab.xl[q];
                const float dy = (yc - tab.yh[q]) - tab.yl[q];
                const float ph = phi_f32(dx, dy, I.f_a, I.f_inv_xi, I.f_rcut2);
                Phi += ph;
                Fx += ph * tab.gxf[q];
                Fy += ph * tab.gyf[q];
            }
        }
        const float nu = I.f_nu_f * (1.0f + I.f_visc_m1 * Phi);
        rates<float>(I.collision, nu, I.f_s_e, I.f_s_eps, I.f_s_q, s_nu, s_e, s_eps, s_q);
    }
}

// One tile of the sweep: tile (bx, by) of instance I at the instance's step
// parity.  The CTA has kTileX x (kTileY / CY) threads; thread (tx, ty) owns
// the CY cells (x, y0 + ty + k kTileY / CY), k < CY, of its column.
template <class S, int CY>
__device__ __forceinline__ void lattice_tile(const Inst &I, S *__restrict__ pool, const BeadTab &tab,
                                             const unsigned *__restrict__ mask_read, unsigned *__restrict__ mask_clear,
                                             const int bx, const int by, const int parity, const int early_load) {
    using R = typename Real<S>::type;
    constexpr int RY = kTileY / CY;
    const int x = bx * kTileX + threadIdx.x;
    const int tile = I.tile_base + by * I.ntx + bx;
    const int W = I.mask_words;
    S *A = pool + I.pop_off;
    int y[CY];
    bool valid[CY];
    Cell C[CY];
    R g[CY][9];
#pragma unroll
    for (int k = 0; k < CY; ++k) {
        y[k] = by * kTileY + threadIdx.y + k * RY;
        valid[k] = x < I.nx && y[k] < I.ny;
        C[k] = make_cell(I, x, valid[k] ? y[k] : 0);
    }
    // populations come from the previous sweep; when the bead phase runs
    // between the two sweeps they may be loaded before waiting on it
    if (early_load) {
#pragma unroll
        for (int k = 0; k < CY; ++k)
            if (valid[k]) load_pops<S, R>(A, I, C[k], parity, g[k]);
    }
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0 && threadIdx.y == 0)  // the other parity's mask, for the next bead phase
        for (int w = 0; w < W; ++w) mask_clear[tile * W + w] = 0u;
    if (!valid[0]) return;  // cells further down the column are invalid too
    if (!early_load) {
#pragma unroll
        for (int k = 0; k < CY; ++k)
            if (valid[k]) load_pops<S, R>(A, I, C[k], parity, g[k]);
    }
    const unsigned *m = mask_read + tile * W;
    unsigned any = 0u;
    for (int w = 0; w < W; ++w) any |= m[w];
#pragma unroll
    for (int k = 0; k < CY; ++k) {
        if (!valid[k]) continue;
        R Fx, Fy, s_nu, s_e, s_eps, s_q;
        cell_overlay<R>(I, tab, m, W, any, x, y[k], Fx, Fy, s_nu, s_e, s_eps, s_q);
        collide<R>(g[k], Fx, Fy, s_nu, s_e, s_eps, s_q);
        store_pops<S, R>(A, I, C[k], parity, g[k]);
    }
}

template <class S, int CY>
__global__ void __launch_bounds__(kTileX *kTileY / CY)
    k_lattice(const Inst I, S *__restrict__ pool, const BeadTab tab, const unsigned *__restrict__ mask_read,
              unsigned *__restrict__ mask_clear, const int parity, const int early_load) {
    lattice_tile<S, CY>(I, pool, tab, mask_read, mask_clear, blockIdx.x, blockIdx.y, parity, early_load);
}

// Batched sweep over a packed tile list: tiles[t] = (instance slot,
// by << 16 | bx).  Each instance reads table and layout of its own parity
// (global parity ^ par_xor); the record is copied to shared memory per CTA.
template <class S, int CY>
__global__ void __launch_bounds__(kTileX *kTileY / CY)
    k_lattice_batch(const Inst *__restrict__ insts, const int2 *__restrict__ tiles, S *__restrict__ pool,
                    const BeadTab tab0, const BeadTab tab1, const unsigned *__restrict__ mask_read,
                    unsigned *__restrict__ mask_clear, const int gparity, const int early_load) {
    __shared__ Inst sI;
    const int2 t = tiles[blockIdx.x];
    {
        const unsigned *src = (const unsigned *)(insts + t.x);
        unsigned *dst = (unsigned *)&sI;
        const int tid = threadIdx.y * kTileX + threadIdx.x;
        for (int wd = tid; wd < (int)(sizeof(Inst) / 4); wd += kTileX * kTileY / CY) dst[wd] = src[wd];
    }
    __syncthreads();
    const int parity = gparity ^ sI.par_xor;
    lattice_tile<S, CY>(sI, pool, parity ? tab1 : tab0, mask_read, mask_clear, t.y & 0xffff, t.y >> 16, parity,
                        early_load);
}

// Equilibrium start: f_k = f_k^eq(rho = 1, u = (u_wall(y), 0)) with the
// linear wall profile, or the rest state; stored as deviations for parity 0.
template <class S>
__global__ void k_init(const Inst I, S *__restrict__ pool, int couette) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    const double ux = couette ? I.u_bot + (I.u_top - I.u_bot) * (y + 0.5) / I.ny : 0.0;
    S *A = pool + I.pop_off;
    const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double cu = cxs[k] * ux;
        const double gk = ws[k] * (3.0 * cu + 4.5 * cu * cu - 1.5 * ux * ux);
        Store<S>::st(A + (int64_t)k * I.plane + (int64_t)y * I.pitch + x,
                     (typename Real<S>::type)gk, I.scale[k]);
    }
}

// Force density of Eq. 4 at a cell from the beads marked in its tile.
__device__ __forceinline__ void overlay_f64(const Inst &I, const BeadTab &tab, const unsigned *mask, int x, int y,
                                            double &fx, double &fy) {
    fx = I.gx;
    fy = I.gy;
    const int tile = I.tile_base + (y / kTileY) * I.ntx + x / kTileX;
    const double xc = x + 0.5, yc = y + 0.5;
    for (int w = 0; w < I.mask_words; ++w) {
        // without masks every bead of the instance is visited (cutoff exact)
        const int left = I.nb - 32 * w;
        unsigned bits = mask ? mask[tile * I.mask_words + w] : (left >= 32 ? 0xffffffffu : ((1u << left) - 1u));
        while (bits) {
            const int q = I.bead_off + 32 * w + __ffs(bits) - 1;
            bits &= bits - 1u;
            const double ph = phi_f64(I, xc, yc, tab.Rx[q], tab.Ry[q]);
            if (ph != 0.0) {
                fx += ph * tab.Gx[q];
                fy += ph * tab.Gy[q];
            }
        }
    }
}

template <class S>
__global__ void k_fields(const Inst I, const S *__restrict__ pool, const BeadTab tab, const unsigned *mask,
                         int parity, double *__restrict__ ux, double *__restrict__ uy, double *__restrict__ rho) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    double g[9];
    load_pops<S, double>(pool + I.pop_off, I, make_cell(I, x, y), parity, g);
    double dr = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) dr += g[k];
    const double r = 1.0 + dr;
    const double jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    const double jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    double fx, fy;
    overlay_f64(I, tab, mask, x, y, fx, fy);
    const int64_t c = (int64_t)y * I.nx + x;
    ux[c] = (jx + 0.5 * fx) / r;
    uy[c] = (jy + 0.5 * fy) / r;
    rho[c] = r;
}

template <class S>
__global__ void k_read_pops(const Inst I, const S *__restrict__ pool, int parity, double *__restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    double g[9];
    load_pops<S, double>(pool + I.pop_off, I, make_cell(I, x, y), parity, g);
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k * n + c] = g[k] + ws[k];
}

// Inverse of the parity read: place the deviations of a given state where
// the next step will gather them (bounce-back term removed at the walls).
template <int k, class S>
__device__ __forceinline__ void write_one(S *A, const Inst &I, const Cell &C, int parity, double gk) {
    using R = typename Real<S>::type;
    constexpr int cx = Q<k>::cx, cy = Q<k>::cy, o = Q<k>::opp;
    if (parity == 0) {
        Store<S>::st(A + (k * I.plane32 + C.r0 + C.x), (R)gk, I.scale[k]);
        return;
    }
    const bool wall = (cy > 0 && C.bot) || (cy < 0 && C.top);
    if (wall) {
        Store<S>::st(A + (k * I.plane32 + C.r0 + C.x), (R)(gk - I.bbd[cy > 0 ? 0 : 1][k]), I.scale[k]);
    } else {
        const int rs = cy > 0 ? C.rm : (cy < 0 ? C.rp : C.r0);
        const int xs = cx > 0 ? C.xm : (cx < 0 ? C.xp : C.x);
        Store<S>::st(A + (o * I.plane32 + rs + xs), (R)gk, I.scale[o]);
    }
}

template <class S>
__global__ void k_write_pops(const Inst I, S *__restrict__ pool, int parity, const double *__restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    S *A = pool + I.pop_off;
    const Cell C = make_cell(I, x, y);
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
    write_one<0>(A, I, C, parity, f[0 * n + c] - Q<0>::w);
    write_one<1>(A, I, C, parity, f[1 * n + c] - Q<1>::w);
    write_one<2>(A, I, C, parity, f[2 * n + c] - Q<2>::w);
    write_one<3>(A, I, C, parity, f[3 * n + c] - Q<3>::w);
    write_one<4>(A, I, C, parity, f[4 * n + c] - Q<4>::w);
    write_one<5>(A, I, C, parity, f[5 * n + c] - Q<5>::w);
    write_one<6>(A, I, C, parity, f[6 * n + c] - Q<6>::w);
    write_one<7>(A, I, C, parity, f[7 * n + c] - Q<7>::w);
    write_one<8>(A, I, C, parity, f[8 * n + c] - Q<8>::w);
}

constexpr int kDiagThreads = 256;

template <class S>
__global__ void __launch_bounds__(kDiagThreads)
    k_diag(const Inst I, const S *__restrict__ pool, int parity, double *__restrict__ partial) {
    __shared__ double sh[4][kDiagThreads / 32];
    double m = 0.0, px = 0.0, py = 0.0, bad = 0.0;
    const int64_t ncell = (int64_t)I.nx * I.ny;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(c / I.nx), x = (int)(c - (int64_t)y * I.nx);
        double g[9];
        load_pops<S, double>(pool + I.pop_off, I, make_cell(I, x, y), parity, g);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            m += g[k];
            if (!isfinite(g[k])) bad += 1.0;
        }
        px += g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
        py += g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    }
    double v[4] = {m, px, py, bad};
#pragma unroll
    for (int i = 0; i < 4; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0)
        for (int i = 0; i < 4; ++i) sh[i][w] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) {
            double t = 0.0;
            for (int j = 0; j < kDiagThreads / 32; ++j) t += sh[i][j];
            partial[4 * blockIdx.x + i] = t;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <class S, int CY>
static cudaError_t lattice_t(const Inst &I, void *pool, BeadTab tab, const unsigned *mask_read,
                             unsigned *mask_clear, int parity, int after_beads, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(I.ntx, I.nty);
    cfg.blockDim = dim3(kTileX, kTileY / CY);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_beads ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_lattice<S, CY>, I, (S *)pool, tab, mask_read, mask_clear, parity,
                              after_beads);
}

template <class S>
static cudaError_t lattice_v(int variant, const Inst &I, void *pool, BeadTab tab, const unsigned *mask_read,
                             unsigned *mask_clear, int parity, int after_beads, cudaStream_t st) {
    if (variant == 1) return lattice_t<S, 2>(I, pool, tab, mask_read, mask_clear, parity, after_beads, st);
    return lattice_t<S, 1>(I, pool, tab, mask_read, mask_clear, parity, after_beads, st);
}

cudaError_t launch_lattice(int precision, const Inst *, const Inst &inst_h, void *pool, BeadTab tab,
                           const unsigned *mask_read, unsigned *mask_clear, int parity, int after_beads,
                           int variant, cudaStream_t st) {
    switch (precision) {
        case 0: return lattice_v<double>(variant, inst_h, pool, tab, mask_read, mask_clear, parity, after_beads, st);
        case 1: return lattice_v<float>(variant, inst_h, pool, tab, mask_read, mask_clear, parity, after_beads, st);
        case 2: return lattice_v<__half>(variant, inst_h, pool, tab, mask_read, mask_clear, parity, after_beads, st);
    }
    return cudaErrorInvalidValue;
}

template <class S, int CY>
static cudaError_t lattice_batch_t(const Inst *insts, const int2 *tiles, int ntiles, void *pool, BeadTab tab0,
                                   BeadTab tab1, const unsigned *mask_read, unsigned *mask_clear, int gparity,
                                   int after_beads, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntiles);
    cfg.blockDim = dim3(kTileX, kTileY / CY);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_beads ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_lattice_batch<S, CY>, insts, tiles, (S *)pool, tab0, tab1, mask_read,
                              mask_clear, gparity, after_beads);
}

template <class S>
static cudaError_t lattice_batch_v(int variant, const Inst *insts, const int2 *tiles, int ntiles, void *pool,
                                   BeadTab tab0, BeadTab tab1, const unsigned *mask_read, unsigned *mask_clear,
                                   int gparity, int after_beads, cudaStream_t st) {
    if (variant == 1)
        return lattice_batch_t<S, 2>(insts, tiles, ntiles, pool, tab0, tab1, mask_read, mask_clear, gparity,
                                     after_beads, st);
    return lattice_batch_t<S, 1>(insts, tiles, ntiles, pool, tab0, tab1, mask_read, mask_clear, gparity,
                                 after_beads, st);
}

cudaError_t launch_lattice_batch(int precision, const Inst *insts, const int2 *tiles, int ntiles, void *pool,
                                 BeadTab tab0, BeadTab tab1, const unsigned *mask_read, unsigned *mask_clear,
                                 int gparity, int after_beads, int variant, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (precision) {
        case 0: return lattice_batch_v<double>(variant, insts, tiles, ntiles, pool, tab0, tab1, mask_read, mask_clear, gparity, after_beads, st);
        case 1: return lattice_batch_v<float>(variant, insts, tiles, ntiles, pool, tab0, tab1, mask_read, mask_clear, gparity, after_beads, st);
        case 2: return lattice_batch_v<__half>(variant, insts, tiles, ntiles, pool, tab0, tab1, mask_read, mask_clear, gparity, after_beads, st);
    }
    return cudaErrorInvalidValue;
}

#define FPD_DISPATCH(precision, CALL)                        \
    switch (precision) {                                     \
        case 0: { using S = double; CALL; } break;           \
        case 1: { using S = float; CALL; } break;            \
        case 2: { using S = __half; CALL; } break;           \
        default: return cudaErrorInvalidValue;               \
    }

static dim3 row_grid(const Inst &I, int bx) { return dim3((I.nx + bx - 1) / bx, I.ny); }

cudaError_t launch_init(int precision, const Inst *, const Inst &I, void *pool, int couette, cudaStream_t st) {
    FPD_DISPATCH(precision, (k_init<S><<<row_grid(I, 128), 128, 0, st>>>(I, (S *)pool, couette)));
    return cudaGetLastError();
}

cudaError_t launch_fields(int precision, const Inst *, const Inst &I, const void *pool, BeadTab tab,
                          const unsigned *mask, int parity, double *ux, double *uy, double *rho, cudaStream_t st) {
    FPD_DISPATCH(precision, (k_fields<S><<<row_grid(I, 128), 128, 0, st>>>(I, (const S *)pool, tab, mask, parity,
                                                                              ux, uy, rho)));
    return cudaGetLastError();
}

cudaError_t launch_read_pops(int precision, const Inst *, const Inst &I, const void *pool, int parity, double *f,
                             cudaStream_t st) {
    FPD_DISPATCH(precision, (k_read_pops<S><<<row_grid(I, 128), 128, 0, st>>>(I, (const S *)pool, parity, f)));
    return cudaGetLastError();
}

cudaError_t launch_write_pops(int precision, const Inst *, const Inst &I, void *pool, int parity, const double *f,
                              cudaStream_t st) {
    FPD_DISPATCH(precision, (k_write_pops<S><<<row_grid(I, 128), 128, 0, st>>>(I, (S *)pool, parity, f)));
    return cudaGetLastError();
}

int diag_blocks(const Inst &I) {
    const int64_t ncell = (int64_t)I.nx * I.ny;
    int64_t b = (ncell + kDiagThreads - 1) / kDiagThreads;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

cudaError_t launch_diag(int precision, const Inst *, const Inst &I, const void *pool, int parity, double *partial,
                        cudaStream_t st) {
    const int nb = diag_blocks(I);
    FPD_DISPATCH(precision, (k_diag<S><<<nb, kDiagThreads, 0, st>>>(I, (const S *)pool, parity, partial)));
    return cudaGetLastError();
}

}  // namespace fpd
