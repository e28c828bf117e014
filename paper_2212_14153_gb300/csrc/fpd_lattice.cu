// fpd_lattice.cu -- the fused lattice sweep of the FPD-MRT step and the
// lattice-wide helper kernels (initialisation, fields, population I/O,
// diagnostics).
//
// The sweep (Sec. 2.3, item (2), with the item-(1) fields of Eqs. 1, 2, 4):
// one thread per cell, 32 x 8 cells per CTA.  Warp 0 first lists, in bead
// order, the beads whose support (|r - R_i| < a + phi_cut xi) can reach the
// tile; only such "hot" tiles evaluate phi_i, the viscosity of Eq. 1 and the
// spread force of Eq. 4 per cell, cold tiles use the fluid rates and no
// force.  Every cell then gathers its 9 populations (AA pattern, bounce-back
// at the walls), collides (MRT + Guo) and scatters them back in place.
#include <cuda_fp16.h>

#include <type_traits>

#include "fpd_kernels.h"

namespace fpd {

namespace {

template <class S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Distance from a bead at (Rx, Ry) to the rectangle of cell centres
// [xa, xb] x [ya, yb], minimised over the periodic images in x.
__device__ __forceinline__ double tile_dist2(double Rx, double Ry, double xa, double xb, double ya, double yb,
                                             double nx) {
    const double cxm = 0.5 * (xa + xb), hx = 0.5 * (xb - xa);
    double d = Rx - cxm;
    d = d - nx * floor(d / nx + 0.5);
    double ad = fabs(d);
    ad = fmin(ad, fabs(d - nx));
    ad = fmin(ad, fabs(d + nx));
    const double dxr = fmax(0.0, ad - hx);
    const double cym = 0.5 * (ya + yb), hy = 0.5 * (yb - ya);
    const double dyr = fmax(0.0, fabs(Ry - cym) - hy);
    return dxr * dxr + dyr * dyr;
}

template <class S>
__global__ void __launch_bounds__(kTileX *kTileY)
    k_lattice(const Inst I, S *__restrict__ pool, const BeadTab tab, const int parity) {
    using R = typename Real<S>::type;
    constexpr bool kF64 = std::is_same<R, double>::value;
    // hot-tile bead list: FP64 path keeps (Rx, Ry, Gx, Gy) in double; the
    // FP32 paths keep the hi/lo float split and G in float
    __shared__ int s_n;
    __shared__ R s_bx[kMaxBeads], s_by[kMaxBeads], s_gx[kMaxBeads], s_gy[kMaxBeads];
    __shared__ float s_xl[kF64 ? 1 : kMaxBeads], s_yl[kF64 ? 1 : kMaxBeads];

    const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kTileY;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < I.nx && y < I.ny;
    S *A = pool + I.pop_off;

    // the population loads do not depend on the bead list: issue them first
    R g[9];
    if (valid) load_pops<S, R>(A, I, x, y, parity, g);

    if (ty == 0) {
        // list the beads whose support reaches this tile, in bead order
        int n = 0;
        for (int base = 0; base < I.nb; base += 32) {
            const int b = base + tx;
            bool hit = false;
            if constexpr (kF64) {
                double Rx = 0.0, Ry = 0.0;
                if (b < I.nb) {
                    Rx = tab.Rx[I.bead_off + b];
                    Ry = tab.Ry[I.bead_off + b];
                    const double reach = I.rcut + 1e-6;
                    hit = tile_dist2(Rx, Ry, x0 + 0.5, x0 + kTileX - 0.5, y0 + 0.5, y0 + kTileY - 0.5,
                                     (double)I.nx) < reach * reach;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = n + __popc(mask & ((1u << tx) - 1u));
                    s_bx[pos] = Rx;
                    s_by[pos] = Ry;
                    s_gx[pos] = tab.Gx[I.bead_off + b];
                    s_gy[pos] = tab.Gy[I.bead_off + b];
                }
                n += __popc(mask);
            } else {
                float xh = 0.f, yh = 0.f;
                if (b < I.nb) {
                    xh = tab.xh[I.bead_off + b];
                    yh = tab.yh[I.bead_off + b];
                    // FP32 distance from the tile's cell-centre rectangle,
                    // nearest periodic image, 0.05 margin for the rounding
                    const float fnx = (float)I.nx;
                    float d = xh - ((float)x0 + 0.5f * kTileX);
                    d -= fnx * rintf(d / fnx);
                    float ad = fminf(fabsf(d), fminf(fabsf(d - fnx), fabsf(d + fnx)));
                    const float dxr = fmaxf(0.f, ad - 0.5f * (kTileX - 1));
                    const float dyr = fmaxf(0.f, fabsf(yh - ((float)y0 + 0.5f * kTileY)) - 0.5f * (kTileY - 1));
                    const float reach = I.f_rcut + 0.05f;
                    hit = dxr * dxr + dyr * dyr < reach * reach;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = n + __popc(mask & ((1u << tx) - 1u));
                    s_bx[pos] = xh;
                    s_by[pos] = yh;
                    s_xl[pos] = tab.xl[I.bead_off + b];
                    s_yl[pos] = tab.yl[I.bead_off + b];
                    s_gx[pos] = tab.gxf[I.bead_off + b];
                    s_gy[pos] = tab.gyf[I.bead_off + b];
                }
                n += __popc(mask);
            }
        }
        if (tx == 0) s_n = n;
    }
    __syncthreads();
    if (!valid) return;

    const int nhot = s_n;
    R s_nu, s_e, s_eps, s_q, Fx, Fy;
    if constexpr (kF64) {
        Fx = I.gx;
        Fy = I.gy;
        if (nhot == 0) {
            s_nu = I.fluid_rates_d[0];
            s_e = I.fluid_rates_d[1];
            s_eps = I.fluid_rates_d[2];
            s_q = I.fluid_rates_d[3];
        } else {
            double Phi = 0.0;
            const double xc = x + 0.5, yc = y + 0.5;
            for (int q = 0; q < nhot; ++q) {
                const double ph = phi_f64(I, xc, yc, s_bx[q], s_by[q]);
                if (ph != 0.0) {
                    Phi += ph;
                    Fx += ph * s_gx[q];
                    Fy += ph * s_gy[q];
                }
            }
            const double nu = I.nu_f * (1.0 + (I.visc_ratio - 1.0) * Phi);
            rates<double>(I.collision, nu, I.s_e, I.s_eps, I.s_q, s_nu, s_e, s_eps, s_q);
        }
    } else {
        Fx = I.f_gx;
        Fy = I.f_gy;
        if (nhot == 0) {
            s_nu = I.fluid_rates_f[0];
            s_e = I.fluid_rates_f[1];
            s_eps = I.fluid_rates_f[2];
            s_q = I.fluid_rates_f[3];
        } else {
            float Phi = 0.f;
            const float hnx = 0.5f * I.nx, fnx = (float)I.nx;
            const float xc = (float)x + 0.5f, yc = (float)y + 0.5f;
            for (int q = 0; q < nhot; ++q) {
                // (x_c - R_x) with R_x = hi + lo; the periodic shift is
                // applied to the cell centre first so that xc - hi is exact
                float xcl = xc;
                const float d0 = xcl - s_bx[q];
                xcl = (d0 > hnx) ? xcl - fnx : ((d0 < -hnx) ? xcl + fnx : xcl);
                const float dx = (xcl - s_bx[q]) - s_xl[q];
                const float dy = (yc - s_by[q]) - s_yl[q];
                const float ph = phi_f32(dx, dy, I.f_a, I.f_inv_xi, I.f_rcut2);
                Phi += ph;
                Fx += ph * s_gx[q];
                Fy += ph * s_gy[q];
            }
            const float nu = I.f_nu_f * (1.0f + I.f_visc_m1 * Phi);
            rates<float>(I.collision, nu, I.f_s_e, I.f_s_eps, I.f_s_q, s_nu, s_e, s_eps, s_q);
        }
    }
    collide<R>(g, Fx, Fy, s_nu, s_e, s_eps, s_q);
    store_pops<S, R>(A, I, x, y, parity, g);
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

__device__ __forceinline__ void overlay_f64(const Inst &I, const BeadTab &tab, double xc, double yc, double &fx,
                                            double &fy) {
    fx = I.gx;
    fy = I.gy;
    for (int q = 0; q < I.nb; ++q) {
        const double ph = phi_f64(I, xc, yc, tab.Rx[I.bead_off + q], tab.Ry[I.bead_off + q]);
        if (ph != 0.0) {
            fx += ph * tab.Gx[I.bead_off + q];
            fy += ph * tab.Gy[I.bead_off + q];
        }
    }
}

template <class S>
__global__ void k_fields(const Inst I, const S *__restrict__ pool, const BeadTab tab, int parity,
                         double *__restrict__ ux, double *__restrict__ uy, double *__restrict__ rho) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    double g[9];
    load_pops<S, double>(pool + I.pop_off, I, x, y, parity, g);
    double dr = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) dr += g[k];
    const double r = 1.0 + dr;
    const double jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    const double jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    double fx, fy;
    overlay_f64(I, tab, x + 0.5, y + 0.5, fx, fy);
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
    load_pops<S, double>(pool + I.pop_off, I, x, y, parity, g);
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k * n + c] = g[k] + ws[k];
}

// Inverse of the parity read: place the deviations of a given state where
// the next step will gather them (bounce-back term removed at the walls).
template <int k, class S>
__device__ __forceinline__ void write_one(S *A, const Inst &I, int x, int y, int parity, double gk) {
    if (parity == 0) {
        Store<S>::st(A + (int64_t)k * I.plane + (int64_t)y * I.pitch + x, (typename Real<S>::type)gk,
                     I.scale[k]);
        return;
    }
    const int ys = y - Q<k>::cy;
    if (ys >= 0 && ys < I.ny) {
        int xs = x - Q<k>::cx;
        xs = (xs < 0) ? xs + I.nx : (xs >= I.nx ? xs - I.nx : xs);
        Store<S>::st(A + (int64_t)Q<k>::opp * I.plane + (int64_t)ys * I.pitch + xs, (typename Real<S>::type)gk,
                     I.scale[Q<k>::opp]);
    } else {
        const double uw = (ys < 0) ? I.u_bot : I.u_top;
        Store<S>::st(A + (int64_t)k * I.plane + (int64_t)y * I.pitch + x,
                     (typename Real<S>::type)(gk - 6.0 * Q<k>::w * Q<k>::cx * uw), I.scale[k]);
    }
}

template <class S>
__global__ void k_write_pops(const Inst I, S *__restrict__ pool, int parity, const double *__restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    S *A = pool + I.pop_off;
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
    write_one<0>(A, I, x, y, parity, f[0 * n + c] - Q<0>::w);
    write_one<1>(A, I, x, y, parity, f[1 * n + c] - Q<1>::w);
    write_one<2>(A, I, x, y, parity, f[2 * n + c] - Q<2>::w);
    write_one<3>(A, I, x, y, parity, f[3 * n + c] - Q<3>::w);
    write_one<4>(A, I, x, y, parity, f[4 * n + c] - Q<4>::w);
    write_one<5>(A, I, x, y, parity, f[5 * n + c] - Q<5>::w);
    write_one<6>(A, I, x, y, parity, f[6 * n + c] - Q<6>::w);
    write_one<7>(A, I, x, y, parity, f[7 * n + c] - Q<7>::w);
    write_one<8>(A, I, x, y, parity, f[8 * n + c] - Q<8>::w);
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
        load_pops<S, double>(pool + I.pop_off, I, x, y, parity, g);
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
template <class S> static cudaError_t lattice_t(const Inst &I, void *pool, BeadTab tab, int parity, cudaStream_t st) {
    dim3 block(kTileX, kTileY);
    dim3 grid((I.nx + kTileX - 1) / kTileX, (I.ny + kTileY - 1) / kTileY);
    k_lattice<S><<<grid, block, 0, st>>>(I, (S *)pool, tab, parity);
    return cudaGetLastError();
}

cudaError_t launch_lattice(int precision, const Inst *, const Inst &inst_h, void *pool, BeadTab tab, int parity,
                           cudaStream_t st) {
    switch (precision) {
        case 0: return lattice_t<double>(inst_h, pool, tab, parity, st);
        case 1: return lattice_t<float>(inst_h, pool, tab, parity, st);
        case 2: return lattice_t<__half>(inst_h, pool, tab, parity, st);
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

cudaError_t launch_fields(int precision, const Inst *, const Inst &I, const void *pool, BeadTab tab, int parity,
                          double *ux, double *uy, double *rho, cudaStream_t st) {
    FPD_DISPATCH(precision,
                 (k_fields<S><<<row_grid(I, 128), 128, 0, st>>>(I, (const S *)pool, tab, parity, ux, uy, rho)));
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
