// fpd_beads.cu -- the bead phase of the FPD step.
//
// One CTA per bead b (any number of instances in one launch):
//   Eq. 5   V_b = sum_x phi_b(x; R_b) u(x) / S_b, with u = (sum_k f_k c_k +
//           f/2) / rho and f the force density of the table that drove the
//           last collision (recomputed from that table, Eq. 4);
//   Sec 2.3 R_b <- R_b + V_b (forward Euler, dt = 1);
//   S_b = sum_x phi_b(x; R_b) at the new position (the discrete int phi_b);
// then the last CTA of an instance to finish (device-wide atomic counter, no
// waiting) computes every bead force of that instance from the new positions:
//   Eq. 11 springs, Eq. 12 bending in its general form (tangents of missing
//   segments are zero, which reproduces the edge cases of Eqs. 12b-12e),
//   plus the excluded-volume repulsion k_ev (d - r) r_hat of non-bonded beads
//   closer than d, and G = F / S for the spreading of Eq. 4; it also writes
//   the FP32 overlay table (positions split hi + lo, G) read by the lattice
//   sweep of the reduced-precision paths.
//
// Arithmetic: positions, velocities, forces and every reduction are FP64.
// In the FP64 (parity) path phi is evaluated in FP64 exactly as a plain IEEE
// evaluation would; in the FP32/FP16-storage paths phi and u are FP32 from
// bead-relative offsets, accumulated in FP64.  Only beads whose support can
// overlap bead b's support are visited per cell.  Reductions use a fixed
// tree so results do not depend on scheduling.
#include <cuda_fp16.h>

#include <type_traits>

#include "fpd_kernels.h"

namespace fpd {

namespace {

constexpr int kWarps = kBeadThreads / 32;

// Deterministic block sum of two doubles; result valid in every thread.
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*sh)[kWarps]) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
    }
    __syncthreads();
    double ta = 0.0, tb = 0.0;
    for (int i = 0; i < kWarps; ++i) {
        ta += sh[0][i];
        tb += sh[1][i];
    }
    a = ta;
    b = tb;
}

// Cells whose centre may lie within the cutoff of (Rx, Ry): a box clipped at
// the walls; in x it wraps periodically, or spans the lattice once.  iu is
// the unwrapped x index of the first column (column c sits at iu + c).
struct Box {
    int i0, j0, w, h;
    double iu;
};
__device__ __forceinline__ Box support_box(const Inst &I, double Rx, double Ry) {
    Box b;
    b.i0 = b.j0 = b.w = b.h = 0;
    b.iu = 0.0;
    // a non-finite or far-away bead has no support cells (the NaN then shows
    // up in the diagnostics, not as an out-of-range index)
    if (!isfinite(Rx) || !isfinite(Ry) || fabs(Rx) > 1.0e9 || fabs(Ry) > 1.0e9) return b;
    const double ylo = fmax(floor(Ry - I.rcut - 0.5) - 1.0, 0.0);
    const double yhi = fmin(ceil(Ry + I.rcut - 0.5) + 1.0, (double)(I.ny - 1));
    if (yhi < ylo) return b;
    double xlo = floor(Rx - I.rcut - 0.5) - 1.0, xhi = ceil(Rx + I.rcut - 0.5) + 1.0;
    if (xhi - xlo + 1.0 >= (double)I.nx) {
        // the support spans the lattice: the nx columns around Rx, once each
        xlo = floor(Rx - 0.5 * I.nx);
        xhi = xlo + I.nx - 1;
    }
    b.iu = xlo;
    b.i0 = (int)(xlo - I.nx * floor(xlo / I.nx));  // in [0, nx)
    b.j0 = (int)ylo;
    b.w = (int)(xhi - xlo) + 1;
    b.h = (int)(yhi - ylo) + 1;
    return b;
}

__device__ __forceinline__ double min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

// Unit tangent of segment k (1-based, joins beads k and k+1 of a fiber whose
// first bead has global index f0) and its length; zero outside 1..N-1.
__device__ __forceinline__ void seg(const double *Rx, const double *Ry, int f0, int N, int k, double &tx,
                                    double &ty, double &L) {
    if (k < 1 || k > N - 1) {
        tx = ty = 0.0;
        L = 1.0;
        return;
    }
    const double dx = __ldcg(Rx + f0 + k) - __ldcg(Rx + f0 + k - 1);
    const double dy = __ldcg(Ry + f0 + k) - __ldcg(Ry + f0 + k - 1);
    L = sqrt(dx * dx + dy * dy);
    tx = dx / L;
    ty = dy / L;
}

// Force on bead q (instance-local index) from the positions in tab.
__device__ void bead_force(const Inst &I, const BeadTab &tab, int q, double &Fx, double &Fy) {
    const int N = I.n_beads;
    const int fib = q / N, i = q % N + 1;  // 1-based index within the fiber
    const int f0 = I.bead_off + fib * N;
    double t_m2x, t_m2y, L_m2, t_m1x, t_m1y, L_m1, t_ix, t_iy, L_i, t_p1x, t_p1y, L_p1;
    seg(tab.Rx, tab.Ry, f0, N, i - 2, t_m2x, t_m2y, L_m2);
    seg(tab.Rx, tab.Ry, f0, N, i - 1, t_m1x, t_m1y, L_m1);
    seg(tab.Rx, tab.Ry, f0, N, i, t_ix, t_iy, L_i);
    seg(tab.Rx, tab.Ry, f0, N, i + 1, t_p1x, t_p1y, L_p1);
    const bool has_m1 = (i - 1 >= 1), has_i = (i <= N - 1);
    const double ks = I.k_s / (I.l0 * I.l0);
    Fx = 0.0;
    Fy = 0.0;
    // Eq. 11 (zero-padded tangents)
    if (has_m1) {
        Fx -= ks * (L_m1 - I.l0) * t_m1x;
        Fy -= ks * (L_m1 - I.l0) * t_m1y;
    }
    if (has_i) {
        Fx += ks * (L_i - I.l0) * t_ix;
        Fy += ks * (L_i - I.l0) * t_iy;
    }
    // Eq. 12: k_b [ (t_i + t_{i-2}).(I - t_{i-1} t_{i-1}) / R_{i-1,i}
    //              - (t_{i+1} + t_{i-1}).(I - t_i t_i) / R_{i,i+1} ]
    if (has_m1) {
        const double vx = t_ix + t_m2x, vy = t_iy + t_m2y;
        const double vt = vx * t_m1x + vy * t_m1y;
        Fx += I.k_b * (vx - vt * t_m1x) / L_m1;
        Fy += I.k_b * (vy - vt * t_m1y) / L_m1;
    }
    if (has_i) {
        const double vx = t_p1x + t_m1x, vy = t_p1y + t_m1y;
        const double vt = vx * t_ix + vy * t_iy;
        Fx -= I.k_b * (vx - vt * t_ix) / L_i;
        Fy -= I.k_b * (vy - vt * t_iy) / L_i;
    }
    // excluded volume between beads that share no spring; an FP32 distance
    // test (1% margin) selects the pairs evaluated in FP64
    if (I.k_ev != 0.0) {
        const double Rqx = __ldcg(tab.Rx + I.bead_off + q), Rqy = __ldcg(tab.Ry + I.bead_off + q);
        const float l0f2 = (float)(I.l0 * I.l0) * 1.0201f;
        for (int p = 0; p < I.nb; ++p) {
            if (p == q) continue;
            if (p / N == fib && abs(p - q) < 2) continue;
            double dx = Rqx - __ldcg(tab.Rx + I.bead_off + p);
            const double dy = Rqy - __ldcg(tab.Ry + I.bead_off + p);
            dx = min_image(dx, (double)I.nx);
            const float fx = (float)dx, fy = (float)dy;
            if (fx * fx + fy * fy >= l0f2) continue;
            const double r = sqrt(dx * dx + dy * dy);
            if (r < I.l0 && r > 0.0) {
                const double m = I.k_ev * (I.l0 - r) / r;
                Fx += m * dx;
                Fy += m * dy;
            }
        }
    }
}

template <class S>
__global__ void __launch_bounds__(kBeadThreads)
    k_beads(const Inst *__restrict__ insts, const int *__restrict__ bead_inst, const S *__restrict__ pool,
            const BeadTab told, const BeadTab tnew, int parity, int advance, unsigned *__restrict__ counters) {
    constexpr bool kF64 = std::is_same<S, double>::value;
    __shared__ Inst sI;
    // beads whose support can overlap bead b's: old-table position (FP64
    // path), offset R_b - R_q (FP32 paths) and spreading coefficients G
    __shared__ double s_rx[kMaxBeads], s_ry[kMaxBeads], s_gx[kMaxBeads], s_gy[kMaxBeads];
    __shared__ float s_ox[kMaxBeads], s_oy[kMaxBeads];
    __shared__ double sh[2][kWarps];
    __shared__ int s_last, s_nn;

    const int b = blockIdx.x;
    const int ii = bead_inst ? bead_inst[b] : 0;
    const int tid = threadIdx.x;
    if (tid == 0) sI = insts[ii];
    __syncthreads();
    const Inst &I = sI;
    const S *A = pool + I.pop_off;

    double Rx, Ry;
    if (advance) {
        Rx = told.Rx[b];
        Ry = told.Ry[b];
        if (tid < 32) {
            const double reach = 2.0 * I.rcut + 1e-6;
            const bool all = I.nx < 2.0 * reach + 2.0;  // small lattice: keep every bead
            int n = 0;
            for (int base = 0; base < I.nb; base += 32) {
                const int q = base + tid;
                bool hit = false;
                double qx = 0.0, qy = 0.0;
                if (q < I.nb) {
                    qx = told.Rx[I.bead_off + q];
                    qy = told.Ry[I.bead_off + q];
                    const double dx = min_image(qx - Rx, (double)I.nx), dy = qy - Ry;
                    hit = all || dx * dx + dy * dy < reach * reach;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = n + __popc(m & ((1u << tid) - 1u));
                    s_rx[pos] = qx;
                    s_ry[pos] = qy;
                    s_ox[pos] = (float)min_image(Rx - qx, (double)I.nx);
                    s_oy[pos] = (float)(Ry - qy);
                    s_gx[pos] = told.Gx[I.bead_off + q];
                    s_gy[pos] = told.Gy[I.bead_off + q];
                }
                n += __popc(m);
            }
            if (tid == 0) s_nn = n;
        }
        __syncthreads();
        const int nn = s_nn;
        const Box bx = support_box(I, Rx, Ry);
        // cell centre relative to R_b: (rel0x + column, rel0y + row)
        const float rel0x = (float)(bx.iu + 0.5 - Rx), rel0y = (float)(bx.j0 + 0.5 - Ry);
        const float af = (float)I.a, inv_xi = (float)(1.0 / I.xi), rc2 = (float)I.rcut2;
        const float hnx = 0.5f * (float)I.nx, fnx = (float)I.nx;
        double ax = 0.0, ay = 0.0;
        for (int c = tid; c < bx.w * bx.h; c += blockDim.x) {
            const int cj = c / bx.w, ci = c - cj * bx.w;
            const int j = bx.j0 + cj;
            int i = bx.i0 + ci;
            i = (i >= I.nx) ? i - I.nx : i;
            if (kF64) {
                const double xc = i + 0.5, yc = j + 0.5;
                const double phb = phi_f64(I, xc, yc, Rx, Ry);
                if (phb == 0.0) continue;
                double g[9];
                load_pops<S, double>(A, I, i, j, parity, g);
                double dr = 0.0;
#pragma unroll
                for (int k = 0; k < 9; ++k) dr += g[k];
                const double rho = 1.0 + dr;
                const double jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
                const double jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
                double fx = I.gx, fy = I.gy;
                for (int q = 0; q < nn; ++q) {
                    const double ph = phi_f64(I, xc, yc, s_rx[q], s_ry[q]);
                    if (ph != 0.0) {
                        fx += ph * s_gx[q];
                        fy += ph * s_gy[q];
                    }
                }
                ax += phb * ((jx + 0.5 * fx) / rho);
                ay += phb * ((jy + 0.5 * fy) / rho);
            } else {
                const float dx = rel0x + (float)ci, dy = rel0y + (float)cj;
                const float phb = phi_f32(dx, dy, af, inv_xi, rc2);
                if (phb == 0.0f) continue;
                float g[9];
                load_pops<S, float>(A, I, i, j, parity, g);
                const float rho = 1.0f + (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8]);
                const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
                const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
                float fx = (float)I.gx, fy = (float)I.gy;
                for (int q = 0; q < nn; ++q) {
                    float ddx = dx + s_ox[q];
                    ddx = (ddx > hnx) ? ddx - fnx : ((ddx < -hnx) ? ddx + fnx : ddx);
                    const float ph = phi_f32(ddx, dy + s_oy[q], af, inv_xi, rc2);
                    fx += ph * (float)s_gx[q];
                    fy += ph * (float)s_gy[q];
                }
                const float irho = 1.0f / rho;
                ax += (double)(phb * ((jx + 0.5f * fx) * irho));
                ay += (double)(phb * ((jy + 0.5f * fy) * irho));
            }
        }
        block_sum2(ax, ay, sh);
        const double S_old = told.S[b];
        const double Vx = ax / S_old, Vy = ay / S_old;
        Rx += Vx;
        Ry += Vy;
        if (tid == 0) {
            tnew.Rx[b] = Rx;
            tnew.Ry[b] = Ry;
            tnew.Vx[b] = Vx;
            tnew.Vy[b] = Vy;
        }
    } else {
        Rx = tnew.Rx[b];
        Ry = tnew.Ry[b];
    }

    // S_b = sum_x phi_b at the new position
    {
        const Box bx = support_box(I, Rx, Ry);
        const float rel0x = (float)(bx.iu + 0.5 - Rx), rel0y = (float)(bx.j0 + 0.5 - Ry);
        const float af = (float)I.a, inv_xi = (float)(1.0 / I.xi), rc2 = (float)I.rcut2;
        double s = 0.0, dummy = 0.0;
        for (int c = tid; c < bx.w * bx.h; c += blockDim.x) {
            const int cj = c / bx.w, ci = c - cj * bx.w;
            if (kF64) {
                int i = bx.i0 + ci;
                i = (i >= I.nx) ? i - I.nx : i;
                s += phi_f64(I, i + 0.5, bx.j0 + cj + 0.5, Rx, Ry);
            } else {
                s += (double)phi_f32(rel0x + (float)ci, rel0y + (float)cj, af, inv_xi, rc2);
            }
        }
        block_sum2(s, dummy, sh);
        if (tid == 0) tnew.S[b] = s;
    }

    // the last CTA of this instance computes the forces of all its beads
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(&counters[ii], 1u);
        s_last = (prev == (unsigned)(I.nb - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int q = tid; q < I.nb; q += blockDim.x) {
        double Fx, Fy;
        bead_force(I, tnew, q, Fx, Fy);
        const int gq = I.bead_off + q;
        const double Sq = __ldcg(tnew.S + gq);
        const double Gx = Fx / Sq, Gy = Fy / Sq;
        tnew.Fx[gq] = Fx;
        tnew.Fy[gq] = Fy;
        tnew.Gx[gq] = Gx;
        tnew.Gy[gq] = Gy;
        // FP32 overlay table: x wrapped into [0, nx), split into hi + lo
        const double rx = __ldcg(tnew.Rx + gq);
        const double xw = rx - I.nx * floor(rx / I.nx);
        const double yw = __ldcg(tnew.Ry + gq);
        const float xh = (float)xw, yh = (float)yw;
        tnew.xh[gq] = xh;
        tnew.xl[gq] = (float)(xw - (double)xh);
        tnew.yh[gq] = yh;
        tnew.yl[gq] = (float)(yw - (double)yh);
        tnew.gxf[gq] = (float)Gx;
        tnew.gyf[gq] = (float)Gy;
    }
    if (tid == 0) counters[ii] = 0u;
}

}  // namespace

cudaError_t launch_beads(int precision, const Inst *inst_d, const int *bead_inst, int nb_total, const void *pool,
                         BeadTab tab_old, BeadTab tab_new, int parity, int advance, unsigned *counters,
                         cudaStream_t st) {
    if (nb_total <= 0) return cudaSuccess;
    switch (precision) {
        case 0:
            k_beads<double><<<nb_total, kBeadThreads, 0, st>>>(inst_d, bead_inst, (const double *)pool, tab_old,
                                                              tab_new, parity, advance, counters);
            break;
        case 1:
            k_beads<float><<<nb_total, kBeadThreads, 0, st>>>(inst_d, bead_inst, (const float *)pool, tab_old,
                                                             tab_new, parity, advance, counters);
            break;
        case 2:
            k_beads<__half><<<nb_total, kBeadThreads, 0, st>>>(inst_d, bead_inst, (const __half *)pool, tab_old,
                                                              tab_new, parity, advance, counters);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fpd
