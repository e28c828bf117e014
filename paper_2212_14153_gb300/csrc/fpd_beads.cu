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
// Arithmetic: positions, velocities, forces and the reductions over the
// support are FP64.  In the FP64 (parity) path phi is evaluated in FP64
// exactly as a plain IEEE evaluation would; in the FP32/FP16-storage paths
// phi and u are FP32 from bead-relative offsets, each of 256 virtual lanes
// adds its few support cells (ceil(cells / 256), 3 for a = 4, xi = 1) in
// FP32 and the lanes are reduced to FP64.  FP64 instructions are kept out of
// per-cell work: this GPU issues one FP64 warp instruction per ~16 cycles
// per SM.  Only beads whose support can overlap bead b's support are visited
// per cell.  Reductions use a fixed tree over the virtual lanes, so results
// depend neither on scheduling nor on the CTA size (256 threads while the
// beads of a launch fit on the SMs one per SM, 128 otherwise).
//
// Chaining: the kernel first waits for the preceding sweep and then lets the
// next sweep launch; that sweep's unmarked tiles run beside this phase, its
// marked tiles wait for it to complete.
#include <cuda_fp16.h>

#include <atomic>
#include <type_traits>

#include "fpd_kernels.h"

namespace fpd {

namespace {

// The per-bead sums over the support (Eqs. 4-5) are taken over kBeadLanes
// virtual lanes whatever the CTA size NT: lane v adds the cells v, v +
// kBeadLanes, ... in that order, thread t holds lanes t and t + NT (when NT <
// kBeadLanes), and the lanes are reduced in one fixed tree.  A bead therefore
// gives the same bits in a CTA of either size (a batch may use the other
// size than the instance alone).
constexpr int kLaneGroups = kBeadLanes / 32;

// Sum of two doubles over the virtual lanes; partial j of this thread
// belongs to lane threadIdx.x + j NT.  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ void lanes_sum2_to0(double a0, double b0, double a1, double b1, double &ra, double &rb,
                                               double (*sh)[kLaneGroups]) {
    constexpr int L = kBeadLanes / NT;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < L; ++j) {
        double a = j ? a1 : a0, b = j ? b1 : b0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (l == 0) {
            sh[0][w + j * (NT / 32)] = a;
            sh[1][w + j * (NT / 32)] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < kLaneGroups; ++i) {
            ta += sh[0][i];
            tb += sh[1][i];
        }
        ra = ta;
        rb = tb;
    }
}

// Error-free sum of two floats (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The same for FP32 partials, with FP64-level accuracy: compensated (hi, lo)
// float pairs inside each group of 32 lanes, FP64 for the final value.  The
// FP64 pipe of this GPU issues a warp instruction only every few tens of
// cycles, so FP64 is kept to the last step.  Result valid in thread 0.
template <int NT>
__device__ __forceinline__ void lanes_sum2f_to0(float a0, float b0, float a1, float b1, double &ra, double &rb,
                                                double (*sh)[kLaneGroups]) {
    constexpr int L = kBeadLanes / NT;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    float *shf = (float *)sh;  // 4 floats a group fit in its 2 doubles
    __syncthreads();
#pragma unroll
    for (int j = 0; j < L; ++j) {
        float ah = j ? a1 : a0, al = 0.f, bh = j ? b1 : b0, bl = 0.f;
        for (int o = 16; o > 0; o >>= 1) {
            const float oah = __shfl_down_sync(0xffffffffu, ah, o), oal = __shfl_down_sync(0xffffffffu, al, o);
            const float obh = __shfl_down_sync(0xffffffffu, bh, o), obl = __shfl_down_sync(0xffffffffu, bl, o);
            float s, e;
            two_sum(ah, oah, s, e);
            e += al + oal;
            two_sum(s, e, ah, al);
            two_sum(bh, obh, s, e);
            e += bl + obl;
            two_sum(s, e, bh, bl);
        }
        if (l == 0) {
            const int g = w + j * (NT / 32);
            shf[4 * g + 0] = ah;
            shf[4 * g + 1] = al;
            shf[4 * g + 2] = bh;
            shf[4 * g + 3] = bl;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float th = shf[0], tl = shf[1], uh = shf[2], ul = shf[3];
        for (int i = 1; i < kLaneGroups; ++i) {
            float s, e;
            two_sum(th, shf[4 * i], s, e);
            e += tl + shf[4 * i + 1];
            two_sum(s, e, th, tl);
            two_sum(uh, shf[4 * i + 2], s, e);
            e += ul + shf[4 * i + 3];
            two_sum(s, e, uh, ul);
        }
        ra = (double)th + (double)tl;
        rb = (double)uh + (double)ul;
    }
}

// d reduced to its nearest periodic image (period L = nx, or ny): the image
// index is found in FP32 (it is an integer) and removed exactly in FP64.
__device__ __forceinline__ double min_image(double d, int nx, float inv_nx) {
    const float k = rintf((float)d * inv_nx);
    return d - (double)k * (double)nx;
}
// A box widened by one cell on every side: wrapped (x, and y when periodic),
// clipped at the walls, covering each direction at most once.
__device__ __forceinline__ Box widen_box(const Inst &I, Box b) {
    if (b.w <= 0 || b.h <= 0) return b;
    if (b.w < I.nx) {
        b.i0 = (b.i0 == 0) ? I.nx - 1 : b.i0 - 1;
        b.w = (b.w + 2 < I.nx) ? b.w + 2 : I.nx;
    }
    if (I.periodic_y) {
        if (b.h < I.ny) {
            b.j0 = (b.j0 == 0) ? I.ny - 1 : b.j0 - 1;
            b.h = (b.h + 2 < I.ny) ? b.h + 2 : I.ny;
        }
    } else {
        const int lo = b.j0 > 0 ? b.j0 - 1 : 0;
        const int hi = (b.j0 + b.h < I.ny) ? b.j0 + b.h : I.ny - 1;
        b.j0 = lo;
        b.h = hi - lo + 1;
    }
    return b;
}

// the same for the y separation, applied only when y is periodic
__device__ __forceinline__ double min_image_y(const Inst &I, double d) {
    return I.periodic_y ? min_image(d, I.ny, I.f_inv_ny) : d;
}
__device__ __forceinline__ float min_image_yf(const Inst &I, float d) {
    return I.periodic_y ? d - (float)I.ny * rintf(d * I.f_inv_ny) : d;
}

// Force on bead q (instance-local index), given the instance's positions
// and the unit tangents/lengths of every segment (index j joins beads j and
// j+1 of the instance-local numbering), all staged in shared memory.
__device__ __forceinline__ void bead_force(const Inst &I, const double *Rx, const double *Ry, const float *Xf,
                                           const float *Yf, const double *Tx, const double *Ty, const double *Ln, int q,
                                           double &Fx, double &Fy) {
    const int N = I.n_beads;
    const int fib = q / N, i0 = q - fib * N;  // 0-based index within the fiber
    // segments around bead q, as in Eqs. 11-12 with 1-based i = i0 + 1:
    // t_{i-2}, t_{i-1} (ends at q), t_i (starts at q), t_{i+1}; missing = 0
    const bool h_m2 = i0 >= 2, h_m1 = i0 >= 1, h_i = i0 <= N - 2, h_p1 = i0 + 1 <= N - 2;
    const double tm2x = h_m2 ? Tx[q - 2] : 0.0, tm2y = h_m2 ? Ty[q - 2] : 0.0;
    const double tm1x = h_m1 ? Tx[q - 1] : 0.0, tm1y = h_m1 ? Ty[q - 1] : 0.0;
    const double tix = h_i ? Tx[q] : 0.0, tiy = h_i ? Ty[q] : 0.0;
    const double tp1x = h_p1 ? Tx[q + 1] : 0.0, tp1y = h_p1 ? Ty[q + 1] : 0.0;
    const double ks = I.ks_l02;
    Fx = 0.0;
    Fy = 0.0;
    if (h_m1) {
        const double Lm1 = Ln[q - 1];
        // Eq. 11, spring to the previous bead
        Fx -= ks * (Lm1 - I.l0) * tm1x;
        Fy -= ks * (Lm1 - I.l0) * tm1y;
        // Eq. 12, first term: (t_i + t_{i-2}).(I - t_{i-1} t_{i-1}) / R_{i-1,i}
        const double vx = tix + tm2x, vy = tiy + tm2y;
        const double vt = vx * tm1x + vy * tm1y;
        Fx += I.k_b * (vx - vt * tm1x) / Lm1;
        Fy += I.k_b * (vy - vt * tm1y) / Lm1;
    }
    if (h_i) {
        const double Li = Ln[q];
        // Eq. 11, spring to the next bead
        Fx += ks * (Li - I.l0) * tix;
        Fy += ks * (Li - I.l0) * tiy;
        // Eq. 12, second term: -(t_{i+1} + t_{i-1}).(I - t_i t_i) / R_{i,i+1}
        const double vx = tp1x + tm1x, vy = tp1y + tm1y;
        const double vt = vx * tix + vy * tiy;
        Fx -= I.k_b * (vx - vt * tix) / Li;
        Fy -= I.k_b * (vy - vt * tiy) / Li;
    }
    // excluded volume between beads that share no spring; an FP32 distance
    // test (1% margin) selects the pairs evaluated in FP64
    if (I.k_ev != 0.0) {
        const double Rqx = Rx[q], Rqy = Ry[q];
        const float l0f2 = (float)(I.l0 * I.l0) * 1.0201f;
        const float fnx = (float)I.nx;
        const float xq = Xf[q], yq = Yf[q];
        const int lo = fib * N;
        for (int p = 0; p < I.nb; ++p) {
            float fx = xq - Xf[p];
            fx -= fnx * rintf(fx * I.f_inv_nx);
            const float fy = min_image_yf(I, yq - Yf[p]);
            if (fx * fx + fy * fy >= l0f2) continue;
            if (p == q || (p >= lo && p < lo + N && abs(p - q) < 2)) continue;
            const double dx = min_image(Rqx - Rx[p], I.nx, I.f_inv_nx);
            const double dy = min_image_y(I, Rqy - Ry[p]);
            const double r = sqrt(dx * dx + dy * dy);
            if (r < I.l0 && r > 0.0) {
                const double m = I.k_ev * (I.l0 - r) / r;
                Fx += m * dx;
                Fy += m * dy;
            }
        }
    }
    // constant external force F_0 (driven particle, Sec. 3.2)
    Fx += I.ext_fx;
    Fy += I.ext_fy;
}

// FP32 version of bead_force for the reduced-precision paths.  Positions
// stay FP64; each segment's tangent and length are FP32, and its stretch
// L - l0 = (|d|^2 - l0^2) / (L + l0) is formed from the FP64 |d|^2 so that
// the small strain of a stiff spring does not cancel away in FP32.
__device__ __forceinline__ void bead_force_f32(const Inst &I, const double *Rx, const double *Ry, const float *Xf,
                                               const float *Yf, const float *Tx, const float *Ty, const float *Ln,
                                               const float *Dl, int q, float &Fx, float &Fy) {
    // the record's fields in registers, the force in local accumulators:
    // with stores through Fx, Fy inside the loop the fields would be
    // reloaded from the shared record on every pass
    const int N = I.n_beads, nb = I.nb, nx = I.nx, ny = I.ny;
    const bool py = I.periodic_y != 0;
    const float inv_nx = I.f_inv_nx, inv_ny = I.f_inv_ny, fnx = (float)nx, fny = (float)ny;
    const int fib = q / N, i0 = q - fib * N;
    const bool h_m2 = i0 >= 2, h_m1 = i0 >= 1, h_i = i0 <= N - 2, h_p1 = i0 + 1 <= N - 2;
    const float tm2x = h_m2 ? Tx[q - 2] : 0.f, tm2y = h_m2 ? Ty[q - 2] : 0.f;
    const float tm1x = h_m1 ? Tx[q - 1] : 0.f, tm1y = h_m1 ? Ty[q - 1] : 0.f;
    const float tix = h_i ? Tx[q] : 0.f, tiy = h_i ? Ty[q] : 0.f;
    const float tp1x = h_p1 ? Tx[q + 1] : 0.f, tp1y = h_p1 ? Ty[q + 1] : 0.f;
    const float ks = I.f_ks_l02, kb = I.f_kb;
    float ax = 0.f, ay = 0.f;
    if (h_m1) {
        const float Lm1 = Ln[q - 1], dl = Dl[q - 1];
        ax -= ks * dl * tm1x;
        ay -= ks * dl * tm1y;
        const float vx = tix + tm2x, vy = tiy + tm2y;
        const float vt = vx * tm1x + vy * tm1y;
        ax += kb * (vx - vt * tm1x) / Lm1;
        ay += kb * (vy - vt * tm1y) / Lm1;
    }
    if (h_i) {
        const float Li = Ln[q], dl = Dl[q];
        ax += ks * dl * tix;
        ay += ks * dl * tiy;
        const float vx = tp1x + tm1x, vy = tp1y + tm1y;
        const float vt = vx * tix + vy * tiy;
        ax -= kb * (vx - vt * tix) / Li;
        ay -= kb * (vy - vt * tiy) / Li;
    }
    if (I.k_ev != 0.0) {
        // Xf, Yf: positions relative to bead 0 of the instance in FP32 (a
        // screen with 1% margin); a candidate pair is evaluated from the
        // FP64 positions
        const float l0 = I.f_l0, l0s2 = l0 * l0 * 1.0201f, kev = I.f_kev;
        const float xq = Xf[q], yq = Yf[q];
        const double Rqx = Rx[q], Rqy = Ry[q];
        const int lo = fib * N;
        // screen 32 beads at a time without branches (independent passes
        // the compiler can overlap), then evaluate the few candidates in
        // bead order
        for (int p0 = 0; p0 < nb; p0 += 32) {
            const int pn = min(32, nb - p0);
            unsigned cand = 0u;
#pragma unroll 8
            for (int k = 0; k < pn; ++k) {
                const int p = p0 + k;
                float fx = xq - Xf[p];
                fx -= fnx * rintf(fx * inv_nx);
                float fy = yq - Yf[p];
                if (py) fy -= fny * rintf(fy * inv_ny);
                const bool bonded = p == q || (p >= lo && p < lo + N && abs(p - q) < 2);
                cand |= (unsigned)(fx * fx + fy * fy < l0s2 && !bonded) << k;
            }
            while (cand) {
                const int p = p0 + __ffs(cand) - 1;
                cand &= cand - 1u;
                const double dx = min_image(Rqx - Rx[p], nx, inv_nx);
                const double dy = py ? min_image(Rqy - Ry[p], ny, inv_ny) : Rqy - Ry[p];
                const float r = sqrtf((float)(dx * dx + dy * dy));
                if (r < l0 && r > 0.f) {
                    const float m = kev * (l0 - r) / r;
                    ax += m * (float)dx;
                    ay += m * (float)dy;
                }
            }
        }
    }
    Fx = ax + I.f_ext_fx;
    Fy = ay + I.f_ext_fy;
}

// CTA c handles beads c, c + gridDim.x, ... of the list, so any grid size
// covers every bead; the launcher gives each bead its own CTA.
// Resident bead CTAs per SM the reduced-precision kernels are held to (80
// registers a thread), so that large bead lists of a batch run in few waves;
// the FP64 parity path keeps its registers.
template <class S, int NT> struct BeadMinBlocks { static constexpr int value = 6 * kBeadThreads / NT; };
template <int NT> struct BeadMinBlocks<double, NT> { static constexpr int value = 1; };

// NT threads per bead CTA: kBeadThreads for long bead lists (more CTAs
// resident), kBeadThreadsFew when every bead has an SM of its own (shorter
// per-bead loops).
template <class S, int NT>
__global__ void __launch_bounds__(NT, BeadMinBlocks<S, NT>::value)
    k_beads(const Inst *__restrict__ insts, const int2 *__restrict__ blist, const int nb_total,
            const S *__restrict__ pool, const BeadTab tab0, const BeadTab tab1, unsigned *__restrict__ mask_write,
            int gparity, int advance, unsigned *__restrict__ counters, BeadExport ex,
            unsigned *__restrict__ status) {
    constexpr bool kF64 = std::is_same<S, double>::value;
    __shared__ Inst sI;
    // neighbour beads: old-table position (FP64 path), offset R_b - R_q and
    // spreading coefficients (FP32 paths); reused by the last CTA to stage
    // positions, support sums and segment tangents
    __shared__ double s_rx[kMaxBeads], s_ry[kMaxBeads], s_gx[kMaxBeads], s_gy[kMaxBeads];
    __shared__ double s_tx[kMaxBeads], s_ty[kMaxBeads], s_ln[kMaxBeads];
    __shared__ float s_ox[kMaxBeads], s_oy[kMaxBeads], s_gxf[kMaxBeads], s_gyf[kMaxBeads];
    __shared__ float s_xf[kMaxBeads], s_yf[kMaxBeads];
    constexpr int kWarps = NT / 32;
    __shared__ double sh[2][kLaneGroups];
    // virtual lanes a thread holds (partials 0 and 1: lanes tid, tid + NT)
    constexpr int kL = kBeadLanes / NT;
    __shared__ double s_R[2];
    __shared__ float s_rel[2];
    __shared__ Box s_box;
    __shared__ double s_invS;
    __shared__ unsigned s_hits[kMaxBeads / 32];
    __shared__ int s_last, s_nn;
    __shared__ unsigned s_stold;

    // wait for the preceding sweep (the populations read below, and through
    // it the previous bead phase), then let the next sweep launch at once:
    // its tiles that no bead marked start while this phase runs, and the
    // set-up below (record copy, neighbour screen) does not delay them
    pdl_wait();
    pdl_trigger();
    for (int it = blockIdx.x; it < nb_total; it += gridDim.x) {
    __syncthreads();  // the shared state of the previous bead is no longer read
    // blist[i] = (instance slot, global bead index); NULL: instance 0, bead i
    const int2 bi = blist ? blist[it] : make_int2(0, it);
    const int ii = bi.x, b = bi.y;
    const int tid = threadIdx.x;
    // this instance's step parity selects the table pair and the population
    // buffer; it is read from the global record so that the old table's
    // loads below need not wait for the shared copy
    const int parity = gparity ^ insts[ii].par_xor;
    const BeadTab &told = parity ? tab0 : tab1;
    const BeadTab &tnew = parity ? tab1 : tab0;
    {
        // cooperative copy of the instance record (one 32-bit word a thread)
        static_assert(sizeof(Inst) % 4 == 0, "Inst is copied as 32-bit words");
        const unsigned *src = (const unsigned *)(insts + ii);
        unsigned *dst = (unsigned *)&sI;
        for (int wd = tid; wd < (int)(sizeof(Inst) / 4); wd += blockDim.x) dst[wd] = src[wd];
    }
    // the bead's old position (every thread) and support sum
    double Rx = 0.0, Ry = 0.0, S_old = 1.0;
    if (advance) {
        Rx = told.Rx[b];
        Ry = told.Ry[b];
        if (tid == 0) S_old = told.S[b];
    }
    __syncthreads();
    const Inst &I = sI;
    // populations are pulled from the current buffer (the instance's parity)
    const S *A = pop_buffer(pool, I, parity);

    if (advance) {
        if (tid == 0) {
            const Box bx = support_box(I, Rx, Ry);
            s_box = bx;
            s_rel[0] = (float)(bx.iu + 0.5 - Rx);
            s_rel[1] = (float)(bx.ju + 0.5 - Ry);
            s_invS = 1.0 / S_old;
        }
        {
            // beads whose support can overlap b's (FP32 screen, 1-cell
            // margin), listed in bead order: warp w screens the 32-bead
            // chunks w, w + kWarps, ...; a chunk's hit mask places its hits
            // after those of the chunks before it
            const float reach = 2.0f * I.f_rcut + 1.0f, fnx = (float)I.nx;
            const int lane = tid & 31, w = tid >> 5;
            const int nchunks = (I.nb + 31) / 32;
            int n = 0;
            for (int r0 = 0; r0 < nchunks; r0 += kWarps) {
                const int c = r0 + w, q = 32 * c + lane;
                bool hit = false;
                double qx = 0.0, qy = 0.0, gx = 0.0, gy = 0.0;
                if (q < I.nb) {
                    qx = told.Rx[I.bead_off + q];
                    qy = told.Ry[I.bead_off + q];
                    gx = told.Gx[I.bead_off + q];
                    gy = told.Gy[I.bead_off + q];
                    float dx = (float)(qx - Rx);
                    dx -= fnx * rintf(dx * I.f_inv_nx);
                    const float dy = min_image_yf(I, (float)(qy - Ry));
                    hit = dx * dx + dy * dy < reach * reach;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (lane == 0 && c < nchunks) s_hits[c] = m;
                __syncthreads();
                if (hit) {
                    int pos = n + __popc(m & ((1u << lane) - 1u));
                    for (int cc = r0; cc < c; ++cc) pos += __popc(s_hits[cc]);
                    s_rx[pos] = qx;
                    s_ry[pos] = qy;
                    s_ox[pos] = (float)min_image(Rx - qx, I.nx, I.f_inv_nx);
                    s_oy[pos] = (float)min_image_y(I, Ry - qy);
                    s_gx[pos] = gx;
                    s_gy[pos] = gy;
                    s_gxf[pos] = (float)gx;
                    s_gyf[pos] = (float)gy;
                }
                for (int cc = r0; cc < r0 + kWarps && cc < nchunks; ++cc) n += __popc(s_hits[cc]);
                __syncthreads();  // s_hits is rewritten by the next round
            }
            if (tid == 0) s_nn = n;
        }
        __syncthreads();
        const int nn = s_nn;
        const Box bx = s_box;
        const float rel0x = s_rel[0], rel0y = s_rel[1];
        const float hnx = 0.5f * (float)I.nx, fnx = (float)I.nx;
        const float hny = 0.5f * (float)I.ny, fny = (float)I.ny;
        // per-lane partials (FP32 paths: few terms a lane); cell c belongs
        // to partial (c / NT) % kL of its thread
        double ax0 = 0.0, ay0 = 0.0, ax1 = 0.0, ay1 = 0.0;
        float axf0 = 0.0f, ayf0 = 0.0f, axf1 = 0.0f, ayf1 = 0.0f;
        // the box row and column of box cell c, wrapped into the lattice
        auto cell_ij = [&](int c, int &ci, int &cj, int &i, int &j) {
            cj = c / bx.w;
            ci = c - cj * bx.w;
            j = bx.j0 + cj;
            j = (j >= I.ny) ? j - I.ny : j;
            i = bx.i0 + ci;
            i = (i >= I.nx) ? i - I.nx : i;
        };
        if constexpr (kF64) {
            for (int c = tid; c < bx.w * bx.h; c += blockDim.x) {
                int ci, cj, i, j;
                cell_ij(c, ci, cj, i, j);
                const double xc = i + 0.5, yc = j + 0.5;
                const double phb = phi_f64(I, xc, yc, Rx, Ry);
                if (phb == 0.0) continue;
                double g[9];
                pull_pops<S, double>(A, I, make_cell(I, i, j), g);
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
                if ((c / NT) % kL) {
                    ax1 += phb * ((jx + 0.5 * fx) / rho);
                    ay1 += phb * ((jy + 0.5 * fy) / rho);
                } else {
                    ax0 += phb * ((jx + 0.5 * fx) / rho);
                    ay0 += phb * ((jy + 0.5 * fy) / rho);
                }
            }
        } else {
            // each thread visits its cells c = tid, tid + blockDim.x, ...
            // with phi_b != 0, loading the populations of the next such cell
            // before it works on the current one
            const int ncell = bx.w * bx.h;
            auto seek = [&](int &c, float &dx, float &dy, float &phb) {
                for (; c < ncell; c += blockDim.x) {
                    const int cj = c / bx.w, ci = c - cj * bx.w;
                    dx = rel0x + (float)ci;
                    dy = rel0y + (float)cj;
                    phb = phi_f32(dx, dy, I.f_a, I.f_inv_xi, I.f_rcut2);
                    if (phb != 0.0f) return;
                }
            };
            auto load = [&](int c, float g[9]) {
                int ci, cj, i, j;
                cell_ij(c, ci, cj, i, j);
                pull_pops<S, float>(A, I, make_cell(I, i, j), g);
            };
            int c = tid;
            float dx = 0.f, dy = 0.f, phb = 0.f, g[9];
            seek(c, dx, dy, phb);
            if (c < ncell) load(c, g);
            while (c < ncell) {
                int cn = c + blockDim.x;
                float dxn = 0.f, dyn = 0.f, phn = 0.f, gn[9];
                seek(cn, dxn, dyn, phn);
                if (cn < ncell) load(cn, gn);
                const float rho = 1.0f + (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8]);
                const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
                const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
                float fx = I.f_gx, fy = I.f_gy;
                for (int q = 0; q < nn; ++q) {
                    float ddx = dx + s_ox[q];
                    ddx = (ddx > hnx) ? ddx - fnx : ((ddx < -hnx) ? ddx + fnx : ddx);
                    float ddy = dy + s_oy[q];
                    if (I.periodic_y) ddy = (ddy > hny) ? ddy - fny : ((ddy < -hny) ? ddy + fny : ddy);
                    const float ph = phi_f32(ddx, ddy, I.f_a, I.f_inv_xi, I.f_rcut2);
                    fx += ph * s_gxf[q];
                    fy += ph * s_gyf[q];
                }
                const float irho = 1.0f / rho;
                if ((c / NT) % kL) {
                    axf1 += phb * ((jx + 0.5f * fx) * irho);
                    ayf1 += phb * ((jy + 0.5f * fy) * irho);
                } else {
                    axf0 += phb * ((jx + 0.5f * fx) * irho);
                    ayf0 += phb * ((jy + 0.5f * fy) * irho);
                }
                c = cn;
                dx = dxn;
                dy = dyn;
                phb = phn;
                if (cn < ncell) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) g[k] = gn[k];
                }
            }
        }
        double ax = 0.0, ay = 0.0;
        if constexpr (kF64) lanes_sum2_to0<NT>(ax0, ay0, ax1, ay1, ax, ay, sh);
        else lanes_sum2f_to0<NT>(axf0, ayf0, axf1, ayf1, ax, ay, sh);
        if (tid == 0) {
            const double inv_S = s_invS;
            const double Vx = ax * inv_S, Vy = ay * inv_S;
            const double Rnx = Rx + Vx, Rny = Ry + Vy;
            tnew.Rx[b] = Rnx;
            tnew.Ry[b] = Rny;
            tnew.Vx[b] = Vx;
            tnew.Vy[b] = Vy;
            const Box nb_ = support_box(I, Rnx, Rny);
            s_R[0] = Rnx;
            s_R[1] = Rny;
            s_box = nb_;
            s_rel[0] = (float)(nb_.iu + 0.5 - Rnx);
            s_rel[1] = (float)(nb_.ju + 0.5 - Rny);
        }
    } else if (tid == 0) {
        const double Rx = tnew.Rx[b], Ry = tnew.Ry[b];
        const Box bx = support_box(I, Rx, Ry);
        s_R[0] = Rx;
        s_R[1] = Ry;
        s_box = bx;
        s_rel[0] = (float)(bx.iu + 0.5 - Rx);
        s_rel[1] = (float)(bx.ju + 0.5 - Ry);
    }
    __syncthreads();

    // mark bead b in the mask of every lattice tile its support box, widened
    // by one cell, reaches (one atomicOr per tile row and tile column the box
    // starts in); the widening covers the bead's move in the next step, so
    // the next sweep may update unmarked tiles before its bead phase ends
    {
        const Box bx = widen_box(I, s_box);
        const int lb = b - I.bead_off;
        const unsigned bit = 1u << (lb & 31);
        if (!I.periodic_y) {
            const int tr0 = bx.j0 / kTileY;
            const int nrows = bx.h > 0 ? (bx.j0 + bx.h - 1) / kTileY - tr0 + 1 : 0;
            for (int t = tid; t < nrows * bx.w; t += blockDim.x) {
                const int r = tr0 + t / bx.w, ci = t - (t / bx.w) * bx.w;
                int col = bx.i0 + ci;
                col = (col >= I.nx) ? col - I.nx : col;
                if (ci != 0 && (col % kTileX) != 0) continue;
                const int tile = I.tile_base + r * I.ntx + col / kTileX;
                atomicOr(mask_write + tile * I.mask_words + (lb >> 5), bit);
            }
        } else {
            // rows wrap: visit each cell of the box that starts a tile row or
            // column inside the box
            for (int t = tid; t < bx.h * bx.w; t += blockDim.x) {
                const int cj = t / bx.w, ci = t - cj * bx.w;
                int row = bx.j0 + cj;
                row = (row >= I.ny) ? row - I.ny : row;
                int col = bx.i0 + ci;
                col = (col >= I.nx) ? col - I.nx : col;
                if ((cj != 0 && (row % kTileY) != 0) || (ci != 0 && (col % kTileX) != 0)) continue;
                const int tile = I.tile_base + (row / kTileY) * I.ntx + col / kTileX;
                atomicOr(mask_write + tile * I.mask_words + (lb >> 5), bit);
            }
        }
    }

    // S_b = sum_x phi_b at the new position
    {
        const double Rx = s_R[0], Ry = s_R[1];
        const Box bx = s_box;
        const float rel0x = s_rel[0], rel0y = s_rel[1];
        double acc0 = 0.0, acc1 = 0.0, acc = 0.0, dummy = 0.0;
        float part0 = 0.0f, part1 = 0.0f;
        for (int c = tid; c < bx.w * bx.h; c += blockDim.x) {
            const int cj = c / bx.w, ci = c - cj * bx.w;
            const bool hi = (c / NT) % kL != 0;  // the thread's second lane
            if constexpr (kF64) {
                int i = bx.i0 + ci;
                i = (i >= I.nx) ? i - I.nx : i;
                int j = bx.j0 + cj;
                j = (j >= I.ny) ? j - I.ny : j;
                const double ph = phi_f64(I, i + 0.5, j + 0.5, Rx, Ry);
                if (hi) acc1 += ph;
                else acc0 += ph;
            } else {
                // each lane sums at most a few terms in FP32 before the
                // FP64-level reduction
                const float ph = phi_f32(rel0x + (float)ci, rel0y + (float)cj, I.f_a, I.f_inv_xi, I.f_rcut2);
                if (hi) part1 += ph;
                else part0 += ph;
            }
        }
        if constexpr (kF64) lanes_sum2_to0<NT>(acc0, 0.0, acc1, 0.0, acc, dummy, sh);
        else lanes_sum2f_to0<NT>(part0, 0.0f, part1, 0.0f, acc, dummy, sh);
        if (tid == 0) tnew.S[b] = acc;
    }

    // the last CTA of this instance computes the forces of all its beads
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(&counters[ii], 1u);
        s_last = (prev == (unsigned)(I.nb - 1));
    }
    __syncthreads();
    if (s_last) {
    __threadfence();
    // this phase's export number (the previous phase wrote the counter)
    const unsigned long long ex_k = ex.ring ? *(volatile unsigned long long *)ex.count : 0ull;
    // the instance's status bits as earlier phases left them
    if (tid == 0) s_stold = (status && advance) ? __ldcg(status + ii) : 0u;
    // stage the instance's new positions and support sums (written by every
    // CTA; the L2-coherent loads see them), then every segment once.  The
    // fast-bead guard below tests this phase's velocities: they are loaded in
    // the same round of loads, so that the guard adds no memory round trip
    // to the phase's last CTA
    const bool guard = status && advance;
    bool fast = false, bad = false;
    for (int q = tid; q < I.nb; q += blockDim.x) {
        s_rx[q] = __ldcg(tnew.Rx + I.bead_off + q);
        s_ry[q] = __ldcg(tnew.Ry + I.bead_off + q);
        s_gx[q] = __ldcg(tnew.S + I.bead_off + q);
        if (guard) {
            const double vx = __ldcg(tnew.Vx + I.bead_off + q), vy = __ldcg(tnew.Vy + I.bead_off + q);
            fast |= !(fabs(vx) < kFastBead && fabs(vy) < kFastBead);
            bad |= !(isfinite(vx) && isfinite(vy));
        }
    }
    __syncthreads();
    // fast-bead guard: the early update of unmarked tiles assumes a bead
    // moves less than a cell per step.  When one of this phase's velocities
    // reaches kFastBead per component (or is not finite), flag the instance;
    // while the flag is set, mark every tile of the instance (bead 0's bit)
    // in this phase's masks, so that the next sweeps wait on all of them
    if (guard) {
        const int any_fast = __syncthreads_or(fast);
        const int any_bad = __syncthreads_or(bad);
        if (any_fast && tid == 0) atomicOr(status + ii, kFlagFastBead | (any_bad ? kFlagNonFinite : 0u));
        if (any_fast || (s_stold & kFlagFastBead))
            for (int t = tid; t < I.ntx * I.nty; t += blockDim.x)
                atomicOr(mask_write + (I.tile_base + t) * I.mask_words, 1u);
    }
    for (int q = tid; q < I.nb; q += blockDim.x) {
        s_xf[q] = (float)(s_rx[q] - s_rx[0]);
        s_yf[q] = (float)(s_ry[q] - s_ry[0]);
    }
    for (int q = tid; q < I.nb; q += blockDim.x) {
        if ((q + 1) % I.n_beads != 0) {
            const double dx = s_rx[q + 1] - s_rx[q], dy = s_ry[q + 1] - s_ry[q];
            if constexpr (kF64) {
                const double L = sqrt(dx * dx + dy * dy);
                const double iL = 1.0 / L;
                s_tx[q] = dx * iL;
                s_ty[q] = dy * iL;
                s_ln[q] = L;
            } else {
                const double d2 = dx * dx + dy * dy;
                const float L = sqrtf((float)d2);
                s_ox[q] = (float)dx / L;                                // tangent x
                s_oy[q] = (float)dy / L;                                // tangent y
                s_gxf[q] = L;                                           // length
                s_gyf[q] = (float)(d2 - I.l0 * I.l0) / (L + I.f_l0);  // L - l0
            }
        }
    }
    __syncthreads();
    for (int q = tid; q < I.nb; q += blockDim.x) {
        double Fx, Fy, Gx, Gy;
        if constexpr (kF64) {
            bead_force(I, s_rx, s_ry, s_xf, s_yf, s_tx, s_ty, s_ln, q, Fx, Fy);
            const double inv_S = 1.0 / s_gx[q];
            Gx = Fx * inv_S;
            Gy = Fy * inv_S;
        } else {
            float fx, fy;
            bead_force_f32(I, s_rx, s_ry, s_xf, s_yf, s_ox, s_oy, s_gxf, s_gyf, q, fx, fy);
            const float inv_S = 1.0f / (float)s_gx[q];
            Fx = fx;
            Fy = fy;
            Gx = fx * inv_S;
            Gy = fy * inv_S;
        }
        const int gq = I.bead_off + q;
        tnew.Fx[gq] = Fx;
        tnew.Fy[gq] = Fy;
        tnew.Gx[gq] = Gx;
        tnew.Gy[gq] = Gy;
        // FP32 overlay table: x (and y when periodic) wrapped into the
        // lattice, split into hi + lo
        const double rx = s_rx[q];
        double xw = rx - (double)floorf((float)rx * I.f_inv_nx) * (double)I.nx;
        xw = (xw < 0.0) ? xw + I.nx : ((xw >= I.nx) ? xw - I.nx : xw);
        double yw = s_ry[q];
        if (I.periodic_y) {
            yw -= (double)floorf((float)yw * I.f_inv_ny) * (double)I.ny;
            yw = (yw < 0.0) ? yw + I.ny : ((yw >= I.ny) ? yw - I.ny : yw);
        }
        const float xh = (float)xw, yh = (float)yw;
        tnew.xh[gq] = xh;
        tnew.xl[gq] = (float)(xw - (double)xh);
        tnew.yh[gq] = yh;
        tnew.yl[gq] = (float)(yw - (double)yh);
        tnew.gxf[gq] = (float)Gx;
        tnew.gyf[gq] = (float)Gy;
        if (ex.ring) {
            // export: R, V, F, S of bead q into the ring slot of this phase
            double *d = ex.ring + (size_t)(ex_k % (unsigned long long)ex.slots) * ex.stride + kExportHeader;
            const int nbq = I.nb;
            d[q] = s_rx[q];
            d[nbq + q] = s_ry[q];
            d[2 * nbq + q] = __ldcg(tnew.Vx + gq);
            d[3 * nbq + q] = __ldcg(tnew.Vy + gq);
            d[4 * nbq + q] = Fx;
            d[5 * nbq + q] = Fy;
            d[6 * nbq + q] = s_gx[q];
        }
    }
    if (ex.ring) {
        // the table is in host memory before its slot header says so
        __threadfence_system();
        __syncthreads();
        if (tid == 0) {
            unsigned long long *hdr =
                (unsigned long long *)(ex.ring + (size_t)(ex_k % (unsigned long long)ex.slots) * ex.stride);
            asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(hdr), "l"(ex_k + 1ull) : "memory");
            *ex.count = ex_k + 1ull;
        }
    }
    if (tid == 0) counters[ii] = 0u;
    }  // last bead of the instance
    }  // beads of this CTA
}

}  // namespace

namespace {

// SMs of the current device (cached per device; 0 if unknown).
int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

template <class S>
cudaError_t launch_beads_t(cudaLaunchConfig_t &cfg, bool few, const Inst *inst_d, const int2 *blist, int nb_total,
                           const void *pool, BeadTab tab0, BeadTab tab1, unsigned *mask_write, int gparity,
                           int advance, unsigned *counters, BeadExport ex, unsigned *status) {
    cfg.blockDim = dim3(few ? kBeadThreadsFew : kBeadThreads);
    if (few)
        return cudaLaunchKernelEx(&cfg, k_beads<S, kBeadThreadsFew>, inst_d, blist, nb_total, (const S *)pool, tab0,
                                  tab1, mask_write, gparity, advance, counters, ex, status);
    return cudaLaunchKernelEx(&cfg, k_beads<S, kBeadThreads>, inst_d, blist, nb_total, (const S *)pool, tab0, tab1,
                              mask_write, gparity, advance, counters, ex, status);
}

}  // namespace

cudaError_t launch_beads(int precision, const Inst *inst_d, const int2 *blist, int nb_total, const void *pool,
                         BeadTab tab0, BeadTab tab1, unsigned *mask_write, int gparity, int advance,
                         unsigned *counters, int pdl, cudaStream_t st, BeadExport ex, unsigned *status) {
    if (nb_total <= 0) return cudaSuccess;
    // one CTA per bead: a grid capped at the resident CTAs (persistent) keeps
    // the bead CTAs on the SMs at once and leaves the sweep that follows
    // too few registers to start its unmarked tiles with (measured with
    // 256-thread CTAs: the batched step 8 % slower), so every bead gets its
    // own CTA; a list that fits on the SMs one bead per SM gets wider CTAs
    const bool few = nb_total <= sm_count();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb_total);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (precision) {
        case 0:
            return launch_beads_t<double>(cfg, few, inst_d, blist, nb_total, pool, tab0, tab1, mask_write, gparity,
                                          advance, counters, ex, status);
        case 1:
            return launch_beads_t<float>(cfg, few, inst_d, blist, nb_total, pool, tab0, tab1, mask_write, gparity,
                                         advance, counters, ex, status);
        case 2:
            return launch_beads_t<__half>(cfg, few, inst_d, blist, nb_total, pool, tab0, tab1, mask_write, gparity,
                                          advance, counters, ex, status);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fpd
