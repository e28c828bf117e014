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
// marked beads in bead order.  Every cell pulls its 9 populations from the
// current buffer (shifted reads, bounce-back at the walls), collides (MRT +
// Guo) and stores them at the cell in the other buffer.  Tiles with no wall
// and no periodic wrap among their cells' neighbours address every source
// with one precomputed offset per direction.  No block-wide barrier: each
// thread reads the tile's mask.
#include <cuda_fp16.h>

#include <type_traits>

#include "fpd_kernels.h"

namespace fpd {

namespace {

template <class S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// A tile with beads marked in its mask (the same for every thread of the
// CTA, so all of them call this): the FP32 overlay entries of those beads
// (x hi + lo, y hi + lo, G = F / S) are staged in shared memory, indexed by
// the bead's place in its instance, in one round of loads.  Each cell's loop
// over the marked beads then reads shared memory instead of waiting on a
// memory round trip per bead, which under the sweep's load made the marked
// tiles the last to finish a step (13 us after the bead phase released them,
// FP32).  kStaged: the single-lattice sweeps; the batched sweep (held to 32
// registers) and the FP64 path read the tables, with the same values in the
// same order, so every launch shape still gives the same bits.
template <class R, bool kStaged>
__device__ __forceinline__ const float *stage_overlay(const Inst &I, const BeadTab &tab,
                                                      const unsigned *__restrict__ m, const unsigned any) {
    if constexpr (std::is_same<R, double>::value || !kStaged) {
        return nullptr;
    } else {
        __shared__ float s_ov[kTabFloats * kMaxBeads];
        if (any != 0u) {
            const int nt = blockDim.x * blockDim.y, t = threadIdx.y * blockDim.x + threadIdx.x;
            for (int q = t; q < I.nb; q += nt)
                if ((m[q >> 5] >> (q & 31)) & 1u) {
                    const int gq = I.bead_off + q;
                    s_ov[q] = tab.xh[gq];
                    s_ov[kMaxBeads + q] = tab.xl[gq];
                    s_ov[2 * kMaxBeads + q] = tab.yh[gq];
                    s_ov[3 * kMaxBeads + q] = tab.yl[gq];
                    s_ov[4 * kMaxBeads + q] = tab.gxf[gq];
                    s_ov[5 * kMaxBeads + q] = tab.gyf[gq];
                }
            __syncthreads();
        }
        return s_ov;
    }
}

// Relaxation rates and force density of one cell (Eqs. 1, 2, 4) from the
// beads marked in its tile's mask (m, W words; any = OR of the words).
// kStaged: the FP32 overlay entries are read from sov (stage_overlay), else
// from the table; the values and their order are the same either way.
template <class R, bool kStaged>
__device__ __forceinline__ void cell_overlay(const Inst &I, const BeadTab &tab, const float *__restrict__ sov,
                                             const unsigned *__restrict__ m,
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
        for (int w = 0; w < W && any; ++w) {
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
        const float hny = 0.5f * I.ny, fny = (float)I.ny;
        const float xc = (float)x + 0.5f, yc = (float)y + 0.5f;
        float Phi = I.sandwich ? sandwich_phi_f32(I, yc) : 0.f;
        for (int w = 0; w < W && any; ++w) {
            unsigned bits = m[w];
            while (bits) {
                const int q = 32 * w + __ffs(bits) - 1;  // place in the instance
                bits &= bits - 1u;
                // entry j of bead q: staged, or from the table
                auto ov = [&](int j) -> float {
                    if constexpr (kStaged) return sov[j * kMaxBeads + q];
                    const float *col[kTabFloats] = {tab.xh, tab.xl, tab.yh, tab.yl, tab.gxf, tab.gyf};
                    return col[j][I.bead_off + q];
                };
                // (x_c - R_x) with R_x = hi + lo; the periodic shift is
                // applied to the cell centre first so that xc - hi is exact
                const float bx = ov(0);
                float xcl = xc;
                const float d0 = xcl - bx;
                xcl = (d0 > hnx) ? xcl - fnx : ((d0 < -hnx) ? xcl + fnx : xcl);
                const float dx = (xcl - bx) - ov(1);
                const float by_ = ov(2);
                float ycl = yc;
                if (I.periodic_y) {
                    const float e0 = ycl - by_;
                    ycl = (e0 > hny) ? ycl - fny : ((e0 < -hny) ? ycl + fny : ycl);
                }
                const float dy = (ycl - by_) - ov(3);
                const float ph = phi_f32(dx, dy, I.f_a, I.f_inv_xi, I.f_rcut2);
                Phi += ph;
                Fx += ph * ov(4);
                Fy += ph * ov(5);
            }
        }
        const float nu = I.f_nu_f * (1.0f + I.f_visc_m1 * Phi);
        rates<float>(I.collision, nu, I.f_s_e, I.f_s_eps, I.f_s_q, s_nu, s_e, s_eps, s_q);
    }
}

// Which collision forms a kernel carries: the moment form only (constant
// Lallemand-Luo rates, collision 1), or the two-relaxation-time form for
// unforced cells of the magic and BGK rate sets (collision 0 and 2) with the
// moment form for the rest, or that choice made per instance (a batch that
// mixes rate sets).  Kernels with fewer forms keep fewer registers.
constexpr int kCollTrt = 0, kCollMrt = 1, kCollAny = 2;

// Collision of one cell on stored values (sigma_k g_k).  The moment form
// serves constant Lallemand-Luo rates and every forced cell (a tile with
// beads marked in it, or a uniform body force); the two-relaxation-time form,
// equal in exact arithmetic, serves the unforced cells of the magic and BGK
// rate sets (most of a lattice).  Every kernel makes the same choice per
// cell, so an instance gives the same bits in every launch shape and in a
// batch.
template <int kColl> __device__ __forceinline__ bool moment_form(const Inst &I, bool forced) {
    return kColl == kCollMrt || (kColl == kCollAny && I.collision == 1) || forced;
}
template <class S, class R, int kColl>
__device__ __forceinline__ void collide_cell(const Inst &I, R g[9], R Fx, R Fy, R s_nu, R s_e, R s_eps, R s_q,
                                             bool forced) {
    constexpr bool kScaled = Store<S>::kScaled;
    if (moment_form<kColl>(I, forced)) {
        if constexpr (kScaled) {
#pragma unroll
            for (int k = 0; k < 9; ++k) g[k] *= (R)I.inv_scale[k];
        }
        collide<R>(g, Fx, Fy, s_nu, s_e, s_eps, s_q);
        if constexpr (kScaled) {
#pragma unroll
            for (int k = 0; k < 9; ++k) g[k] *= (R)I.scale[k];
        }
    } else {
        collide_trt<R, kScaled>(g, s_nu, s_q, I);
    }
}

// Whether the uniform body force of the instance is non-zero.
template <class R> __device__ __forceinline__ bool body_forced(const Inst &I) {
    if constexpr (std::is_same<R, double>::value) return I.gx != 0.0 || I.gy != 0.0;
    else return I.f_gx != 0.0f || I.f_gy != 0.0f;
}

// Whether a tile may be updated without waiting for this step's bead phase:
// no bead marked it in the previous bead phase, whose marks cover each
// support widened by a cell.  A bead moves less than a cell per step (its
// velocity is a weighted mean of fluid velocities, which stay far below the
// lattice's one cell per step), so no support reaches such a tile in this
// step either, and the bead phase reads no population of it.  The bead
// phase checks that assumption (|V| < kFastBead per component, with the
// marks covering moves of more than a cell): once it has failed for an
// instance, that phase and every later one mark all tiles of the instance,
// so that they all wait.  The lead CTA always waits: the next launch in the
// stream then cannot start before the bead phase has completed.
__device__ __forceinline__ bool tile_cold_early(const unsigned *__restrict__ prev, const int W, const int early_cold,
                                                const bool lead) {
    if (!early_cold || lead) return false;
    unsigned any = 0u;
    for (int w = 0; w < W; ++w) any |= prev[w];
    return any == 0u;
}

// Storage types whose variant-1 threads own two x-adjacent cells, moved
// with one paired access per plane (FP16: one packed conversion for both);
// the FP64 path places them kTileX / 2 apart.
template <class S> struct AdjPairs { static constexpr bool value = !std::is_same<S, double>::value; };

// Second half of a tile's update for a thread's CY cells: the fields of
// Eqs. 1, 2, 4 at each cell, the collision (the two-relaxation-time form of
// two unforced cells in packed FP32 pairs, else cell by cell) and the stores
// into buffer Adst.  g holds the pulled populations in stored units; the
// cells' layout is lattice_tile's (kAlongX, CY, kAdj).
template <class S, int CY, bool kInner, bool kAlongX, int kColl, bool kStream>
__device__ __forceinline__ void finish_cells(const Inst &I, const BeadTab &tab, const float *__restrict__ sov,
                                             const unsigned *__restrict__ m, const int W, const unsigned any,
                                             const int x, const int (&y)[CY], const bool (&valid)[CY],
                                             const Cell (&C)[CY], typename Real<S>::type (&g)[CY][9],
                                             S *__restrict__ Adst, const int cx0, const uint64_t pol) {
    using R = typename Real<S>::type;
    constexpr bool kAdj = kAlongX && CY == 2 && AdjPairs<S>::value;
    constexpr int RX = kAlongX ? (kAdj ? 1 : kTileX / CY) : 0;
    const bool forced = any != 0u || body_forced<R>(I);
    // stores of the thread's cells (k < CY); x-adjacent pairs in one access
    // per plane when both are in the lattice
    auto store = [&]() {
        if constexpr (kAdj) {
            S *q = Adst + (y[0] * kRowStride + cx0);
            if (valid[1]) put_adj<S, kStream>(q, g[0], g[1], pol);
            else put_at<S, R, true, kStream>(q, I, g[0], pol);
        } else {
#pragma unroll
            for (int k = 0; k < CY; ++k)
                if (valid[k])
                    put_at<S, R, true, kStream>(Adst + (kInner ? y[k] * kRowStride + cx0 + k * RX : C[k].o), I,
                                                g[k], pol);
        }
    };
    if constexpr (CY == 2 && std::is_same<R, float>::value) {
        // two unforced cells: the two-relaxation-time collision on both at
        // once, in packed FP32 pairs (each lane rounds as a lone cell does)
        if (valid[1] && !moment_form<kColl>(I, forced)) {
            R Fx, Fy, s_e, s_eps, s_nu[2], s_q[2];
#pragma unroll
            for (int k = 0; k < 2; ++k)
                cell_overlay<R, kStream>(I, tab, sov, m, W, any, x + k * RX, y[k], Fx, Fy, s_nu[k], s_e, s_eps,
                                         s_q[k]);
            float2 v[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = make_float2(g[0][q], g[1][q]);
            collide_trt<R, Store<S>::kScaled>(v, make_float2(s_nu[0], s_nu[1]), make_float2(s_q[0], s_q[1]), I);
#pragma unroll
            for (int q = 0; q < 9; ++q) g[0][q] = v[q].x, g[1][q] = v[q].y;
            store();
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < CY; ++k) {
        if (!valid[k]) continue;
        R Fx, Fy, s_nu, s_e, s_eps, s_q;
        cell_overlay<R, kStream>(I, tab, sov, m, W, any, x + k * RX, y[k], Fx, Fy, s_nu, s_e, s_eps, s_q);
        collide_cell<S, R, kColl>(I, g[k], Fx, Fy, s_nu, s_e, s_eps, s_q, forced);
    }
    store();
}

// One tile of the sweep: tile (bx, by) of instance I at the instance's step
// parity, on kTileX x (kTileY / CY) threads; thread (tx, ty) owns the CY
// cells (x, y0 + ty + k kTileY / CY), k < CY, of its column.  kAlongX: on
// (kTileX / CY) x kTileY threads instead, thread (tx, ty) owns the CY cells
// (x0 + tx + k kTileX / CY, y0 + ty) of its row, whose elements in every
// plane lie a constant distance apart, so that one address serves all of
// them (immediate offsets); with two cells and FP32 or FP16 storage they
// are the adjacent cells x0 + 2 tx and x0 + 2 tx + 1 (paired accesses, and
// the two-relaxation-time collision of both in packed FP32 pairs).  kInner:
// tiles away from walls and periodic edges use the in-strip pull offsets.
// kStream: the population loads and stores carry the L2 evict-first
// priority (the single-lattice sweep).
template <class S, int CY, bool kInner, bool kAlongX, int kColl, bool kStream = false>
__device__ __forceinline__ void lattice_tile(const Inst &I, S *__restrict__ pool, const BeadTab &tab,
                                             const unsigned *__restrict__ mask_read,
                                             const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear,
                                             const int bx, const int by, const int parity, const int early_load,
                                             const int early_cold, const bool lead, const int tx, const int ty) {
    using R = typename Real<S>::type;
    // kAdj: the two cells of a thread are x-adjacent (FP32 and FP16
    // storage), moved with paired accesses; otherwise kTileX / 2 apart
    constexpr bool kAdj = kAlongX && CY == 2 && AdjPairs<S>::value;
    constexpr int RY = kAlongX ? 0 : kTileY / CY;
    constexpr int RX = kAlongX ? (kAdj ? 1 : kTileX / CY) : 0;
    const int xt = kAdj ? 2 * tx : tx;  // column within the tile
    const int x = bx * kTileX + xt;
    const int tile = I.tile_base + by * I.ntx + bx;
    const int W = I.mask_words;
    const S *Asrc = pop_buffer(pool, I, parity);
    S *Adst = pop_buffer(pool, I, parity ^ 1);
    // every cell of the tile and its neighbours lie inside the lattice
    const bool inner = kInner && bx > 0 && by > 0 && (bx + 1) * kTileX < I.nx && (by + 1) * kTileY < I.ny;
    int y[CY];
    bool valid[CY];
    Cell C[CY];  // general form only
    R g[CY][9];
#pragma unroll
    for (int k = 0; k < CY; ++k) {
        y[k] = by * kTileY + ty + k * RY;
        valid[k] = x + k * RX < I.nx && y[k] < I.ny;
        if constexpr (!kInner) C[k] = make_cell(I, x + k * RX, valid[k] ? y[k] : 0);
    }
    // the population stream's L2 priority, made once per thread
    uint64_t pol = 0;
    if constexpr (kStream) pol = pol_evict_first();
    // populations in stored units (sigma_k g_k)
    const int cx0 = col_off(I, x);  // the thread's cells k sit k RX columns on, within the strip
    auto pull = [&]() {
        if (inner) {
            const S *p = Asrc + (y[0] * kRowStride + cx0);
            if constexpr (kAdj) {
                pull_adj<S, kStream>(p, strip_left(I, xt), strip_right(I, xt + 1), g[0], g[1], pol);
            } else {
#pragma unroll
                for (int k = 0; k < CY; ++k) {
                    const S *pk = p + (k * RY * kRowStride + k * RX);
                    pull_inner<S, R, true, kStream>(pk, strip_left(I, xt + k * RX), strip_right(I, xt + k * RX), I,
                                                    g[k], pol);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < CY; ++k)
                if (valid[k]) pull_pops<S, R, true, kStream>(Asrc, I, kInner ? make_cell(I, x + k * RX, y[k]) : C[k], g[k], pol);
        }
    };
    // populations come from the previous sweep; when the bead phase runs
    // between the two sweeps they may be loaded before waiting on it
    if (early_load) pull();
    const bool cold = tile_cold_early(mask_prev + tile * W, W, early_cold, lead);
    if (!cold) pdl_wait();
    pdl_trigger();
    if (tx == 0 && ty == 0)  // a mask of two steps back, for the next bead phase
        for (int w = 0; w < W; ++w) mask_clear[tile * W + w] = 0u;
    if constexpr (kAdj && kInner && kStream && kColl == kCollTrt && std::is_same<S, __half>::value) {
        // an unmarked tile away from walls and edges, with no body force or
        // sandwich layer: both cells are unforced at the fluid rates, so
        // finish_cells would take its packed two-relaxation-time branch with
        // s_nu and s_q of Phi = 0; the same operations in a straight line
        // (FP16 storage: step 34.6 -> 33.9 us; FP32 storage measured slower
        // with it, 44.6 -> 45.4 us, and keeps the general path)
        if (cold && inner && !I.sandwich && !body_forced<R>(I)) {
            if (!early_load) pull();
            float2 v[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) v[q] = make_float2(g[0][q], g[1][q]);
            const float sp = I.fluid_rates_f[0], sm = I.fluid_rates_f[3];
            collide_trt<R, Store<S>::kScaled>(v, make_float2(sp, sp), make_float2(sm, sm), I);
#pragma unroll
            for (int q = 0; q < 9; ++q) g[0][q] = v[q].x, g[1][q] = v[q].y;
            put_adj<S, kStream>(Adst + (y[0] * kRowStride + cx0), g[0], g[1], pol);
            return;
        }
    }
    if constexpr (CY == 1 && kInner && kColl == kCollTrt && !std::is_same<S, double>::value) {
        // the same for one cell per thread (variant 0, the batched sweep):
        // the one-cell two-relaxation-time update at the fluid rates that
        // finish_cells takes for an unforced cell, in a straight line; at
        // walls and edges too (the pull handles them)
        if (cold && !I.sandwich && !body_forced<R>(I)) {
            if (!valid[0]) return;
            if (!early_load) pull();
            collide_trt<R, Store<S>::kScaled>(g[0], I.fluid_rates_f[0], I.fluid_rates_f[3], I);
            put_at<S, R, true, kStream>(Adst + (y[0] * kRowStride + cx0), I, g[0], pol);
            return;
        }
    }
    const unsigned *m = mask_read + tile * W;
    unsigned any = 0u;
    if (!cold)
        for (int w = 0; w < W; ++w) any |= m[w];
    const float *sov = stage_overlay<R, kStream>(I, tab, m, any);  // every thread of the CTA
    if (!valid[0]) return;  // the thread's other cells (further along its column or row) are invalid too
    if (!early_load) pull();
    finish_cells<S, CY, kInner, kAlongX, kColl, kStream>(I, tab, sov, m, W, any, x, y, valid, C, g, Adst, cx0, pol);
}

// Tile order of a single-lattice sweep.  Every other step takes the tiles
// in reverse order, so that it starts on the tiles the previous sweep wrote
// last, whose populations are still in L2 (a lattice larger than L2 is
// otherwise read back in the order it was written, which under LRU evicts
// each line before it is read again).  Which tile a CTA takes changes
// nothing in its arithmetic.  The lead CTA (the first dispatched) is
// blockIdx 0 either way.  The batched sweep keeps its tile list in order
// (its state is many times the L2: reversing measured no gain there).
__device__ __forceinline__ int tile_order(int b, int n, int parity) { return (parity & 1) ? n - 1 - b : b; }

template <class S, int CY, bool kAlongX, int kColl>
__global__ void __launch_bounds__(kTileX *kTileY / CY)
    k_lattice(const Inst I, S *__restrict__ pool, const BeadTab tab, const unsigned *__restrict__ mask_read,
              const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear, const int parity,
              const int early_load, const int early_cold) {
    lattice_tile<S, CY, true, kAlongX, kColl, true>(I, pool, tab, mask_read, mask_prev, mask_clear,
                                       tile_order(blockIdx.x, gridDim.x, parity),
                                       tile_order(blockIdx.y, gridDim.y, parity), parity, early_load, early_cold,
                                       (blockIdx.x | blockIdx.y) == 0, threadIdx.x, threadIdx.y);
}

// --------------------------------------------- staged sweep (variants 3, 4)
// A CTA of kTileX / 2 x kTileY threads updates NS tiles stacked in y (a
// block of 32 x 8 NS cells, one strip wide).  Its populations and their y
// halo, rows y0 - 1 .. y0 + 8 NS of the strip, are contiguous in the
// current buffer (the strip layout), so one elected thread moves all of them
// into shared memory with a single bulk copy (cp.async.bulk, completion on
// an mbarrier) the moment the CTA starts; the x halo (column 31 of the
// strip to the left for the three directions with c_kx = +1, column 0 of
// the one to the right for c_kx = -1) comes with plain loads.  The copy
// engine keeps a whole block in flight per CTA without holding registers,
// where the register-fed pull of variant 1 keeps 36 B (FP16) or 72 B (FP32)
// a thread in flight.  Each thread then pulls its two x-adjacent cells of
// every tile from shared memory and runs the same collision and stores as
// variant 1 (finish_cells), so the results are bit-identical to it.  Tiles
// the previous bead phase left unmarked are updated first, without waiting
// for this step's bead phase; the others after it.  Blocks at a wall, at the
// periodic edges or at the lattice's ragged end run variant 1's tile code.
// Every wait on the copy is bounded: a copy that has not completed within
// kCopyWaitNs sets kFlagCopyTimeout in the instance's status word and the
// CTA leaves its block unwritten (reported by fpd_sync).
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barrier visible to the copy engine (async proxy)
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from global src to shared dst, both 16-byte
// aligned, completing as transaction bytes on bar; L2 policy pol
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned phase) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return done != 0u;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `phase` of bar to complete, for at most kCopyWaitNs (and a
// bounded number of polls); false when it did not.
constexpr unsigned long long kCopyWaitNs = 100000000ull;  // 0.1 s
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase) {
    if (mbar_test(bar, phase)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned i = 0; i < (1u << 24); ++i) {
        if (mbar_test(bar, phase)) return true;
        if (globaltimer_ns() - t0 > kCopyWaitNs) break;
    }
    return false;
}

// x-halo slot of the directions with c_kx != 0: 0..2 for k = 1, 5, 8
// (column 31 of the strip to the left), 3..5 for k = 3, 6, 7 (column 0 of
// the strip to the right)
template <int k> struct HaloSlot {
    static constexpr int value = k == 1 ? 0 : k == 5 ? 1 : k == 8 ? 2 : k == 3 ? 3 : k == 6 ? 4 : 5;
};
__device__ __forceinline__ int halo_plane(int j) { return j == 0 ? 1 : j == 1 ? 5 : j == 2 ? 8 : j == 3 ? 3 : j == 4 ? 6 : 7; }

// Pull of direction k for the two x-adjacent cells a (column xt, even) and
// b = a + 1 of staged row r, p = rows + r kRowStride + xt: the same sources
// as pull_adj, read from shared memory, with the strip-edge sources from
// the x halo.
template <int k, class S>
__device__ __forceinline__ void pull_staged_one(const S *__restrict__ p, const float (*__restrict__ halo)[6],
                                                const int r, const int xt, float ga[9], float gb[9]) {
    constexpr int cx = Q<k>::cx, cy = Q<k>::cy, off = PullOff<k>::value;
    if constexpr (cx == 0) {
        Store<S>::ld2_raw(p + off, ga[k], gb[k]);
    } else if constexpr (cx > 0) {
        ga[k] = (xt == 0) ? halo[r - cy][HaloSlot<k>::value] : Store<S>::ld_raw(p + off);
        gb[k] = Store<S>::ld_raw(p + 1 + off);
    } else {
        ga[k] = Store<S>::ld_raw(p + off);
        gb[k] = (xt == kTileX - 2) ? halo[r - cy][HaloSlot<k>::value] : Store<S>::ld_raw(p + 1 + off);
    }
}
template <class S>
__device__ __forceinline__ void pull_staged(const S *__restrict__ p, const float (*__restrict__ halo)[6], const int r,
                                            const int xt, float ga[9], float gb[9]) {
    pull_staged_one<0, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<2, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<4, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<1, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<5, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<8, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<3, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<6, S>(p, halo, r, xt, ga, gb);
    pull_staged_one<7, S>(p, halo, r, xt, ga, gb);
}

// Tiles per CTA of the staged sweep (variant 3: kStagedNS, variant 4: twice
// that), chosen so that a block's staged rows stay near 20 KB and 40 KB.
template <class S> struct StagedNS { static constexpr int value = std::is_same<S, __half>::value ? 4 : 2; };

template <class S, int NS>
__global__ void __launch_bounds__(kTileX *kTileY / 2)
    k_lattice_staged(const Inst I, S *__restrict__ pool, const BeadTab tab, const unsigned *__restrict__ mask_read,
                     const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear, const int parity,
                     const int early_load, const int early_cold, unsigned *__restrict__ status,
                     const unsigned shortfall) {
    using R = float;
    constexpr int kThreads = kTileX * kTileY / 2;
    constexpr int kRows = NS * kTileY + 2;
    constexpr unsigned kBytes = kRows * kRowStride * sizeof(S);
    static_assert(kBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
    __shared__ __align__(128) unsigned char s_raw[kBytes];
    __shared__ float s_halo[kRows][6];
    __shared__ __align__(8) unsigned long long s_bar;
    const int bx = tile_order(blockIdx.x, gridDim.x, parity), bb = tile_order(blockIdx.y, gridDim.y, parity);
    const bool lead = (blockIdx.x | blockIdx.y) == 0;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * (kTileX / 2) + tx;
    const int by0 = bb * NS;
    // the block's cells, their neighbours and the staged rows lie inside the
    // lattice, away from walls and periodic edges
    const bool inner = bx > 0 && by0 > 0 && (bx + 1) * kTileX < I.nx && (by0 + NS) * kTileY < I.ny;
    if (!inner) {
        for (int s = 0; s < NS && by0 + s < I.nty; ++s) {
            if (s) __syncthreads();  // the previous tile's cells no longer read the staged overlay
            lattice_tile<S, 2, true, true, kCollTrt, true>(I, pool, tab, mask_read, mask_prev, mask_clear, bx, by0 + s,
                                                           parity, early_load, early_cold, lead, tx, ty);
        }
        return;
    }
    const S *Asrc = pop_buffer(pool, I, parity);
    S *Adst = pop_buffer(pool, I, parity ^ 1);
    const int y0 = by0 * kTileY;
    // row y0 - 1 of the block's strip; its populations come from the previous
    // sweep, complete before this launch began (the bead phase in between
    // waited for it), so they are read at once
    const S *g0 = Asrc + ((y0 - 1) * kRowStride + col_off(I, bx * kTileX));
    const uint64_t pol = pol_evict_first();
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&s_bar, kBytes + shortfall);  // shortfall: 0 but in a failure test
        bulk_g2s(s_raw, g0, kBytes, &s_bar, pol);
    }
    for (int h = tid; h < kRows * 6; h += kThreads) {
        const int r = h / 6, j = h - 6 * r;
        const int col = j < 3 ? kStripW - 1 - I.strip : I.strip;  // from column 0 of the block's strip
        s_halo[r][j] = Store<S>::ld_stream(g0 + (r * kRowStride + halo_plane(j) * kPlaneStride + col), pol);
    }
    const int W = I.mask_words;
    unsigned cold = 0u;
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (tile_cold_early(mask_prev + (I.tile_base + (by0 + s) * I.ntx + bx) * W, W, early_cold, lead))
            cold |= 1u << s;
    if (tid == 0)  // masks of two steps back, for the next bead phase
        for (int s = 0; s < NS; ++s)
            for (int w = 0; w < W; ++w) mask_clear[(I.tile_base + (by0 + s) * I.ntx + bx) * W + w] = 0u;
    __syncthreads();  // the barrier is initialised, the x halo staged
    const bool copied = mbar_wait_bounded(&s_bar, 0);
    if (__syncthreads_or(!copied)) {
        if (tid == 0 && status) atomicOr(status, kFlagCopyTimeout);
        if (!copied) mbar_wait_bounded(&s_bar, 0);  // let a late copy land before the CTA ends
        if (lead) pdl_wait();
        return;
    }
    if (cold == (1u << NS) - 1u) pdl_trigger();
    const int xt = 2 * tx, x = bx * kTileX + xt, cx0 = col_off(I, x);
    const S *rows = reinterpret_cast<const S *>(s_raw);
    bool waited = false;
    // the unmarked tiles first, then, after this step's bead phase, the rest
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 1
        for (int s = 0; s < NS; ++s) {
            const bool c = (cold >> s) & 1u;
            if (c != (pass == 0)) continue;
            if (!c && !waited) {
                pdl_wait();
                pdl_trigger();
                waited = true;
            }
            const unsigned *m = mask_read + (I.tile_base + (by0 + s) * I.ntx + bx) * W;
            unsigned any = 0u;
            if (!c)
                for (int w = 0; w < W; ++w) any |= m[w];
            if (any != 0u) __syncthreads();  // the previous tile's cells no longer read the staged overlay
            const float *sov = stage_overlay<R, true>(I, tab, m, any);
            const int r = s * kTileY + ty + 1;  // staged row of the thread's cells
            const int y[2] = {y0 + r - 1, y0 + r - 1};
            const bool valid[2] = {true, true};
            Cell C[2];  // unused: inner cells
            R g[2][9];
            pull_staged<S>(rows + (r * kRowStride + xt), s_halo, r, xt, g[0], g[1]);
            finish_cells<S, 2, true, true, kCollTrt, true>(I, tab, sov, m, W, any, x, y, valid, C, g, Adst, cx0, pol);
        }
    }
}

// Batched sweep over a packed tile list: tiles[t] = (instance slot,
// by << 16 | bx).  Each instance reads table and layout of its own parity
// (global parity ^ par_xor); the record is copied to shared memory per CTA.
// Resident CTAs per SM the batched sweep is compiled for: one cell per
// thread in the reduced-precision paths fits the in-strip pull offsets in
// 32 registers (8 CTAs of 256 threads); the other shapes keep the register
// counts they had without a bound.
template <class S, int CY> struct BatchMinBlocks {
    static constexpr int value = std::is_same<S, double>::value ? 4 : (CY == 1 ? 8 : 7);
};
// Which batched shapes use the in-strip pull offsets of inner tiles.
template <class S, int CY, bool kAlongX> struct BatchInner {
    static constexpr bool value = (CY == 1 || kAlongX) && !std::is_same<S, double>::value;
};

template <class S, int CY, bool kAlongX, int kColl>
__global__ void __launch_bounds__(kTileX *kTileY / CY, BatchMinBlocks<S, CY>::value)
    k_lattice_batch(const Inst *__restrict__ insts, const int2 *__restrict__ tiles, S *__restrict__ pool,
                    const BeadTab tab0, const BeadTab tab1, const unsigned *__restrict__ mask_read,
                    const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear, const int gparity,
                    const int early_load, const int early_cold) {
    __shared__ Inst sI;
    const int2 t = tiles[blockIdx.x];
    {
        const unsigned *src = (const unsigned *)(insts + t.x);
        unsigned *dst = (unsigned *)&sI;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        for (int wd = tid; wd < (int)(sizeof(Inst) / 4); wd += kTileX * kTileY / CY) dst[wd] = src[wd];
    }
    __syncthreads();
    const int parity = gparity ^ sI.par_xor;
    lattice_tile<S, CY, BatchInner<S, CY, kAlongX>::value, kAlongX, kColl>(
        sI, pool, parity ? tab1 : tab0, mask_read, mask_prev, mask_clear, t.y & 0xffff, t.y >> 16, parity,
        early_load, early_cold, blockIdx.x == 0, threadIdx.x, threadIdx.y);
}

// ------------------------------------------------ vectorised sweep (variant 2)
// Each thread owns NV consecutive cells of one tile row and moves each of its
// nine planes with one 16-byte access (8 bytes for FP16 storage).  A tile row
// of 32 cells is a segment of G = 32 / NV lanes of one warp.  Stores are
// aligned.  A pulled direction with c_kx = +1 needs the element one to the
// left of the thread's vector (mirrored for c_kx = -1): it comes from the
// neighbouring lane by a shuffle, and at the segment ends (tile edges, the
// periodic wrap, the last cell of a row) the edge lane reads that single
// element with a scalar access.  Requires nx % NV == 0.

template <class S, int NV> struct VecIO;
template <> struct VecIO<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float, float v[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float *p, const float v[4], float) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct VecIO<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, float, double v[2]) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x, v[1] = t.y;
    }
    static __device__ __forceinline__ void st(double *p, const double v[2], float) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};
template <> struct VecIO<__half, 4> {
    // stored values (sigma_k g_k): exact widening; round-to-nearest narrowing
    static __device__ __forceinline__ void ld(const __half *p, float, float v[4]) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    static __device__ __forceinline__ void st(__half *p, const float v[4], float) {
        const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 t;
        t.x = *reinterpret_cast<const unsigned *>(&a);
        t.y = *reinterpret_cast<const unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = t;
    }
};

template <class S> struct VecWidth { static constexpr int value = 16 / (int)sizeof(S); };
template <> struct VecWidth<__half> { static constexpr int value = 4; };

// The NV cells x0 .. x0 + NV - 1 of row y owned by one thread.
struct VCell {
    int x0, xm, xp;  // first cell, the cell left of it, the cell right of the last (periodic): element offsets
    int r0, rm, rp;  // element offsets of rows y, y - 1, y + 1 (wrapped when y is periodic)
    bool bot, top, valid;
    bool left, right;  // first lane of its segment / last lane holding cells of its row segment
};
template <int NV>
__device__ __forceinline__ VCell make_vcell(const Inst &I, int x0, int y, int lane_in_seg) {
    constexpr int G = kTileX / NV;
    VCell c;
    c.valid = x0 < I.nx && y < I.ny;
    const int yy = c.valid ? y : 0;
    // column element offsets (NV divides the strip width: a vector stays in its strip)
    c.x0 = col_off(I, x0 < I.nx ? x0 : 0);
    c.xm = col_off(I, (x0 == 0) ? I.nx - 1 : x0 - 1);
    c.xp = col_off(I, (x0 + NV >= I.nx) ? 0 : x0 + NV);
    c.r0 = yy * kRowStride;
    c.rm = ((yy == 0) ? I.ny - 1 : yy - 1) * kRowStride;
    c.rp = ((yy == I.ny - 1) ? 0 : yy + 1) * kRowStride;
    c.bot = (yy == 0) && !I.periodic_y;
    c.top = (yy == I.ny - 1) && !I.periodic_y;
    c.left = lane_in_seg == 0;
    c.right = lane_in_seg == G - 1 || x0 + NV == I.nx;
    return c;
}

// Pull of direction k into g[j][k] for the thread's NV cells (see pull_one
// for the scalar form).  Every lane executes the shuffles.
template <int k, class S, int NV, class R>
__device__ __forceinline__ void vload_one(const S *__restrict__ A, const Inst &I, const VCell &C, R g[NV][9]) {
    constexpr int cx = Q<k>::cx, cy = Q<k>::cy, o = Q<k>::opp;
    constexpr int G = kTileX / NV;
    R v[NV];
    const bool wall = (cy > 0 && C.bot) || (cy < 0 && C.top);
    const int row = wall ? C.r0 : (cy > 0 ? C.rm : (cy < 0 ? C.rp : C.r0));
    // stored values (scale[k] == scale[opp k]: the wall's reflected plane
    // is in the same units)
    if (C.valid) VecIO<S, NV>::ld(A + ((wall ? o : k) * kPlaneStride + row + C.x0), 1.0f, v);
    else {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = (R)0;
    }
    R nb = (R)0;
    if constexpr (cx > 0) nb = __shfl_up_sync(0xffffffffu, v[NV - 1], 1, G);
    if constexpr (cx < 0) nb = __shfl_down_sync(0xffffffffu, v[0], 1, G);
    if (wall) {
        const R b = bb_stored<R>(I, cy > 0 ? 0 : 1, k);
#pragma unroll
        for (int j = 0; j < NV; ++j) g[j][k] = v[j] + b;
        return;
    }
    if constexpr (cx == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) g[j][k] = v[j];
    } else if constexpr (cx > 0) {
        if (C.left && C.valid) nb = (R)Store<S>::ld_raw(A + (k * kPlaneStride + row + C.xm));
        g[0][k] = nb;
#pragma unroll
        for (int j = 1; j < NV; ++j) g[j][k] = v[j - 1];
    } else {
        if (C.right && C.valid) nb = (R)Store<S>::ld_raw(A + (k * kPlaneStride + row + C.xp));
#pragma unroll
        for (int j = 0; j < NV - 1; ++j) g[j][k] = v[j + 1];
        g[NV - 1][k] = nb;
    }
}

// Aligned store of the post-collision populations of direction k.
template <int k, class S, int NV, class R>
__device__ __forceinline__ void vstore_one(S *__restrict__ D, const Inst &I, const VCell &C, const R g[NV][9]) {
    if (!C.valid) return;
    R v[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = g[j][k];
    VecIO<S, NV>::st(D + (k * kPlaneStride + C.r0 + C.x0), v, 1.0f);
}

template <class S, int NV, class R>
__device__ __forceinline__ void vload_pops(const S *__restrict__ A, const Inst &I, const VCell &C, R g[NV][9]) {
    vload_one<0, S, NV>(A, I, C, g);
    vload_one<1, S, NV>(A, I, C, g);
    vload_one<2, S, NV>(A, I, C, g);
    vload_one<3, S, NV>(A, I, C, g);
    vload_one<4, S, NV>(A, I, C, g);
    vload_one<5, S, NV>(A, I, C, g);
    vload_one<6, S, NV>(A, I, C, g);
    vload_one<7, S, NV>(A, I, C, g);
    vload_one<8, S, NV>(A, I, C, g);
}

template <class S, int NV, class R>
__device__ __forceinline__ void vstore_pops(S *__restrict__ A, const Inst &I, const VCell &C, const R g[NV][9]) {
    vstore_one<0, S, NV>(A, I, C, g);
    vstore_one<1, S, NV>(A, I, C, g);
    vstore_one<2, S, NV>(A, I, C, g);
    vstore_one<3, S, NV>(A, I, C, g);
    vstore_one<4, S, NV>(A, I, C, g);
    vstore_one<5, S, NV>(A, I, C, g);
    vstore_one<6, S, NV>(A, I, C, g);
    vstore_one<7, S, NV>(A, I, C, g);
    vstore_one<8, S, NV>(A, I, C, g);
}

// One tile with (32 / NV) x 8 threads; thread (tx, ty) owns cells
// x0 = bx 32 + tx NV .. x0 + NV - 1 of row by 8 + ty.  No lane returns
// before the scatter: the shuffles need the whole warp.
template <class S>
__device__ __forceinline__ void lattice_tile_vec(const Inst &I, S *__restrict__ pool, const BeadTab &tab,
                                                 const unsigned *__restrict__ mask_read,
                                                 const unsigned *__restrict__ mask_prev,
                                                 unsigned *__restrict__ mask_clear, const int bx, const int by,
                                                 const int parity, const int early_load, const int early_cold,
                                                 const bool lead) {
    using R = typename Real<S>::type;
    constexpr int NV = VecWidth<S>::value;
    const int x0 = bx * kTileX + threadIdx.x * NV;
    const int y = by * kTileY + threadIdx.y;
    const int tile = I.tile_base + by * I.ntx + bx;
    const int W = I.mask_words;
    const S *Asrc = pop_buffer(pool, I, parity);
    S *Adst = pop_buffer(pool, I, parity ^ 1);
    const VCell C = make_vcell<NV>(I, x0, y, threadIdx.x);
    R g[NV][9];
    if (early_load) vload_pops<S, NV>(Asrc, I, C, g);
    const bool cold = tile_cold_early(mask_prev + tile * W, W, early_cold, lead);
    if (!cold) pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int w = 0; w < W; ++w) mask_clear[tile * W + w] = 0u;
    if (!early_load) vload_pops<S, NV>(Asrc, I, C, g);
    const unsigned *m = mask_read + tile * W;
    unsigned any = 0u;
    if (!cold)
        for (int w = 0; w < W; ++w) any |= m[w];
    const float *sov = stage_overlay<R, true>(I, tab, m, any);  // every thread of the CTA
    if (C.valid) {
        const bool forced = any != 0u || body_forced<R>(I);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            R Fx, Fy, s_nu, s_e, s_eps, s_q;
            cell_overlay<R, true>(I, tab, sov, m, W, any, x0 + j, y, Fx, Fy, s_nu, s_e, s_eps, s_q);
            collide_cell<S, R, kCollTrt>(I, g[j], Fx, Fy, s_nu, s_e, s_eps, s_q, forced);
        }
    }
    vstore_pops<S, NV>(Adst, I, C, g);
}

template <class S>
__global__ void __launch_bounds__(kTileX / VecWidth<S>::value * kTileY)
    k_lattice_vec(const Inst I, S *__restrict__ pool, const BeadTab tab, const unsigned *__restrict__ mask_read,
                  const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear, const int parity,
                  const int early_load, const int early_cold) {
    lattice_tile_vec<S>(I, pool, tab, mask_read, mask_prev, mask_clear, tile_order(blockIdx.x, gridDim.x, parity),
                        tile_order(blockIdx.y, gridDim.y, parity), parity, early_load, early_cold,
                        (blockIdx.x | blockIdx.y) == 0);
}

// The column form needs more registers than the vector form: cap them at
// 128 (8 CTAs of 64 threads) for FP32 / FP16 storage; FP64 (128 threads)
// keeps 3 CTAs per SM without spilling
template <class S> struct BatchVecMinBlocks { static constexpr int value = sizeof(S) == 8 ? 3 : 8; };
template <class S>
__global__ void __launch_bounds__(kTileX / VecWidth<S>::value * kTileY, BatchVecMinBlocks<S>::value)
    k_lattice_batch_vec(const Inst *__restrict__ insts, const int2 *__restrict__ tiles, S *__restrict__ pool,
                        const BeadTab tab0, const BeadTab tab1, const unsigned *__restrict__ mask_read,
                        const unsigned *__restrict__ mask_prev, unsigned *__restrict__ mask_clear, const int gparity,
                        const int early_load, const int early_cold) {
    constexpr int NT = kTileX / VecWidth<S>::value * kTileY;
    __shared__ Inst sI;
    const int2 t = tiles[blockIdx.x];
    {
        const unsigned *src = (const unsigned *)(insts + t.x);
        unsigned *dst = (unsigned *)&sI;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        for (int wd = tid; wd < (int)(sizeof(Inst) / 4); wd += NT) dst[wd] = src[wd];
    }
    __syncthreads();
    const int parity = gparity ^ sI.par_xor;
    // an instance whose width is not a multiple of NV runs the column form
    // on the same threads: NV cells per thread along y
    constexpr int NV = VecWidth<S>::value;
    if (sI.nx % NV == 0) {
        lattice_tile_vec<S>(sI, pool, parity ? tab1 : tab0, mask_read, mask_prev, mask_clear, t.y & 0xffff,
                            t.y >> 16, parity, early_load, early_cold, blockIdx.x == 0);
    } else {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        lattice_tile<S, NV, false, false, kCollTrt>(sI, pool, parity ? tab1 : tab0, mask_read, mask_prev,
                                                    mask_clear, t.y & 0xffff, t.y >> 16, parity, early_load,
                                                    early_cold, blockIdx.x == 0, tid % kTileX, tid / kTileX);
    }
}

// Equilibrium start: f_k = f_k^eq(rho = 1, u = (u_wall(y), 0)) with the
// linear wall profile, or the rest state; placed (as deviations) in buffer 0
// so that the first step pulls exactly these values.
template <class S>
__global__ void k_init(const Inst I, S *__restrict__ pool, int couette) {
    using R = typename Real<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    const double ux = couette ? I.u_bot + (I.u_top - I.u_bot) * (y + 0.5) / I.ny : 0.0;
    const int cxs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    R g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double cu = cxs[k] * ux;
        g[k] = (R)(ws[k] * (3.0 * cu + 4.5 * cu * cu - 1.5 * ux * ux));
    }
    place_pops<S, R>(pop_buffer(pool, I, 0), I, make_cell(I, x, y), g);
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
    pull_pops<S, double>(pop_buffer(pool, I, parity), I, make_cell(I, x, y), g);
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

// eps_v of each bead (Sec. 3.2): one CTA per bead over its support box,
// FP64; out[2 q] = sum phi_q |u - V_q|^2, out[2 q + 1] = sum phi_q.
constexpr int kFlowThreads = 256;
template <class S>
__global__ void __launch_bounds__(kFlowThreads)
    k_internal_flow(const Inst I, const S *__restrict__ pool, const BeadTab tab, int parity, double *__restrict__ out) {
    __shared__ double sh[2][kFlowThreads / 32];
    const int q = I.bead_off + blockIdx.x;
    const double Rx = tab.Rx[q], Ry = tab.Ry[q], Vx = tab.Vx[q], Vy = tab.Vy[q];
    const Box bx = support_box(I, Rx, Ry);
    double num = 0.0, den = 0.0;
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        const int cj = c / bx.w, ci = c - cj * bx.w;
        int i = bx.i0 + ci, j = bx.j0 + cj;
        i = (i >= I.nx) ? i - I.nx : i;
        j = (j >= I.ny) ? j - I.ny : j;
        const double ph = phi_f64(I, i + 0.5, j + 0.5, Rx, Ry);
        if (ph == 0.0) continue;
        double g[9];
        pull_pops<S, double>(pop_buffer(pool, I, parity), I, make_cell(I, i, j), g);
        double dr = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) dr += g[k];
        const double r = 1.0 + dr;
        const double jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
        const double jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
        double fx, fy;
        overlay_f64(I, tab, nullptr, i, j, fx, fy);
        const double ex = (jx + 0.5 * fx) / r - Vx, ey = (jy + 0.5 * fy) / r - Vy;
        num += ph * (ex * ex + ey * ey);
        den += ph;
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane_id() == 0) {
        sh[0][threadIdx.x >> 5] = num;
        sh[1][threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kFlowThreads / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        out[2 * blockIdx.x] = a;
        out[2 * blockIdx.x + 1] = b;
    }
}

template <class S>
__global__ void k_read_pops(const Inst I, const S *__restrict__ pool, int parity, double *__restrict__ f) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    double g[9];
    pull_pops<S, double>(pop_buffer(pool, I, parity), I, make_cell(I, x, y), g);
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k * n + c] = g[k] + ws[k];
}

// Place a given state (populations f) where the next step pulls it from.
template <class S>
__global__ void k_write_pops(const Inst I, S *__restrict__ pool, int parity, const double *__restrict__ f) {
    using R = typename Real<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= I.nx || y >= I.ny) return;
    const int64_t n = (int64_t)I.nx * I.ny, c = (int64_t)y * I.nx + x;
    const double ws[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    R g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = (R)(f[k * n + c] - ws[k]);
    place_pops<S, R>(pop_buffer(pool, I, parity), I, make_cell(I, x, y), g);
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
        pull_pops<S, double>(pop_buffer(pool, I, parity), I, make_cell(I, x, y), g);
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

// Watchdog: one tile per CTA (32 x 8 cells, a thread a cell) reads every
// stored population of its cells in the instance's current buffer (each
// plane at the cell's own element: the whole buffer but its row padding)
// and sets kFlagNonFinite in the instance's status word if any is NaN or
// infinite.  A non-finite population spreads to all nine outputs of the
// next collision at its cell, so a pass every few hundred steps sees any
// instance that has diverged.
template <class S>
__global__ void __launch_bounds__(kTileX *kTileY)
    k_watch(const Inst *__restrict__ insts, const __grid_constant__ Inst I1, const int2 *__restrict__ tiles,
            const S *__restrict__ pool, const int gparity, unsigned *__restrict__ status) {
    int slot = 0, bx = blockIdx.x, by = blockIdx.y;
    const Inst *Ip = &I1;
    if (tiles) {
        const int2 t = tiles[blockIdx.x];
        slot = t.x;
        bx = t.y & 0xffff;
        by = t.y >> 16;
        Ip = insts + slot;
    }
    const Inst &I = *Ip;
    const int x = bx * kTileX + threadIdx.x, y = by * kTileY + threadIdx.y;
    bool bad = false;
    if (x < I.nx && y < I.ny) {
        const S *A = pop_buffer(pool, I, gparity ^ I.par_xor) + (y * kRowStride + col_off(I, x));
#pragma unroll
        for (int k = 0; k < 9; ++k) bad |= !isfinite(Store<S>::ld(A + k * kPlaneStride, 1.0f));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(status + slot, kFlagNonFinite);
}

}  // namespace

// ---------------------------------------------------------------- launchers
static cudaLaunchConfig_t sweep_config(dim3 grid, dim3 block, int after_beads, cudaStream_t st,
                                       cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_beads ? 1 : 0;
    return cfg;
}

// The staged sweep on blocks of NS tiles (FP32 / FP16 storage).
template <class S, int NS>
static cudaError_t launch_staged(const Inst &I, void *pool, BeadTab tab, const SweepMasks &mk, int parity,
                                 int after_beads, cudaStream_t st) {
    cudaLaunchAttribute attr[1];
    const dim3 grid(I.ntx, (I.nty + NS - 1) / NS);
    const int ec = after_beads ? mk.early_cold : 0;
    const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX / 2, kTileY), after_beads, st, attr);
    return cudaLaunchKernelEx(&cfg, k_lattice_staged<S, NS>, I, (S *)pool, tab, mk.read, mk.prev, mk.clear, parity,
                              after_beads, ec, mk.status, mk.copy_shortfall);
}

template <class S>
static cudaError_t lattice_v(int variant, const Inst &I, void *pool, BeadTab tab, const SweepMasks &mk, int parity,
                             int after_beads, cudaStream_t st) {
    cudaLaunchAttribute attr[1];
    const dim3 grid(I.ntx, I.nty);
    const int ec = after_beads ? mk.early_cold : 0;
    // constant Lallemand-Luo rates: the moment form, one cell per thread
    if (I.collision == 1) {
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX, kTileY), after_beads, st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice<S, 1, false, kCollMrt>, I, (S *)pool, tab, mk.read, mk.prev,
                                  mk.clear, parity, after_beads, ec);
    }
    if (variant == 2 && I.nx % VecWidth<S>::value == 0) {
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX / VecWidth<S>::value, kTileY), after_beads,
                                                    st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice_vec<S>, I, (S *)pool, tab, mk.read, mk.prev, mk.clear,
                                  parity, after_beads, ec);
    }
    if constexpr (AdjPairs<S>::value) {
        // the bulk copies need the buffers 16-byte aligned (strips and rows
        // are multiples of 16 bytes long)
        const bool aligned = (reinterpret_cast<uintptr_t>((S *)pool + I.pop_off) & 15u) == 0;
        if ((variant == 3 || variant == 4) && mk.status != nullptr && aligned) {
            if (variant == 3) return launch_staged<S, StagedNS<S>::value>(I, pool, tab, mk, parity, after_beads, st);
            return launch_staged<S, 2 * StagedNS<S>::value>(I, pool, tab, mk, parity, after_beads, st);
        }
    }
    if (variant == 1 || variant == 3 || variant == 4) {
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX / 2, kTileY), after_beads, st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice<S, 2, true, kCollTrt>, I, (S *)pool, tab, mk.read, mk.prev,
                                  mk.clear, parity, after_beads, ec);
    }
    const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX, kTileY), after_beads, st, attr);
    return cudaLaunchKernelEx(&cfg, k_lattice<S, 1, false, kCollTrt>, I, (S *)pool, tab, mk.read, mk.prev,
                              mk.clear, parity, after_beads, ec);
}

// The staged sweep's CTAs keep 20-46 KB of static shared memory: its
// kernels prefer the largest shared-memory carveout, so that shared memory
// does not limit the CTAs per SM before registers do.  Host-side attribute
// calls on the current device, made before any launch or stream capture.
cudaError_t prepare_lattice_kernels() {
    const void *k[] = {(const void *)k_lattice_staged<float, StagedNS<float>::value>,
                       (const void *)k_lattice_staged<float, 2 * StagedNS<float>::value>,
                       (const void *)k_lattice_staged<__half, StagedNS<__half>::value>,
                       (const void *)k_lattice_staged<__half, 2 * StagedNS<__half>::value>};
    for (const void *f : k) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_lattice(int precision, const Inst *, const Inst &inst_h, void *pool, BeadTab tab,
                           const SweepMasks &masks, int parity, int after_beads, int variant, cudaStream_t st) {
    switch (precision) {
        case 0: return lattice_v<double>(variant, inst_h, pool, tab, masks, parity, after_beads, st);
        case 1: return lattice_v<float>(variant, inst_h, pool, tab, masks, parity, after_beads, st);
        case 2: return lattice_v<__half>(variant, inst_h, pool, tab, masks, parity, after_beads, st);
    }
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t lattice_batch_v(int variant, const Inst *insts, const int2 *tiles, int ntiles, void *pool,
                                   BeadTab tab0, BeadTab tab1, const SweepMasks &mk, int gparity, int after_beads,
                                   int any_mrt, cudaStream_t st) {
    cudaLaunchAttribute attr[1];
    const dim3 grid(ntiles);
    const int ec = after_beads ? mk.early_cold : 0;
    // a batch holding instances with constant Lallemand-Luo rates: both
    // collision forms, one cell per thread
    if (any_mrt) {
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX, kTileY), after_beads, st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice_batch<S, 1, false, kCollAny>, insts, tiles, (S *)pool, tab0, tab1,
                                  mk.read, mk.prev, mk.clear, gparity, after_beads, ec);
    }
    if (variant == 2) {
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX / VecWidth<S>::value, kTileY), after_beads,
                                                    st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice_batch_vec<S>, insts, tiles, (S *)pool, tab0, tab1, mk.read,
                                  mk.prev, mk.clear, gparity, after_beads, ec);
    }
    if (variant == 1 || variant == 3 || variant == 4) {  // the staged blocks are single-lattice only
        const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX / 2, kTileY), after_beads, st, attr);
        return cudaLaunchKernelEx(&cfg, k_lattice_batch<S, 2, true, kCollTrt>, insts, tiles, (S *)pool, tab0, tab1,
                                  mk.read, mk.prev, mk.clear, gparity, after_beads, ec);
    }
    const cudaLaunchConfig_t cfg = sweep_config(grid, dim3(kTileX, kTileY), after_beads, st, attr);
    return cudaLaunchKernelEx(&cfg, k_lattice_batch<S, 1, false, kCollTrt>, insts, tiles, (S *)pool, tab0, tab1,
                              mk.read, mk.prev, mk.clear, gparity, after_beads, ec);
}

cudaError_t launch_lattice_batch(int precision, const Inst *insts, const int2 *tiles, int ntiles, void *pool,
                                 BeadTab tab0, BeadTab tab1, const SweepMasks &masks, int gparity, int after_beads,
                                 int variant, int any_mrt, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (precision) {
        case 0: return lattice_batch_v<double>(variant, insts, tiles, ntiles, pool, tab0, tab1, masks, gparity, after_beads, any_mrt, st);
        case 1: return lattice_batch_v<float>(variant, insts, tiles, ntiles, pool, tab0, tab1, masks, gparity, after_beads, any_mrt, st);
        case 2: return lattice_batch_v<__half>(variant, insts, tiles, ntiles, pool, tab0, tab1, masks, gparity, after_beads, any_mrt, st);
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

cudaError_t launch_internal_flow(int precision, const Inst &I, const void *pool, BeadTab tab, int parity,
                                 double *out, cudaStream_t st) {
    if (I.nb <= 0) return cudaSuccess;
    FPD_DISPATCH(precision, (k_internal_flow<S><<<I.nb, kFlowThreads, 0, st>>>(I, (const S *)pool, tab, parity, out)));
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

cudaError_t launch_watch(int precision, const Inst *insts, const Inst &I, const int2 *tiles, int ntiles,
                         const void *pool, int gparity, unsigned *status, cudaStream_t st) {
    const dim3 grid = tiles ? dim3(ntiles) : dim3(I.ntx, I.nty);
    if (tiles && ntiles <= 0) return cudaSuccess;
    FPD_DISPATCH(precision, (k_watch<S><<<grid, dim3(kTileX, kTileY), 0, st>>>(insts, I, tiles, (const S *)pool,
                                                                               gparity, status)));
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
