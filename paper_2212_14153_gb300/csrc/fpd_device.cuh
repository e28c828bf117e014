// fpd_device.cuh -- device-side building blocks of the FPD-MRT step:
// D2Q9 constants, the two-buffer pull population access with half-way
// moving-wall bounce-back, the bead support profile of Eq. 2 and the MRT
// collision with Guo forcing written out in moment space.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fpd {

// D2Q9 velocities in the order (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
// (-1,-1) (1,-1); weights 4/9, 1/9, 1/36.
template <int k> struct Q {
    static constexpr int cx = (k == 1 || k == 5 || k == 8) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0;
    static constexpr int cy = (k == 2 || k == 5 || k == 6) ? 1 : (k == 4 || k == 7 || k == 8) ? -1 : 0;
    static constexpr int opp = (k == 0) ? 0 : (k <= 4) ? ((k + 1) % 4 + 1) : ((k - 5 + 2) % 4 + 5);
    static constexpr double w = (k == 0) ? 4.0 / 9.0 : (k <= 4) ? 1.0 / 9.0 : 1.0 / 36.0;
};

// Population layout.  A buffer holds the nine planes of g_k in strips of
// kStripW columns: strip x / kStripW is one block of ny rows, and each row of
// a strip holds its kStripW elements of plane 0, then of plane 1, ... plane
// 8.  Element (x, y, k) sits at
//   (x / kStripW) strip + y kRowStride + k kPlaneStride + x % kStripW.
// Plane and row strides are compile-time constants, so the nine planes of a
// cell and of its y neighbours lie at immediate offsets from one address;
// only a pull across a strip edge needs the runtime strip length.  A strip is
// one lattice tile wide, so a tile's cells and their y halo are contiguous.
constexpr int kStripW = 32;
constexpr int kPlaneStride = kStripW;
constexpr int kRowStride = 9 * kStripW;

// Per-instance constants, device resident (an array of them for batches).
struct Inst {
    int32_t nx, ny, pitch, precision;  // pitch: nx rounded up to whole strips
    int64_t plane;        // elements per direction plane (pitch * ny)
    int64_t pop_off;      // element offset of this instance's planes
    double u_bot, u_top;  // wall speeds
    double nu_f, visc_ratio, a, xi, rcut, rcut2, l0;
    double gx, gy;        // uniform body force
    double k_s, k_b, k_ev;
    int32_t collision, n_beads, n_fibers, nb;
    int32_t bead_off;     // offset of this instance's beads in the tables
    int32_t strip;        // elements per strip of kStripW columns: ny kRowStride
    int32_t ntx, nty;     // lattice tiles (kTileX x kTileY cells) in x and y
    int32_t tile_base;    // first tile of this instance in the tile-mask arrays
    int32_t mask_words;   // 32-bit words per tile mask: ceil(nb / 32), >= 1
    int32_t par_xor;      // local step parity = global step parity ^ par_xor
    int32_t pad1_;
    double s_e, s_eps, s_q;
    float scale[9];       // FP16 storage: stored = (f_k - w_k) * scale[k]
    float inv_scale[9];
    // Host-precomputed terms, so that no kernel converts or divides doubles
    // per cell (FP64 throughput is a small fraction of FP32 on this GPU):
    double inv_xi;
    double bbd[2][9];     // 6 w_k c_kx u_wall, [0] bottom wall, [1] top wall
    double fluid_rates_d[4];  // s_nu, s_e, s_eps, s_q where Phi = 0
    float bbf[2][9];
    float fluid_rates_f[4];
    float f_nu_f, f_visc_m1, f_gx, f_gy, f_a, f_inv_xi, f_rcut, f_rcut2;
    float f_s_e, f_s_eps, f_s_q;
    // bead-force constants: k_s / l0^2, k_b, k_ev, l0, 1 / nx
    double ks_l02;
    float f_ks_l02, f_kb, f_kev, f_l0, f_inv_nx;
    // static solid layers of the sandwich Couette benchmark (Eq. 14)
    int32_t sandwich, pad2_;
    double sw_zl, sw_zr, half_h;
    float f_sw_zl, f_sw_zr, f_half_h;
    // periodic y without walls, and the constant external force on every
    // bead (the driven particle of Sec. 3.2)
    int32_t periodic_y;
    float f_inv_ny;
    double ext_fx, ext_fy;
    float f_ext_fx, f_ext_fy;
    // Stored units (FP16 storage keeps sigma_k g_k, sigma_k = scale[k]; the
    // other precisions sigma = 1): bounce-back terms sigma_k bbf, and per
    // weight class c (rest, axis, diagonal) sigma_c w_c, 4.5 and 3 times
    // that, for the two-relaxation-time collision in stored units
    float bbs[2][9];
    float trt_sw[3], trt_k45[3], trt_k3[3];
};

// Element offset of column x (>= 0) within its row of plane 0.
static_assert(kStripW == 32, "col_off, strip_left and strip_right shift by 5");
__device__ __forceinline__ int col_off(const Inst &I, int x) { return (x >> 5) * I.strip + (x & 31); }

// phi(y) of the sandwich layers (Eq. 14) at height y
__device__ __forceinline__ double sandwich_phi_f64(const Inst &I, double y) {
    return y <= I.half_h ? 0.5 * (tanh((I.sw_zl - y) / I.xi) + 1.0) : 0.5 * (tanh((y - I.sw_zr) / I.xi) + 1.0);
}
__device__ __forceinline__ float sandwich_phi_f32(const Inst &I, float y) {
    return y <= I.f_half_h ? 0.5f * (tanhf((I.f_sw_zl - y) * I.f_inv_xi) + 1.0f)
                           : 0.5f * (tanhf((y - I.f_sw_zr) * I.f_inv_xi) + 1.0f);
}

template <class R> __device__ __forceinline__ R bb_term(const Inst &I, int wall, int k);
template <> __device__ __forceinline__ double bb_term<double>(const Inst &I, int wall, int k) {
    return I.bbd[wall][k];
}
template <> __device__ __forceinline__ float bb_term<float>(const Inst &I, int wall, int k) {
    return I.bbf[wall][k];
}
// The same in stored units (scaled by sigma_k under FP16 storage).
template <class R> __device__ __forceinline__ R bb_stored(const Inst &I, int wall, int k);
template <> __device__ __forceinline__ double bb_stored<double>(const Inst &I, int wall, int k) {
    return I.bbd[wall][k];
}
template <> __device__ __forceinline__ float bb_stored<float>(const Inst &I, int wall, int k) {
    return I.bbs[wall][k];
}

// Bead table, structure of arrays.  FP64 state (Sec. 2.3 keeps R, V
// off-lattice) plus an FP32 copy for the reduced-precision lattice sweep:
// x wrapped into [0, nx) and both coordinates split as hi + lo floats.
struct BeadTab {
    double *Rx, *Ry, *Vx, *Vy, *Fx, *Fy, *S, *Gx, *Gy;  // G = F / S
    float *xh, *xl, *yh, *yl, *gxf, *gyf;
};
constexpr int kTabDoubles = 9;  // per bead
constexpr int kTabFloats = 6;

// ------------------------------------------------- programmatic dependent launch
// A kernel launched with programmatic stream serialization may start while
// its predecessor in the stream is still running.  Every kernel of the step
// sequence therefore touches, before pdl_wait(), only data whose producers
// are at least two launches back, and signals its own dependents only after
// pdl_wait() has returned (so the chain stays transitively ordered).  Both
// instructions are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------- storage
// ld / st convert between the stored value and g_k; ld_raw / st_raw move
// the stored value itself (sigma_k g_k), converted to the arithmetic type.
template <class T> struct Store;
template <> struct Store<double> {
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ double ld(const double *p, float) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v, float) { *p = v; }
    static __device__ __forceinline__ double ld_raw(const double *p) { return *p; }
    static __device__ __forceinline__ void st_raw(double *p, double v) { *p = v; }
    // the FP64 path keeps plain accesses
    static __device__ __forceinline__ double ld_stream(const double *p, uint64_t) { return *p; }
    static __device__ __forceinline__ void st_stream(double *p, double v, uint64_t) { *p = v; }
};
// L2 eviction priority of the population stream of a single-lattice sweep
// (createpolicy, applied per access through .L2::cache_hint).  Each element
// is read once and written once per step and one sweep moves more than the
// L2 holds; with its loads and stores marked to be evicted first, the two
// FP32 and FP16 steps measured 6.6 % and 8.8 % faster (neither mark alone
// helped; the batched sweep, whose state is many times the L2, keeps plain
// accesses, which measured faster there).
__device__ __forceinline__ uint64_t pol_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
template <> struct Store<float> {
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float ld(const float *p, float) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
    static __device__ __forceinline__ float ld_raw(const float *p) { return *p; }
    static __device__ __forceinline__ void st_raw(float *p, float v) { *p = v; }
    // population stream of a sweep: read-only during the sweep (the other
    // buffer takes the writes), both marked first to leave L2
    static __device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
        float v;
        asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
        return v;
    }
    static __device__ __forceinline__ void st_stream(float *p, float v, uint64_t pol) {
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
    }
    // two adjacent elements, p 8-byte aligned
    static __device__ __forceinline__ void ld2_raw(const float *p, float &a, float &b) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        a = t.x, b = t.y;
    }
    static __device__ __forceinline__ void st2_raw(float *p, float a, float b) {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
    static __device__ __forceinline__ void ld2_stream(const float *p, uint64_t pol, float &a, float &b) {
        asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(a), "=f"(b) : "l"(p), "l"(pol));
    }
    static __device__ __forceinline__ void st2_stream(float *p, float a, float b, uint64_t pol) {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(a), "f"(b), "l"(pol)
                     : "memory");
    }
};
template <> struct Store<__half> {
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float ld(const __half *p, float inv_scale) {
        return __half2float(*p) * inv_scale;
    }
    static __device__ __forceinline__ void st(__half *p, float v, float scale) {
        *p = __float2half_rn(v * scale);
    }
    static __device__ __forceinline__ float ld_raw(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st_raw(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float ld_stream(const __half *p, uint64_t pol) {
        unsigned short h;
        asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(h) : "l"(p), "l"(pol));
        return __half2float(__ushort_as_half(h));
    }
    static __device__ __forceinline__ void st_stream(__half *p, float v, uint64_t pol) {
        asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(__half_as_ushort(__float2half_rn(v))),
                     "l"(pol)
                     : "memory");
    }
    // two adjacent elements, p 4-byte aligned: exact widening, and one
    // packed round-to-nearest narrowing of both (each as __float2half_rn)
    static __device__ __forceinline__ void ld2_raw(const __half *p, float &a, float &b) {
        const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a = t.x, b = t.y;
    }
    static __device__ __forceinline__ void st2_raw(__half *p, float a, float b) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
    static __device__ __forceinline__ void ld2_stream(const __half *p, uint64_t pol, float &a, float &b) {
        unsigned u;
        asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
        const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&u));
        a = t.x, b = t.y;
    }
    static __device__ __forceinline__ void st2_stream(__half *p, float a, float b, uint64_t pol) {
        const __half2 h = __floats2half2_rn(a, b);
        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(*reinterpret_cast<const unsigned *>(&h)),
                     "l"(pol)
                     : "memory");
    }
};

// ------------------------------------------------------ population access
// Two buffers of 9 planes per instance (in strips, see kStripW) hold deviations g_k =
// f_k - w_k.  After t completed steps, buffer t & 1 holds the post-collision
// populations g*_k(x) of the last step at their own cell (the initial state
// is placed so that the same pull yields it).  A step pulls
//   g_k(x) = g*_k(x - c_k)                          (streaming, Sec. 2.3)
// from it, collides, and stores g*_k(x) at x in the other buffer.  A source
// beyond a wall is replaced by half-way bounce-back from the same cell:
//   g_k(x) = g*_{opp k}(x) + 6 w_k (c_k . u_w).
// Pulling costs only shifted reads; every store is aligned.  FP16 storage:
// plane k is encoded with scale[k] (scale[k] == scale[opp k]).

// Buffer `which` (0 or 1) of an instance.
template <class S>
__device__ __forceinline__ S *pop_buffer(S *pool, const Inst &I, int which) {
    return pool + I.pop_off + (which ? (int64_t)9 * I.plane : (int64_t)0);
}

// A cell as the element offset of its own element in plane 0 and the
// corrections a pull needs on top of the in-strip offset PullOff<k> (below):
// across a strip edge or the periodic wrap in x, and across the periodic
// wrap in y (walls do not wrap: a source beyond one is replaced by
// bounce-back, and bot / top mark the rows next to them).
struct Cell {
    int o;          // y kRowStride + col_off(x)
    int shl, shr;   // added for sources at x - 1 (c_kx = +1) and x + 1 (c_kx = -1)
    bool y0, yn;    // first / last row: a source beyond it wraps by ny rows when y is periodic
    bool bot, top;  // first / last fluid row next to a wall (half a cell beyond)
};
__device__ __forceinline__ Cell make_cell(const Inst &I, int x, int y) {
    Cell c;
    const int cx = col_off(I, x);
    c.o = y * kRowStride + cx;
    // in-strip offsets assume the neighbour column at cx -/+ 1
    c.shl = (x == 0) ? col_off(I, I.nx - 1) - cx + 1 : ((x & 31) == 0 ? kStripW - I.strip : 0);
    c.shr = (x == I.nx - 1) ? -cx - 1 : ((x & 31) == 31 ? I.strip - kStripW : 0);
    c.y0 = y == 0;
    c.yn = y == I.ny - 1;
    c.bot = (y == 0) && !I.periodic_y;
    c.top = (y == I.ny - 1) && !I.periodic_y;
    return c;
}

// Element offset of the pull source of direction k, x - c_k, from the
// cell's own element in plane 0, within the cell's strip.
template <int k> struct PullOff {
    static constexpr int value = k * kPlaneStride - Q<k>::cy * kRowStride - Q<k>::cx;
};
// Element offset of the source of direction k of cell C (no wall between).
template <int k> __device__ __forceinline__ int src_off(const Inst &I, const Cell &C) {
    constexpr int cx = Q<k>::cx, cy = Q<k>::cy;
    int off = C.o + PullOff<k>::value + (cx > 0 ? C.shl : (cx < 0 ? C.shr : 0));
    if (cy > 0 && C.y0) off += I.ny * kRowStride;
    if (cy < 0 && C.yn) off -= I.ny * kRowStride;
    return off;
}

// g_k(x) from the current buffer A (kRaw: in stored units, sigma_k g_k;
// kStream: with the sweep's L2 eviction priority, raw only).
template <int k, class S, class R, bool kRaw = false, bool kStream = false>
__device__ __forceinline__ void pull_one(const S *__restrict__ A, const Inst &I, const Cell &C, R &g, uint64_t pol = 0) {
    constexpr int cy = Q<k>::cy, o = Q<k>::opp;
    // source cell x - c_k; beyond a wall when it is row -1 or row ny
    const bool wall = (cy > 0 && C.bot) || (cy < 0 && C.top);
    if (wall) {
        const S *p = A + (C.o + o * kPlaneStride);
        if constexpr (kRaw && kStream) g = (R)Store<S>::ld_stream(p, pol) + bb_stored<R>(I, cy > 0 ? 0 : 1, k);
        else if constexpr (kRaw) g = (R)Store<S>::ld_raw(p) + bb_stored<R>(I, cy > 0 ? 0 : 1, k);
        else g = (R)Store<S>::ld(p, I.inv_scale[o]) + bb_term<R>(I, cy > 0 ? 0 : 1, k);
    } else {
        const S *p = A + src_off<k>(I, C);
        if constexpr (kRaw && kStream) g = (R)Store<S>::ld_stream(p, pol);
        else if constexpr (kRaw) g = (R)Store<S>::ld_raw(p);
        else g = (R)Store<S>::ld(p, I.inv_scale[k]);
    }
}

// Inverse of pull_one: store g so that the next pull of direction k at x
// yields it (initial state, writes of a given state).
template <int k, class S, class R>
__device__ __forceinline__ void place_one(S *__restrict__ A, const Inst &I, const Cell &C, R g) {
    constexpr int cy = Q<k>::cy, o = Q<k>::opp;
    const bool wall = (cy > 0 && C.bot) || (cy < 0 && C.top);
    if (wall) {
        Store<S>::st(A + (C.o + o * kPlaneStride), g - bb_term<R>(I, cy > 0 ? 0 : 1, k), I.scale[o]);
    } else {
        Store<S>::st(A + src_off<k>(I, C), g, I.scale[k]);
    }
}

template <class S, class R, bool kRaw = false, bool kStream = false>
__device__ __forceinline__ void pull_pops(const S *__restrict__ A, const Inst &I, const Cell &C, R g[9], uint64_t pol = 0) {
    // grouped by the x shift of the source (c_kx = 0, +1, -1)
    pull_one<0, S, R, kRaw, kStream>(A, I, C, g[0], pol);
    pull_one<2, S, R, kRaw, kStream>(A, I, C, g[2], pol);
    pull_one<4, S, R, kRaw, kStream>(A, I, C, g[4], pol);
    pull_one<1, S, R, kRaw, kStream>(A, I, C, g[1], pol);
    pull_one<5, S, R, kRaw, kStream>(A, I, C, g[5], pol);
    pull_one<8, S, R, kRaw, kStream>(A, I, C, g[8], pol);
    pull_one<3, S, R, kRaw, kStream>(A, I, C, g[3], pol);
    pull_one<6, S, R, kRaw, kStream>(A, I, C, g[6], pol);
    pull_one<7, S, R, kRaw, kStream>(A, I, C, g[7], pol);
}

template <int k, class S, class R, bool kRaw, bool kStream>
__device__ __forceinline__ void pull_inner_one(const S *__restrict__ p, const Inst &I, R &g, uint64_t pol) {
    const S *q = p + PullOff<k>::value;
    if constexpr (kRaw && kStream) g = (R)Store<S>::ld_stream(q, pol);
    else if constexpr (kRaw) g = (R)Store<S>::ld_raw(q);
    else g = (R)Store<S>::ld(q, I.inv_scale[k]);
}
// Pull of all nine directions for a cell with no wall and no periodic wrap
// among its neighbours; p points at the cell's element in plane 0.  A source
// left of the strip (c_kx = +1 from its first column) is reached from
// pl = p + shl, one right of it (c_kx = -1 from its last column) from
// pr = p + shr: shl and shr (strip_left, strip_right) shift by a strip less
// or more one row of a plane there, and are 0 elsewhere.
template <class S, class R, bool kRaw = false, bool kStream = false>
__device__ __forceinline__ void pull_inner(const S *__restrict__ p, const int shl, const int shr, const Inst &I,
                                           R g[9], uint64_t pol = 0) {
    pull_inner_one<0, S, R, kRaw, kStream>(p, I, g[0], pol);
    pull_inner_one<2, S, R, kRaw, kStream>(p, I, g[2], pol);
    pull_inner_one<4, S, R, kRaw, kStream>(p, I, g[4], pol);
    const S *pl = p + shl;
    pull_inner_one<1, S, R, kRaw, kStream>(pl, I, g[1], pol);
    pull_inner_one<5, S, R, kRaw, kStream>(pl, I, g[5], pol);
    pull_inner_one<8, S, R, kRaw, kStream>(pl, I, g[8], pol);
    const S *pr = p + shr;
    pull_inner_one<3, S, R, kRaw, kStream>(pr, I, g[3], pol);
    pull_inner_one<6, S, R, kRaw, kStream>(pr, I, g[6], pol);
    pull_inner_one<7, S, R, kRaw, kStream>(pr, I, g[7], pol);
}
static_assert(Q<1>::cx > 0 && Q<5>::cx > 0 && Q<8>::cx > 0 && Q<3>::cx < 0 && Q<6>::cx < 0 && Q<7>::cx < 0 &&
                  Q<0>::cx == 0 && Q<2>::cx == 0 && Q<4>::cx == 0,
              "pull_inner's choice of base pointer per direction");
// Shifts of pull_inner's pl and pr for column x (an element offset from p).
__device__ __forceinline__ int strip_left(const Inst &I, int x) { return (x & 31) == 0 ? kStripW - I.strip : 0; }
__device__ __forceinline__ int strip_right(const Inst &I, int x) { return (x & 31) == 31 ? I.strip - kStripW : 0; }

// Two x-adjacent cells a (even column, element p in plane 0) and b = a + 1
// with no wall and no periodic wrap among their neighbours, in stored
// units: a direction with c_kx = 0 pulls both from adjacent elements (one
// paired access); c_kx = +1 pulls a from column x - 1 (p + shl across the
// strip's left edge) and b from a's column; c_kx = -1 pulls a from b's
// column and b from x + 2 (p + 1 + shr across the right edge).
template <class S, bool kStream> __device__ __forceinline__ float ld1(const S *q, uint64_t pol) {
    if constexpr (kStream) return Store<S>::ld_stream(q, pol);
    else return Store<S>::ld_raw(q);
}
template <int k, class S, bool kStream>
__device__ __forceinline__ void pull_adj_one(const S *__restrict__ p, int shl, int shr, float ga[9], float gb[9],
                                             uint64_t pol) {
    constexpr int cx = Q<k>::cx, off = PullOff<k>::value;
    if constexpr (cx == 0) {
        if constexpr (kStream) Store<S>::ld2_stream(p + off, pol, ga[k], gb[k]);
        else Store<S>::ld2_raw(p + off, ga[k], gb[k]);
    } else if constexpr (cx > 0) {
        ga[k] = ld1<S, kStream>(p + shl + off, pol);
        gb[k] = ld1<S, kStream>(p + 1 + off, pol);
    } else {
        ga[k] = ld1<S, kStream>(p + off, pol);
        gb[k] = ld1<S, kStream>(p + 1 + shr + off, pol);
    }
}
template <class S, bool kStream>
__device__ __forceinline__ void pull_adj(const S *__restrict__ p, int shl, int shr, float ga[9], float gb[9],
                                         uint64_t pol) {
    pull_adj_one<0, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<2, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<4, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<1, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<5, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<8, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<3, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<6, S, kStream>(p, shl, shr, ga, gb, pol);
    pull_adj_one<7, S, kStream>(p, shl, shr, ga, gb, pol);
}
// Post-collision populations of two x-adjacent cells, p (even column) in
// plane 0, one paired store per plane.
template <class S, bool kStream>
__device__ __forceinline__ void put_adj(S *__restrict__ p, const float ga[9], const float gb[9], uint64_t pol) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if constexpr (kStream) Store<S>::st2_stream(p + k * kPlaneStride, ga[k], gb[k], pol);
        else Store<S>::st2_raw(p + k * kPlaneStride, ga[k], gb[k]);
    }
}

// Post-collision populations stored at the cell whose plane-0 element p is.
template <class S, class R, bool kRaw = false, bool kStream = false>
__device__ __forceinline__ void put_at(S *__restrict__ p, const Inst &I, const R g[9], uint64_t pol = 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if constexpr (kRaw && kStream) Store<S>::st_stream(p + k * kPlaneStride, g[k], pol);
        else if constexpr (kRaw) Store<S>::st_raw(p + k * kPlaneStride, g[k]);
        else Store<S>::st(p + k * kPlaneStride, g[k], I.scale[k]);
    }
}

template <class S, class R>
__device__ __forceinline__ void place_pops(S *__restrict__ A, const Inst &I, const Cell &C, const R g[9]) {
    place_one<0>(A, I, C, g[0]);
    place_one<1>(A, I, C, g[1]);
    place_one<2>(A, I, C, g[2]);
    place_one<3>(A, I, C, g[3]);
    place_one<4>(A, I, C, g[4]);
    place_one<5>(A, I, C, g[5]);
    place_one<6>(A, I, C, g[6]);
    place_one<7>(A, I, C, g[7]);
    place_one<8>(A, I, C, g[8]);
}

// ---------------------------------------------------------------- Eq. 2
// Minimum-image separation in x and the hard support cutoff, with every
// rounding spelled out (no contraction), so that the cutoff decision and the
// distance equal those of a plain IEEE evaluation.
__device__ __forceinline__ double min_image_rn(double d, double L) {
    return __dsub_rn(d, __dmul_rn(L, floor(__dadd_rn(__ddiv_rn(d, L), 0.5))));
}

// phi_i at cell centre (xc, yc) of bead (Rx, Ry); 0 beyond the cutoff.
// Minimum image in x, and in y when the lattice is periodic in y.
__device__ __forceinline__ double phi_f64(const Inst &I, double xc, double yc, double Rx, double Ry) {
    const double dx = min_image_rn(__dsub_rn(xc, Rx), (double)I.nx);
    double dy = __dsub_rn(yc, Ry);
    if (I.periodic_y) dy = min_image_rn(dy, (double)I.ny);
    const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (!(r2 < I.rcut2)) return 0.0;
    const double r = sqrt(r2);
    return 0.5 * (tanh((I.a - r) / I.xi) + 1.0);
}

// Cells whose centre may lie within the cutoff of (Rx, Ry): a box that wraps
// periodically in x (and in y when y is periodic), or spans that direction
// once, and is clipped at the walls otherwise.  (iu, ju) are the unwrapped
// indices of its first column and row (column c, row r sit at iu + c, ju + r);
// (i0, j0) the same wrapped into the lattice.
struct Box {
    int i0, j0, w, h;
    double iu, ju;
};

// Rows [lo, hi] of a box: wrapped (periodic y; spanning the lattice once at
// most, starting at span_lo when it would wrap onto itself) or clipped at the
// walls.  Returns false when no row is left.
__device__ __forceinline__ bool box_rows(const Inst &I, long long lo, long long hi, long long span_lo, Box &b) {
    if (I.periodic_y) {
        if (hi - lo + 1 >= I.ny) {
            lo = span_lo;
            hi = lo + I.ny - 1;
        }
        b.ju = (double)lo;
        b.j0 = (int)(((lo % I.ny) + I.ny) % I.ny);
        b.h = (int)(hi - lo + 1);
        return true;
    }
    lo = lo < 0 ? 0 : lo;
    hi = hi > I.ny - 1 ? I.ny - 1 : hi;
    if (hi < lo) return false;
    b.ju = (double)lo;
    b.j0 = (int)lo;
    b.h = (int)(hi - lo + 1);
    return true;
}

__device__ __forceinline__ Box support_box(const Inst &I, double Rx, double Ry) {
    Box b;
    b.i0 = b.j0 = b.w = b.h = 0;
    b.iu = b.ju = 0.0;
    // a non-finite or far-away bead has no support cells (the NaN then shows
    // up in the diagnostics, not as an out-of-range index)
    if (!isfinite(Rx) || !isfinite(Ry) || fabs(Rx) > 1.0e9 || fabs(Ry) > 1.0e9) return b;
    if (fabs(Rx) < 1.0e6 && fabs(Ry) < 1.0e6) {
        // bounds with one cell of margin: FP32 rounding (< 0.07 here) cannot
        // drop a cell whose centre lies within the cutoff
        const float rx = (float)Rx, ry = (float)Ry, rc = I.f_rcut;
        const int ylo = (int)floorf(ry - rc - 0.5f) - 1;
        const int yhi = (int)ceilf(ry + rc - 0.5f) + 1;
        int xlo = (int)floorf(rx - rc - 0.5f) - 1;
        int xhi = (int)ceilf(rx + rc - 0.5f) + 1;
        if (xhi - xlo + 1 >= I.nx) {
            xlo = (int)floorf(rx - 0.5f * (float)I.nx);
            xhi = xlo + I.nx - 1;
        }
        if (!box_rows(I, ylo, yhi, (long long)floorf(ry - 0.5f * (float)I.ny), b)) return b;
        b.iu = (double)xlo;
        b.i0 = ((xlo % I.nx) + I.nx) % I.nx;  // in [0, nx)
        b.w = xhi - xlo + 1;
        return b;
    }
    const long long ylo = (long long)floor(Ry - I.rcut - 0.5) - 1, yhi = (long long)ceil(Ry + I.rcut - 0.5) + 1;
    if (!box_rows(I, ylo, yhi, (long long)floor(Ry - 0.5 * I.ny), b)) return b;
    const double xl = floor(Rx - I.rcut - 0.5) - 1.0, xh = ceil(Rx + I.rcut - 0.5) + 1.0;
    if (xh - xl + 1.0 >= (double)I.nx) {
        const double x0 = floor(Rx - 0.5 * I.nx);
        b.iu = x0;
        const long long xi = (long long)x0;
        b.i0 = (int)(((xi % I.nx) + I.nx) % I.nx);
        b.w = I.nx;
    } else {
        b.iu = xl;
        const long long xi = (long long)xl;
        b.i0 = (int)(((xi % I.nx) + I.nx) % I.nx);
        b.w = (int)(xh - xl) + 1;
    }
    return b;
}

// FP32 variant for the reduced-precision lattice path: dx, dy relative to a
// tile origin already reduced to small numbers by the caller.
__device__ __forceinline__ float phi_f32(float dx, float dy, float a, float inv_xi, float rcut2) {
    const float r2 = dx * dx + dy * dy;
    if (!(r2 < rcut2)) return 0.0f;
    const float r = sqrtf(r2);
    return 0.5f * (tanhf((a - r) * inv_xi) + 1.0f);
}

// ---------------------------------------------------------------- collision
// MRT collision with Guo forcing on deviations g_k = f_k - w_k (rho_0 = 1).
// Moments in the Lallemand-Luo basis (rho, e, eps, jx, qx, jy, qy, pxx, pxy),
// with m = M g + (1, -2, 1, 0, ...).  With u = (j + F/2) / rho:
//   m* = m - S (m - m_eq) + (I - S/2) M F_guo,   g* = M^-1 (m* - m_rest),
// M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
// Rates: s_e, s_eps, s_q as given, s_nu from the local viscosity.
// 1 / rho.  rho stays within a few per cent of 1, far from subnormals, so
// the FP32 path takes the hardware's approximate reciprocal (one
// instruction, within about an ulp); the FP64 path divides.
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <class R>
__device__ __forceinline__ void collide(R g[9], R Fx, R Fy, R s_nu, R s_e, R s_eps, R s_q) {
    const R g1 = g[1], g2 = g[2], g3 = g[3], g4 = g[4];
    const R g5 = g[5], g6 = g[6], g7 = g[7], g8 = g[8];
    const R ax = g1 + g2 + g3 + g4, dg = g5 + g6 + g7 + g8;
    const R drho = g[0] + ax + dg;
    const R e = (R)-4 * g[0] - ax + (R)2 * dg;
    const R eps = (R)4 * g[0] - (R)2 * ax + dg;
    const R d57 = g5 - g7, d68 = g6 - g8;
    const R jx = g1 - g3 + d57 - d68;
    const R jy = g2 - g4 + d57 + d68;
    const R qx = (R)-2 * (g1 - g3) + d57 - d68;
    const R qy = (R)-2 * (g2 - g4) + d57 + d68;
    const R pxx = g1 - g2 + g3 - g4;
    const R pxy = g5 - g6 + g7 - g8;

    const R rho = (R)1 + drho;
    const R irho = recip(rho);
    const R ux = (jx + (R)0.5 * Fx) * irho;
    const R uy = (jy + (R)0.5 * Fy) * irho;
    const R rux = rho * ux, ruy = rho * uy;
    const R u2r = rho * (ux * ux + uy * uy);
    const R uF = ux * Fx + uy * Fy;

    // post-collision deviation moments
    const R e_s = e - s_e * (e + (R)2 * drho - (R)3 * u2r) + ((R)1 - (R)0.5 * s_e) * (R)6 * uF;
    const R eps_s = eps - s_eps * (eps - drho + (R)3 * u2r) - ((R)1 - (R)0.5 * s_eps) * (R)6 * uF;
    const R jx_s = jx + Fx;
    const R jy_s = jy + Fy;
    const R qx_s = qx - s_q * (qx + rux) - ((R)1 - (R)0.5 * s_q) * Fx;
    const R qy_s = qy - s_q * (qy + ruy) - ((R)1 - (R)0.5 * s_q) * Fy;
    const R hn = (R)1 - (R)0.5 * s_nu;
    const R pxx_s = pxx - s_nu * (pxx - rux * ux + ruy * uy) + hn * (R)2 * (ux * Fx - uy * Fy);
    const R pxy_s = pxy - s_nu * (pxy - rux * uy) + hn * (ux * Fy + uy * Fx);

    // back to populations: g*_k = sum_r M[r][k] m*_r / |M_r|^2
    const R a0 = drho * (R)(1.0 / 9.0);
    const R a1 = e_s * (R)(1.0 / 36.0);
    const R a2 = eps_s * (R)(1.0 / 36.0);
    const R a3 = jx_s * (R)(1.0 / 6.0);
    const R a4 = qx_s * (R)(1.0 / 12.0);
    const R a5 = jy_s * (R)(1.0 / 6.0);
    const R a6 = qy_s * (R)(1.0 / 12.0);
    const R a7 = pxx_s * (R)0.25;
    const R a8 = pxy_s * (R)0.25;

    const R base_ax = a0 - a1 - (R)2 * a2;
    const R base_dg = a0 + (R)2 * a1 + a2;
    const R xa = a3 - (R)2 * a4, ya = a5 - (R)2 * a6;
    const R xd = a3 + a4, yd = a5 + a6;
    g[0] = a0 - (R)4 * a1 + (R)4 * a2;
    g[1] = base_ax + xa + a7;
    g[2] = base_ax + ya - a7;
    g[3] = base_ax - xa + a7;
    g[4] = base_ax - ya - a7;
    g[5] = base_dg + xd + yd + a8;
    g[6] = base_dg - xd + yd - a8;
    g[7] = base_dg - xd - yd + a8;
    g[8] = base_dg + xd - yd - a8;
}

// The same collision in two-relaxation-time form for an unforced cell, for
// the rate sets in which every even non-conserved moment (e, eps, p_xx,
// p_xy) relaxes at one rate sp = s_nu and every odd one (q_x, q_y) at
// sm = s_q: the magic rates (s_e = s_eps = s_nu) and BGK.  There the
// moment-space update above with F = 0 is, in exact arithmetic, the
// link-pair update
//   g*_k = g_k - sp (g+_k - eq+_k) - sm (g-_k - eq-_k)
// with g+-_k = (g_k +- g_opp k) / 2 and the even and odd parts of the
// quadratic equilibrium (deviation form, rho_0 = 1)
//   eq+_k = w_k [(rho - 1) + rho (9/2 (c_k.u)^2 - 3/2 u^2)],  eq-_k = 3 w_k rho c_k.u,
// u = sum_k g_k c_k / rho.  It works on stored values x_k = sigma_k g_k
// (sigma = 1 unless FP16 storage; one sigma per weight class) and returns
// stored values, so the FP16 path needs no per-population rescaling, and it
// keeps only the pair sums and differences live: about 60 operations per
// cell against ~115 for the moment form.
// Correctly rounded arithmetic on one value or on a pair of FP32 values.
// The pair form issues one packed instruction (f32x2) for both lanes, and
// each lane rounds exactly as the scalar form does, so a thread that
// advances two cells with it gets the bits each cell gets alone.  Every
// operation is spelled out (no contraction left to the compiler).
template <class V> struct Ar;
template <> struct Ar<double> {
    static __device__ __forceinline__ double c(double a) { return a; }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double d) { return __fma_rn(a, b, d); }
    static __device__ __forceinline__ double rcp(double a) { return recip(a); }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float c(float a) { return a; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float d) { return __fmaf_rn(a, b, d); }
    static __device__ __forceinline__ float rcp(float a) { return recip(a); }
};
template <> struct Ar<float2> {
    static __device__ __forceinline__ float2 c(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b as fma(b, -1, a): one rounding of the exact difference, as __fsub_rn
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 d) { return __ffma2_rn(a, b, d); }
    static __device__ __forceinline__ float2 rcp(float2 a) { return make_float2(recip(a.x), recip(a.y)); }
};

template <class R, bool kScaled, class V>
__device__ __forceinline__ void collide_trt(V x[9], V sp, V sm, const Inst &I) {
    using A = Ar<V>;
    // per weight class c = 0 (rest), 1 (axis), 2 (diagonal): sigma_c w_c
    // and multiples, and 1 / sigma_c
    V sw0, sw1, sw2, k45_1, k45_2, k3_1, k3_2, i0, i1, i2;
    if constexpr (kScaled) {
        sw0 = A::c(I.trt_sw[0]), sw1 = A::c(I.trt_sw[1]), sw2 = A::c(I.trt_sw[2]);
        k45_1 = A::c(I.trt_k45[1]), k45_2 = A::c(I.trt_k45[2]);
        k3_1 = A::c(I.trt_k3[1]), k3_2 = A::c(I.trt_k3[2]);
        i0 = A::c(I.inv_scale[0]), i1 = A::c(I.inv_scale[1]), i2 = A::c(I.inv_scale[5]);
    } else {
        sw0 = A::c((R)(4.0 / 9.0)), sw1 = A::c((R)(1.0 / 9.0)), sw2 = A::c((R)(1.0 / 36.0));
        k45_1 = A::c((R)0.5), k45_2 = A::c((R)0.125), k3_1 = A::c((R)(1.0 / 3.0)), k3_2 = A::c((R)(1.0 / 12.0));
        i0 = i1 = i2 = A::c((R)1);  // unused
    }
    const V one = A::c((R)1), half = A::c((R)0.5), mhalf = A::c((R)-0.5);
    // link pairs: a = x_k + x_opp = 2 sigma g+_k, b = x_k - x_opp = 2 sigma g-_k
    const V a13 = A::add(x[1], x[3]), b13 = A::sub(x[1], x[3]);
    const V a24 = A::add(x[2], x[4]), b24 = A::sub(x[2], x[4]);
    const V a57 = A::add(x[5], x[7]), b57 = A::sub(x[5], x[7]);
    const V a68 = A::add(x[6], x[8]), b68 = A::sub(x[6], x[8]);
    V drho, jx, jy;
    if constexpr (kScaled) {
        drho = A::fma(i2, A::add(a57, a68), A::fma(i1, A::add(a13, a24), A::mul(i0, x[0])));
        jx = A::fma(i2, A::sub(b57, b68), A::mul(i1, b13));
        jy = A::fma(i2, A::add(b57, b68), A::mul(i1, b24));
    } else {
        drho = A::add(A::add(x[0], A::add(a13, a24)), A::add(a57, a68));
        jx = A::add(b13, A::sub(b57, b68));
        jy = A::add(b24, A::add(b57, b68));
    }
    const V rho = A::add(one, drho);
    const V irho = A::rcp(rho);
    const V ux = A::mul(jx, irho), uy = A::mul(jy, irho);
    // sigma eq+_k = sigma w D + 4.5 sigma w rho (c.u)^2, D = rho - 1 - 1.5 rho u^2;
    // sigma eq-_k = 3 sigma w rho c.u; here already times the rates
    const V D = A::fma(A::c((R)-1.5), A::mul(rho, A::fma(ux, ux, A::mul(uy, uy))), drho);
    const V spD = A::mul(sp, D), spr = A::mul(sp, rho), smr = A::mul(sm, rho);
    const V es1 = A::mul(sw1, spD), es2 = A::mul(sw2, spD);
    const V qs1 = A::mul(k45_1, spr), qs2 = A::mul(k45_2, spr);
    const V ts1 = A::mul(k3_1, smr), ts2 = A::mul(k3_2, smr);
    const V c1 = A::fma(mhalf, sp, half), c2 = A::fma(mhalf, sm, half);
    // rest population: x0 - sp (x0 - sigma_0 w_0 D)
    x[0] = A::fma(A::sub(one, sp), x[0], A::mul(sw0, spD));
    // each pair: the even half (a/2) and the odd half (b/2) relax separately,
    //   A = a/2 - sp (a/2 - sigma eq+),  B = b/2 - sm (b/2 - sigma eq-),
    // and x*_k = A + B, x*_opp = A - B
    auto pair = [&](int k, int ko, V cu, V a, V b, V es, V qs, V ts) {
        const V ev = A::fma(c1, a, A::fma(qs, A::mul(cu, cu), es));
        const V od = A::fma(c2, b, A::mul(ts, cu));
        x[k] = A::add(ev, od);
        x[ko] = A::sub(ev, od);
    };
    pair(1, 3, ux, a13, b13, es1, qs1, ts1);
    pair(2, 4, uy, a24, b24, es1, qs1, ts1);
    pair(5, 7, A::add(ux, uy), a57, b57, es2, qs2, ts2);
    pair(6, 8, A::sub(uy, ux), a68, b68, es2, qs2, ts2);
}

// Relaxation rates of one cell from its kinematic viscosity (Eq. 1 gives nu).
template <class R>
__device__ __forceinline__ void rates(int collision, R nu, R s_e_ll, R s_eps_ll, R s_q_ll, R &s_nu, R &s_e,
                                      R &s_eps, R &s_q) {
    s_nu = (R)1 / ((R)3 * nu + (R)0.5);
    if (collision == 1) {
        s_e = s_e_ll;
        s_eps = s_eps_ll;
        s_q = s_q_ll;
    } else if (collision == 2) {
        s_e = s_eps = s_q = s_nu;
    } else {
        s_e = s_eps = s_nu;
        s_q = (R)1 / ((R)0.5 + (R)0.1875 / ((R)1 / s_nu - (R)0.5));
    }
}

}  // namespace fpd
