// fpd_api.cu -- the C ABI declared in include/fpd.h: parameter validation and
// derivation, device state ownership, the per-step launch sequence, reads.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fpd.h"
#include "fpd_kernels.h"
#include "fpd_sim.h"

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace {

int fail(fpd_sim *s, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(fpd_sim *s, cudaError_t e, const char *what) {
    return fail(s, FPD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t elem_size(int precision) { return precision == 0 ? 8 : (precision == 1 ? 4 : 2); }

bool is_fin(double v) { return std::isfinite(v); }

// Validate p and fill the derived constants (Sec. 2.3 and Eq. 18).
int derive(fpd_sim *s, const fpd_params &p) {
    if (p.nx < 1 || p.ny < 1) return fail(nullptr, FPD_EINVAL, "nx and ny must be >= 1 (got %d, %d)", p.nx, p.ny);
    if ((int64_t)p.nx * p.ny > (int64_t)1 << 31)
        return fail(nullptr, FPD_EINVAL, "lattice of %d x %d cells is too large", p.nx, p.ny);
    if (p.precision < 0 || p.precision > 2) return fail(nullptr, FPD_EINVAL, "precision must be 0, 1 or 2");
    if (p.collision < 0 || p.collision > 2) return fail(nullptr, FPD_EINVAL, "collision must be 0, 1 or 2");
    if (p.n_beads < 0 || p.n_fibers < 0) return fail(nullptr, FPD_EINVAL, "n_beads and n_fibers must be >= 0");
    const int nb = p.n_beads * p.n_fibers;
    if (nb > fpd::kMaxBeads)
        return fail(nullptr, FPD_EINVAL, "at most %d beads per simulation (got %d)", fpd::kMaxBeads, nb);
    if (!is_fin(p.u_bottom) || !is_fin(p.u_top) || !is_fin(p.body_force_x) || !is_fin(p.body_force_y))
        return fail(nullptr, FPD_EINVAL, "wall speeds and body force must be finite");
    if (!is_fin(p.bead_force_x) || !is_fin(p.bead_force_y))
        return fail(nullptr, FPD_EINVAL, "bead_force must be finite");
    if (p.periodic_y != 0 && p.periodic_y != 1) return fail(nullptr, FPD_EINVAL, "periodic_y must be 0 or 1");
    if (p.periodic_y && p.sandwich_zl > 0.0)
        return fail(nullptr, FPD_EINVAL, "the sandwich layers need walls (periodic_y = 0)");
    const double l0 = 2.0 * p.bead_radius;
    const double gd = (p.u_top - p.u_bottom) / (double)p.ny;
    const double lc = p.n_beads * l0;
    double nu = p.nu_f;
    if (!(nu > 0.0)) {
        if (!(p.re > 0.0) || !(std::fabs(gd) > 0.0) || !(lc > 0.0))
            return fail(nullptr, FPD_EINVAL,
                        "nu_f <= 0 needs re > 0, moving walls and a fiber to derive nu_f = gamma_dot l_c^2 / re");
        nu = std::fabs(gd) * lc * lc / p.re;
    }
    if (!is_fin(nu) || nu <= 0.0) return fail(nullptr, FPD_EINVAL, "fluid viscosity must be positive");
    if (!(p.visc_ratio > 0.0) || !is_fin(p.visc_ratio)) return fail(nullptr, FPD_EINVAL, "visc_ratio must be > 0");
    if (nb > 0) {
        if (!(p.bead_radius > 0.0)) return fail(nullptr, FPD_EINVAL, "bead_radius must be > 0");
        if (!(p.xi > 0.0)) return fail(nullptr, FPD_EINVAL, "xi must be > 0");
        if (!(p.phi_cut > 0.0)) return fail(nullptr, FPD_EINVAL, "phi_cut must be > 0");
        if (!p.bead_xy && (!p.centre_xy || !p.theta0))
            return fail(nullptr, FPD_EINVAL, "fibers need centre_xy and theta0, or bead_xy");
    }
    s->nu_f = nu;
    s->gamma_dot = gd;
    s->k_s = (p.k_s < 0.0) ? 0.25 * M_PI * p.bead_radius * p.bead_radius * l0 * l0 : p.k_s;
    s->k_b = (p.stiffness_K > 0.0) ? p.stiffness_K * nu * std::fabs(gd) * lc * lc / 2.0 : p.k_b;
    s->k_ev = (p.k_ev < 0.0) ? s->k_s / (l0 * l0) : p.k_ev;

    fpd::Inst &I = s->inst;
    std::memset(&I, 0, sizeof I);
    I.nx = p.nx;
    I.ny = p.ny;
    // populations in strips of kStripW columns (fpd_device.cuh): the width is
    // padded to whole strips
    I.pitch = (p.nx + fpd::kStripW - 1) / fpd::kStripW * fpd::kStripW;
    I.precision = p.precision;
    I.plane = (int64_t)I.pitch * p.ny;
    if (9 * I.plane > (int64_t)INT32_MAX)
        return fail(nullptr, FPD_EINVAL, "lattice of %d x %d cells exceeds 32-bit element offsets", p.nx, p.ny);
    I.strip = p.ny * fpd::kRowStride;
    I.pop_off = 0;
    I.ntx = (p.nx + fpd::kTileX - 1) / fpd::kTileX;
    I.nty = (p.ny + fpd::kTileY - 1) / fpd::kTileY;
    I.tile_base = 0;
    I.mask_words = nb > 0 ? (nb + 31) / 32 : 1;
    I.u_bot = p.u_bottom;
    I.u_top = p.u_top;
    I.nu_f = nu;
    I.visc_ratio = p.visc_ratio;
    I.a = p.bead_radius;
    I.xi = p.xi > 0 ? p.xi : 1.0;
    I.rcut = p.bead_radius + p.phi_cut * I.xi;
    I.rcut2 = I.rcut * I.rcut;
    I.l0 = l0;
    I.gx = p.body_force_x;
    I.gy = p.body_force_y;
    I.k_s = s->k_s;
    I.k_b = s->k_b;
    I.k_ev = s->k_ev;
    I.collision = p.collision;
    I.n_beads = p.n_beads;
    I.n_fibers = p.n_fibers;
    I.nb = nb;
    I.bead_off = 0;
    I.s_e = p.s_e;
    I.s_eps = p.s_eps;
    I.s_q = p.s_q;
    // host-precomputed FP32 copies, bounce-back terms and fluid rates
    I.inv_xi = 1.0 / I.xi;
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const double wk[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                          1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    for (int k = 0; k < 9; ++k) {
        I.bbd[0][k] = 6.0 * wk[k] * cx[k] * p.u_bottom;
        I.bbd[1][k] = 6.0 * wk[k] * cx[k] * p.u_top;
        I.bbf[0][k] = (float)I.bbd[0][k];
        I.bbf[1][k] = (float)I.bbd[1][k];
    }
    {
        const double s_nu = 1.0 / (3.0 * nu + 0.5);
        double se = s_nu, seps = s_nu, sq = 1.0 / (0.5 + 0.1875 / (1.0 / s_nu - 0.5));
        if (p.collision == 1) {
            se = p.s_e;
            seps = p.s_eps;
            sq = p.s_q;
        } else if (p.collision == 2) {
            sq = s_nu;
        }
        const double r4[4] = {s_nu, se, seps, sq};
        for (int i = 0; i < 4; ++i) {
            I.fluid_rates_d[i] = r4[i];
            I.fluid_rates_f[i] = (float)r4[i];
        }
        // FP32 fluid rates evaluated in FP32 like the per-cell path does
        const float fnu = (float)nu;
        const float fs_nu = 1.0f / (3.0f * fnu + 0.5f);
        I.fluid_rates_f[0] = fs_nu;
        if (p.collision == 0) {
            I.fluid_rates_f[1] = I.fluid_rates_f[2] = fs_nu;
            I.fluid_rates_f[3] = 1.0f / (0.5f + 0.1875f / (1.0f / fs_nu - 0.5f));
        } else if (p.collision == 2) {
            I.fluid_rates_f[1] = I.fluid_rates_f[2] = I.fluid_rates_f[3] = fs_nu;
        } else {
            I.fluid_rates_f[1] = (float)p.s_e;
            I.fluid_rates_f[2] = (float)p.s_eps;
            I.fluid_rates_f[3] = (float)p.s_q;
        }
    }
    I.f_nu_f = (float)nu;
    I.f_visc_m1 = (float)(p.visc_ratio - 1.0);
    I.f_gx = (float)p.body_force_x;
    I.f_gy = (float)p.body_force_y;
    I.f_a = (float)I.a;
    I.f_inv_xi = (float)I.inv_xi;
    I.f_rcut = (float)I.rcut;
    I.f_rcut2 = (float)I.rcut2;
    if (p.sandwich_zl > 0.0) {
        if (!(p.xi > 0.0)) return fail(nullptr, FPD_EINVAL, "sandwich layers need xi > 0");
        if (!(p.sandwich_zr > p.sandwich_zl)) return fail(nullptr, FPD_EINVAL, "sandwich_zr must exceed sandwich_zl");
        I.sandwich = 1;
        I.sw_zl = p.sandwich_zl;
        I.sw_zr = p.sandwich_zr;
        I.half_h = 0.5 * p.ny;
        I.f_sw_zl = (float)p.sandwich_zl;
        I.f_sw_zr = (float)p.sandwich_zr;
        I.f_half_h = (float)I.half_h;
    }
    I.periodic_y = p.periodic_y;
    I.f_inv_ny = (float)(1.0 / p.ny);
    I.ext_fx = p.bead_force_x;
    I.ext_fy = p.bead_force_y;
    I.f_ext_fx = (float)p.bead_force_x;
    I.f_ext_fy = (float)p.bead_force_y;
    I.ks_l02 = s->k_s / (l0 * l0);
    I.f_ks_l02 = (float)I.ks_l02;
    I.f_kb = (float)s->k_b;
    I.f_kev = (float)s->k_ev;
    I.f_l0 = (float)l0;
    I.f_inv_nx = (float)(1.0 / p.nx);
    I.f_s_e = (float)p.s_e;
    I.f_s_eps = (float)p.s_eps;
    I.f_s_q = (float)p.s_q;
    // FP16 storage scale: a power of two per plane (symmetric under k ->
    // opp k) mapping w_k (6 U + 0.01), a bound of |f_k - w_k|, to 2^10.
    const double U = std::fmax(std::fabs(p.u_bottom), std::fabs(p.u_top));
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int k = 0; k < 9; ++k) {
        double sc = 1.0;
        if (p.precision == 2) {
            const double bound = w[k] * (6.0 * U + 0.01);
            sc = std::ldexp(1.0, (int)std::floor(std::log2(1024.0 / bound)));
        }
        I.scale[k] = (float)sc;
        I.inv_scale[k] = (float)(1.0 / sc);
    }
    // the same constants in stored units (sigma_k = scale[k]): bounce-back
    // terms and, per weight class (rest, axis, diagonal), sigma w and the
    // multiples the two-relaxation-time collision uses
    for (int k = 0; k < 9; ++k)
        for (int wall = 0; wall < 2; ++wall) I.bbs[wall][k] = (float)(I.bbd[wall][k] * I.scale[k]);
    const int rep[3] = {0, 1, 5};
    for (int c = 0; c < 3; ++c) {
        const double sw = (double)I.scale[rep[c]] * w[rep[c]];
        I.trt_sw[c] = (float)sw;
        I.trt_k45[c] = (float)(4.5 * sw);
        I.trt_k3[c] = (float)(3.0 * sw);
    }
    return FPD_OK;
}

void drop_graphs(fpd_sim *s) {
    for (auto &g : s->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_all(fpd_sim *s) {
    if (!s) return;
    if (s->owns_state) cudaFree(s->state);
    s->state = nullptr;
    cudaFree(s->scratch);
    s->inst_d = nullptr;
    s->counters = nullptr;
    for (auto &m : s->masks) m = nullptr;
    if (s->host_stage) cudaFreeHost(s->host_stage);
    s->host_stage = nullptr;
    if (s->ex_ring) cudaFreeHost(s->ex_ring);
    s->ex_ring = s->ex_ring_d = nullptr;
    s->ex_slots = 0;
    drop_graphs(s);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    for (auto &e : s->read_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    for (auto &r : s->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    s->pool = s->tabmem = s->scratch = nullptr;
}

int ensure_scratch(fpd_sim *s, size_t bytes) {
    if (s->scratch_bytes >= bytes) return FPD_OK;
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&s->scratch, bytes);
    if (e != cudaSuccess) return fail(s, FPD_ENOMEM, "cudaMalloc of %zu scratch bytes: %s", bytes, cudaGetErrorString(e));
    s->scratch_bytes = bytes;
    return FPD_OK;
}

cudaEvent_t take_event(fpd_sim *s) {
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void harvest(fpd_sim *s) {
    for (auto &r : s->recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        s->ms[r.kind] += ms;
        s->launches[r.kind] += 1;
        s->ev_pool.push_back(r.a);
        s->ev_pool.push_back(r.b);
    }
    s->recs.clear();
}

// current bead table: the one that drove the last collision (step 0: the
// initial table)
int cur_tab(const fpd_sim *s) { return s->nstep == 0 ? 0 : (int)((s->nstep - 1) & 1); }

}  // namespace

namespace {

// Enqueue one time step (bead phase for t >= 1, then the sweep) on `st`.
// Consecutive launches are programmatic dependents unless profiled.
int enqueue_step(fpd_sim *s, cudaStream_t st, int64_t t, bool profiled) {
    const fpd::Inst &I = s->inst;
    const int parity = (int)(t & 1);
    cudaError_t e;
    if (I.nb > 0 && t >= 1) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (profiled) {
            a = take_event(s);
            b = take_event(s);
            cudaEventRecord(a, st);
        }
        e = fpd::launch_beads(s->precision, s->inst_d, nullptr, I.nb, s->pool, s->tab[0], s->tab[1],
                              s->masks[t % fpd::kMaskBufs], parity, 1, s->counters, profiled ? 0 : 1, st,
                              fpd::BeadExport{s->ex_ring_d, s->ex_count, s->ex_slots, s->ex_stride}, s->status);
        if (e != cudaSuccess) return cuda_fail(s, e, "bead kernel launch");
        if (profiled) {
            cudaEventRecord(b, st);
            s->recs.push_back({a, b, 1});
        }
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (profiled) {
        a = take_event(s);
        b = take_event(s);
        cudaEventRecord(a, st);
    }
    const int after_beads = (I.nb > 0 && t >= 1 && !profiled) ? 1 : 0;
    constexpr int M = fpd::kMaskBufs;
    // from step 1 on, the previous bead phase (or the initial marks) is in
    // the previous buffer
    const fpd::SweepMasks mk{s->masks[t % M], s->masks[(t + M - 1) % M], s->masks[(t + 1) % M],
                             (t >= 1 && s->early_cold) ? 1 : 0, s->status, s->copy_shortfall};
    e = fpd::launch_lattice(s->precision, s->inst_d, I, s->pool, s->tab[parity], mk, parity, after_beads,
                            s->variant, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "lattice kernel launch");
    if (profiled) {
        cudaEventRecord(b, st);
        s->recs.push_back({a, b, 0});
        if (s->recs.size() > 4096) harvest(s);
    }
    return FPD_OK;
}

// Capture kGraphSteps consecutive steps whose first step t (>= 1) has
// t % kMaskBufs == p on a private stream, instantiate them and upload the
// graph; it replays on any stream.
int capture_chunk(fpd_sim *s, int p) {
    const int len = fpd::kGraphSteps;
    cudaError_t e;
    if (!s->cap_stream && (e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(s, e, "capture stream");
    if ((e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(s, e, "begin capture");
    int rc = FPD_OK;
    for (int i = 0; i < len && rc == FPD_OK; ++i) rc = enqueue_step(s, s->cap_stream, fpd::kMaskBufs + p + i, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s->cap_stream, &g);
    if (rc != FPD_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "end capture");
    e = cudaGraphInstantiate(&s->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph[p] = nullptr;
        return cuda_fail(s, e, "graph instantiate");
    }
    // move the graph's work to the device now: its first launch is then as
    // cheap as the later ones
    if ((e = cudaGraphUpload(s->graph[p], s->stream)) != cudaSuccess) return cuda_fail(s, e, "graph upload");
    return FPD_OK;
}

// The chunks fpd_step(s, n) takes from step count t: a captured chunk of
// kGraphSteps steps while that many remain (and t >= 1), single launches
// otherwise (a graph of a shorter run measured no faster than its direct
// launches).  visit(p, len) is called for each chunk (len 1: a direct step)
// in order.
template <class F> void plan_steps(const fpd_sim *s, int64_t t, int64_t n, F visit) {
    const bool graphs = s->use_graphs && !s->profiling;
    while (n > 0) {
        const int len = (graphs && t >= 1 && n >= fpd::kGraphSteps) ? fpd::kGraphSteps : 1;
        visit((int)(t % fpd::kMaskBufs), len);
        t += len;
        n -= len;
    }
}

}  // namespace

namespace fpd {

int derive_params(fpd_sim *s, const fpd_params &p) { return derive(s, p); }

const char *create_error() { return g_create_error.c_str(); }

bool initial_beads(const fpd_params &p, double l0, std::vector<double> &Rx, std::vector<double> &Ry) {
    // R_i = c + (i - (N+1)/2) l0 (cos theta, sin theta), i = 1..N (Sec. 4.1:
    // the fiber centred on c), or the explicit positions
    const int nb = p.n_beads * p.n_fibers;
    Rx.assign(nb, 0.0);
    Ry.assign(nb, 0.0);
    for (int f = 0; f < p.n_fibers; ++f)
        for (int i = 1; i <= p.n_beads; ++i) {
            const int b = f * p.n_beads + i - 1;
            if (p.bead_xy) {
                Rx[b] = p.bead_xy[2 * b];
                Ry[b] = p.bead_xy[2 * b + 1];
            } else {
                const double off = (i - (p.n_beads + 1) / 2.0) * l0;
                Rx[b] = p.centre_xy[2 * f] + off * std::cos(p.theta0[f]);
                Ry[b] = p.centre_xy[2 * f + 1] + off * std::sin(p.theta0[f]);
            }
        }
    for (int b = 0; b < nb; ++b)
        if (!is_fin(Rx[b]) || !is_fin(Ry[b])) return false;
    return true;
}

}  // namespace fpd

extern "C" {

int fpd_version(void) { return FPD_ABI_VERSION; }

void fpd_default_params(fpd_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nx = 80;
    p->ny = 40;
    p->u_bottom = -0.01;
    p->u_top = 0.01;
    p->nu_f = -1.0;
    p->re = 1.0;
    p->visc_ratio = 50.0;
    p->xi = 1.0;
    p->bead_radius = 2.0;
    p->k_s = -1.0;
    p->k_ev = -1.0;
    p->phi_cut = 8.0;
    p->precision = FPD_F64;
    p->collision = FPD_MRT_MAGIC;
    p->init_couette = 1;
    p->s_e = 1.64;
    p->s_eps = 1.54;
    p->s_q = 1.9;
}

namespace {

// Device state of one instance, every part 256-byte aligned, in one block:
// the two population buffers, the two bead tables, the tile masks, the bead
// counter and the instance record.
constexpr size_t kStateAlign = 256;
struct StateLayout {
    size_t pool, tab, masks, counters, inst, total;  // offsets; total = block size
    size_t pool_bytes, tab_bytes, tab_one, mask_bytes, mask_words;
};
size_t up(size_t v) { return (v + kStateAlign - 1) / kStateAlign * kStateAlign; }
StateLayout state_layout(const fpd::Inst &I, size_t elem) {
    StateLayout L{};
    const size_t nbm = I.nb > 0 ? (size_t)I.nb : 1;
    L.pool_bytes = 2 * 9 * (size_t)I.plane * elem;  // two population buffers
    // each table: 9 doubles then 6 floats per bead
    L.tab_one = nbm * (fpd::kTabDoubles * sizeof(double) + fpd::kTabFloats * sizeof(float));
    L.tab_bytes = 2 * L.tab_one;
    L.mask_words = (size_t)I.ntx * I.nty * I.mask_words;
    L.mask_bytes = fpd::kMaskBufs * L.mask_words * sizeof(unsigned);
    L.pool = 0;
    L.tab = up(L.pool + L.pool_bytes);
    L.masks = up(L.tab + L.tab_bytes);
    L.counters = up(L.masks + L.mask_bytes);
    // last-block counter, the 64-bit export counter at +8, the status word at +16
    L.inst = up(L.counters + 32);
    L.total = up(L.inst + sizeof(fpd::Inst));
    return L;
}

int create_impl(const fpd_params *p, void *stream, void *workspace, uint64_t workspace_bytes, fpd_sim **out);

}  // namespace

int fpd_workspace_bytes(const fpd_params *p, uint64_t *bytes) {
    if (!p || !bytes) return fail(nullptr, FPD_EINVAL, "fpd_workspace_bytes: NULL argument");
    fpd_sim tmp;
    int rc = derive(&tmp, *p);
    if (rc != FPD_OK) return rc;
    *bytes = state_layout(tmp.inst, elem_size(p->precision)).total;
    return FPD_OK;
}

int fpd_create(const fpd_params *p, void *stream, fpd_sim **out) {
    return create_impl(p, stream, nullptr, 0, out);
}

int fpd_create_ex(const fpd_params *p, void *stream, void *workspace, uint64_t workspace_bytes, fpd_sim **out) {
    if (!workspace) return fail(nullptr, FPD_EINVAL, "fpd_create_ex: NULL workspace");
    return create_impl(p, stream, workspace, workspace_bytes, out);
}

namespace {

int create_impl(const fpd_params *p, void *stream, void *workspace, uint64_t workspace_bytes, fpd_sim **out) {
    if (!p || !out) return fail(nullptr, FPD_EINVAL, "fpd_create: NULL argument");
    *out = nullptr;
    fpd_sim *s = new (std::nothrow) fpd_sim();
    if (!s) return fail(nullptr, FPD_ENOMEM, "host allocation failed");
    int rc = derive(s, *p);
    if (rc != FPD_OK) {
        delete s;
        return rc;
    }
    s->p = *p;
    s->p.centre_xy = s->p.theta0 = s->p.bead_xy = nullptr;
    s->precision = p->precision;
    s->elem = elem_size(p->precision);
    s->stream = (cudaStream_t)stream;
    {
        const char *ng = std::getenv("FPD_NO_GRAPHS");
        s->use_graphs = !(ng && ng[0] == '1');
        const char *ne = std::getenv("FPD_NO_EARLY_COLD");
        s->early_cold = !(ne && ne[0] == '1');
        const char *cs = std::getenv("FPD_TEST_COPY_SHORTFALL");
        s->copy_shortfall = (cs && cs[0] == '1') ? 16u : 0u;
    }
    const fpd::Inst &I = s->inst;
    const int nb = I.nb;
    cudaError_t e;
#define FPD_TRY(call, what)                                 \
    do {                                                    \
        e = (call);                                         \
        if (e != cudaSuccess) {                             \
            int code = (e == cudaErrorMemoryAllocation) ? FPD_ENOMEM : FPD_ECUDA; \
            fail(nullptr, code, "%s: %s", what, cudaGetErrorString(e)); \
            free_all(s);                                    \
            delete s;                                       \
            return code;                                    \
        }                                                   \
    } while (0)
    FPD_TRY(fpd::prepare_lattice_kernels(), "sweep kernel attributes");
    const StateLayout L = state_layout(I, s->elem);
    if (workspace) {
        if (workspace_bytes < L.total || ((uintptr_t)workspace % kStateAlign) != 0) {
            fail(nullptr, FPD_EINVAL, "workspace must hold %llu bytes at a %zu-byte aligned address",
                 (unsigned long long)L.total, kStateAlign);
            delete s;
            return FPD_EINVAL;
        }
        s->state = workspace;
        s->owns_state = false;
    } else {
        FPD_TRY(cudaMalloc(&s->state, L.total), "cudaMalloc simulation state");
    }
    FPD_TRY(cudaMemsetAsync(s->state, 0, L.total, s->stream), "cudaMemset simulation state");
    char *base = (char *)s->state;
    const int nbm = nb > 0 ? nb : 1;
    s->pool = base + L.pool;
    s->pool_bytes = L.pool_bytes;
    s->tabmem = (double *)(base + L.tab);
    s->tab_bytes = L.tab_bytes;
    for (int t = 0; t < 2; ++t) {
        double *b = (double *)((char *)s->tabmem + t * L.tab_one);
        float *f = (float *)(b + fpd::kTabDoubles * nbm);
        s->tab[t] = fpd::BeadTab{b,           b + nbm,     b + 2 * nbm, b + 3 * nbm, b + 4 * nbm,
                                 b + 5 * nbm, b + 6 * nbm, b + 7 * nbm, b + 8 * nbm, f,
                                 f + nbm,     f + 2 * nbm, f + 3 * nbm, f + 4 * nbm, f + 5 * nbm};
    }
    // tile masks, one buffer per step of the rotation (zeroed with the block)
    s->masks[0] = (unsigned *)(base + L.masks);
    for (int m = 1; m < fpd::kMaskBufs; ++m) s->masks[m] = s->masks[0] + m * L.mask_words;
    s->mask_bytes = L.mask_bytes;
    s->counters = (unsigned *)(base + L.counters);
    s->ex_count = (unsigned long long *)(base + L.counters + 8);
    s->status = (unsigned *)(base + L.counters + 16);
    s->inst_d = (fpd::Inst *)(base + L.inst);
    FPD_TRY(cudaMemcpyAsync(s->inst_d, &I, sizeof I, cudaMemcpyHostToDevice, s->stream), "copy instance");
    FPD_TRY(fpd::launch_init(s->precision, s->inst_d, I, s->pool, p->init_couette, s->stream), "init kernel");
    if (nb > 0) {
        std::vector<double> Rx, Ry;
        if (!fpd::initial_beads(*p, I.l0, Rx, Ry)) {
            free_all(s);
            delete s;
            return fail(nullptr, FPD_EINVAL, "bead positions must be finite");
        }
        FPD_TRY(cudaMemcpyAsync(s->tab[0].Rx, Rx.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                "copy beads");
        FPD_TRY(cudaMemcpyAsync(s->tab[0].Ry, Ry.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s->stream),
                "copy beads");
        FPD_TRY(fpd::launch_beads(s->precision, s->inst_d, nullptr, nb, s->pool, s->tab[0], s->tab[1],
                                  s->masks[0], 0, 0, s->counters, 0, s->stream),
                "initial bead table");
    }
    FPD_TRY(cudaStreamSynchronize(s->stream), "fpd_create");
#undef FPD_TRY
    *out = s;
    return FPD_OK;
}

}  // namespace

int fpd_step(fpd_sim *s, int64_t n_steps) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_step: NULL handle");
    if (n_steps < 0) return fail(s, FPD_EINVAL, "n_steps must be >= 0");
    // watchdog: a pass over the populations each time the step count has
    // crossed a multiple of kWatchSteps (between chunks, never inside one)
    auto watch_if_due = [s]() -> int {
        if (s->nstep < s->watch_next) return FPD_OK;
        cudaError_t e = fpd::launch_watch(s->precision, nullptr, s->inst, nullptr, 0, s->pool, (int)(s->nstep & 1),
                                          s->status, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "watchdog launch");
        s->watch_next = (s->nstep / fpd::kWatchSteps + 1) * fpd::kWatchSteps;
        return FPD_OK;
    };
    // whole chunks of the step loop replay a captured graph (one launch
    // instead of two per step, captured on first use or by fpd_prepare);
    // the first step, remainders and profiled steps are launched directly
    int rc = FPD_OK;
    plan_steps(s, s->nstep, n_steps, [&](int p, int len) {
        if (rc != FPD_OK) return;
        if (len == 1) {
            rc = enqueue_step(s, s->stream, s->nstep, s->profiling);
        } else {
            if (!s->graph[p] && (rc = capture_chunk(s, p)) != FPD_OK) return;
            cudaError_t e = cudaGraphLaunch(s->graph[p], s->stream);
            if (e != cudaSuccess) rc = cuda_fail(s, e, "graph launch");
        }
        if (rc != FPD_OK) return;
        s->nstep += len;
        rc = watch_if_due();
    });
    return rc;
}

int fpd_prepare(fpd_sim *s, int64_t n_steps) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_prepare: NULL handle");
    if (n_steps < 0) return fail(s, FPD_EINVAL, "n_steps must be >= 0");
    int rc = FPD_OK;
    plan_steps(s, s->nstep, n_steps, [&](int p, int len) {
        if (rc == FPD_OK && len > 1 && !s->graph[p]) rc = capture_chunk(s, p);
    });
    return rc;
}

int fpd_set_tuning(fpd_sim *s, int32_t variant) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_set_tuning: NULL handle");
    if (variant < 0 || variant >= fpd::kLatticeVariants)
        return fail(s, FPD_EINVAL, "tuning variant must be in [0, %d)", fpd::kLatticeVariants);
    if (variant != s->variant) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "fpd_set_tuning");
        drop_graphs(s);
        s->variant = variant;
    }
    return FPD_OK;
}

int32_t fpd_sweep_variants(void) { return fpd::kLatticeVariants; }

int fpd_get_tuning(const fpd_sim *s, int32_t *variant, int32_t *n_variants) {
    if (!s) return FPD_EINVAL;
    if (variant) *variant = s->variant;
    if (n_variants) *n_variants = fpd::kLatticeVariants;
    return FPD_OK;
}

int fpd_sync(fpd_sim *s) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_sync: NULL handle");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
    unsigned flags = 0;
    e = cudaMemcpy(&flags, s->status, sizeof flags, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "read status");
    if (flags & fpd::kFlagNonFinite)
        return fail(s, FPD_ENAN, "non-finite state found by step %lld (FPD_FLAG_NONFINITE)", (long long)s->nstep);
    if (flags & fpd::kFlagCopyTimeout)
        return fail(s, FPD_ECUDA, "a staged sweep's bulk copy did not complete (FPD_FLAG_COPY_TIMEOUT)");
    return FPD_OK;
}

int fpd_flags(fpd_sim *s, uint32_t *flags) {
    if (!s || !flags) return fail(s, FPD_EINVAL, "fpd_flags: NULL argument");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream synchronize");
    unsigned v = 0;
    e = cudaMemcpy(&v, s->status, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "read status");
    *flags = v;
    return FPD_OK;
}

int fpd_read_fields(fpd_sim *s, double *ux, double *uy, double *rho) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_read_fields: NULL handle");
    const fpd::Inst &I = s->inst;
    const size_t n = (size_t)I.nx * I.ny;
    int rc = ensure_scratch(s, 3 * n * sizeof(double));
    if (rc) return rc;
    const int ct = cur_tab(s);
    const int cm = s->nstep == 0 ? 0 : (int)((s->nstep - 1) % fpd::kMaskBufs);
    cudaError_t e = fpd::launch_fields(s->precision, s->inst_d, I, s->pool, s->tab[ct], s->masks[cm],
                                       (int)(s->nstep & 1), s->scratch, s->scratch + n, s->scratch + 2 * n,
                                       s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "fields kernel");
    double *dst[3] = {ux, uy, rho};
    for (int i = 0; i < 3; ++i)
        if (dst[i]) {
            e = cudaMemcpyAsync(dst[i], s->scratch + i * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "copy fields");
        }
    return fpd_sync(s);
}

int fpd_internal_flow(fpd_sim *s, double *eps) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_internal_flow: NULL handle");
    if (!eps) return fail(s, FPD_EINVAL, "fpd_internal_flow: NULL output");
    const fpd::Inst &I = s->inst;
    if (I.nb == 0) return fpd_sync(s);
    int rc = ensure_scratch(s, 2 * (size_t)I.nb * sizeof(double));
    if (rc) return rc;
    cudaError_t e = fpd::launch_internal_flow(s->precision, I, s->pool, s->tab[cur_tab(s)], (int)(s->nstep & 1),
                                              s->scratch, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "internal-flow kernel");
    std::vector<double> h(2 * (size_t)I.nb);
    e = cudaMemcpyAsync(h.data(), s->scratch, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy internal flow");
    if ((rc = fpd_sync(s))) return rc;
    for (int q = 0; q < I.nb; ++q) eps[q] = h[2 * q] / h[2 * q + 1];
    return FPD_OK;
}

int fpd_read_beads(fpd_sim *s, double *pos, double *vel, double *force, double *support) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_read_beads: NULL handle");
    const int nb = s->inst.nb;
    if (nb == 0) return fpd_sync(s);
    // R, V, F, S of a table are seven consecutive arrays of nb doubles: one
    // copy into pinned staging memory, ordered after the queued steps
    if (!s->host_stage) {
        cudaError_t e = cudaMallocHost(&s->host_stage, 7 * (size_t)nb * sizeof(double));
        if (e != cudaSuccess) {
            s->host_stage = nullptr;
            return cuda_fail(s, e, "pinned staging for bead reads");
        }
    }
    const fpd::BeadTab &t = s->tab[cur_tab(s)];
    cudaError_t e = cudaMemcpyAsync(s->host_stage, t.Rx, 7 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy beads");
    int rc = fpd_sync(s);
    if (rc) return rc;
    const double *h = s->host_stage;
    auto pair = [&](double *dst, int k) {
        if (!dst) return;
        const double *x = h + (size_t)k * nb, *y = x + nb;
        for (int i = 0; i < nb; ++i) {
            dst[2 * i] = x[i];
            dst[2 * i + 1] = y[i];
        }
    };
    pair(pos, 0);
    pair(vel, 2);  // the initial table keeps V = 0 until the second step overwrites it
    pair(force, 4);
    if (support) std::memcpy(support, h + 6 * (size_t)nb, nb * sizeof(double));
    return FPD_OK;
}

int fpd_read_beads_async(fpd_sim *s, double *dst, uint64_t *ticket) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_read_beads_async: NULL handle");
    if (!dst || !ticket) return fail(s, FPD_EINVAL, "fpd_read_beads_async: NULL destination or ticket");
    const int k = (int)(s->read_seq % fpd_sim::kReadTickets);
    cudaError_t e;
    if (!s->read_ev[k] && (e = cudaEventCreateWithFlags(&s->read_ev[k], cudaEventDisableTiming)) != cudaSuccess) {
        s->read_ev[k] = nullptr;
        return cuda_fail(s, e, "read event");
    }
    const int nb = s->inst.nb;
    if (nb > 0) {
        // R, V, F, S of a table are seven consecutive arrays of nb doubles
        const fpd::BeadTab &t = s->tab[cur_tab(s)];
        if ((e = cudaMemcpyAsync(dst, t.Rx, 7 * (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s->stream)) !=
            cudaSuccess)
            return cuda_fail(s, e, "copy beads");
    }
    if ((e = cudaEventRecord(s->read_ev[k], s->stream)) != cudaSuccess) return cuda_fail(s, e, "record read");
    *ticket = s->read_seq++;
    return FPD_OK;
}

int fpd_export_beads(fpd_sim *s, int32_t slots) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_export_beads: NULL handle");
    if (slots < 0 || slots == 1) return fail(s, FPD_EINVAL, "fpd_export_beads: slots must be 0 or >= 2");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "fpd_export_beads");
    drop_graphs(s);
    if (s->ex_ring) cudaFreeHost(s->ex_ring);
    s->ex_ring = s->ex_ring_d = nullptr;
    s->ex_slots = 0;
    if (slots == 0 || s->inst.nb == 0) return FPD_OK;
    const int stride = fpd::kExportHeader + 7 * s->inst.nb;
    const size_t bytes = (size_t)slots * stride * sizeof(double);
    void *h = nullptr, *d = nullptr;
    if ((e = cudaHostAlloc(&h, bytes, cudaHostAllocMapped)) != cudaSuccess)
        return fail(s, FPD_ENOMEM, "fpd_export_beads: page-locked ring of %zu bytes: %s", bytes,
                    cudaGetErrorString(e));
    if ((e = cudaHostGetDevicePointer(&d, h, 0)) != cudaSuccess) {
        cudaFreeHost(h);
        return cuda_fail(s, e, "fpd_export_beads: device address of the ring");
    }
    std::memset(h, 0, bytes);
    if ((e = cudaMemsetAsync(s->ex_count, 0, sizeof(unsigned long long), s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess) {
        cudaFreeHost(h);
        return cuda_fail(s, e, "fpd_export_beads: reset counter");
    }
    s->ex_ring = (double *)h;
    s->ex_ring_d = (double *)d;
    s->ex_slots = slots;
    s->ex_stride = stride;
    // the bead phase of step index t (t >= 1) finishes the table after t + 1 steps
    s->ex_first = std::max<int64_t>(s->nstep, 1) + 1;
    return FPD_OK;
}

int fpd_take_beads(fpd_sim *s, int64_t n, double *dst) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_take_beads: NULL handle");
    if (!dst) return fail(s, FPD_EINVAL, "fpd_take_beads: NULL destination");
    if (!s->ex_ring) return fail(s, FPD_EINVAL, "fpd_take_beads: bead export is off");
    if (n < s->ex_first || n > s->nstep)
        return fail(s, FPD_EINVAL, "fpd_take_beads: step %lld was not exported or not enqueued (exported from %lld, "
                    "%lld enqueued)", (long long)n, (long long)s->ex_first, (long long)s->nstep);
    const unsigned long long want = (unsigned long long)(n - s->ex_first) + 1ull;
    const double *slot = s->ex_ring + (size_t)((want - 1) % (unsigned long long)s->ex_slots) * s->ex_stride;
    const auto *hdr = reinterpret_cast<const unsigned long long *>(slot);
    const size_t count = 7 * (size_t)s->inst.nb;
    constexpr int kTakeTimeoutS = 60;
    std::chrono::steady_clock::time_point t_start{};
    for (long spin = 0;; ++spin) {
        const unsigned long long h = __atomic_load_n(hdr, __ATOMIC_ACQUIRE);
        if (h > want) return fail(s, FPD_EBUSY, "fpd_take_beads: the ring has reused the entry of step %lld",
                                  (long long)n);
        if (h == want) {
            std::memcpy(dst, slot + fpd::kExportHeader, count * sizeof(double));
            // the entry must not have been rewritten while it was copied
            if (__atomic_load_n(hdr, __ATOMIC_ACQUIRE) != want)
                return fail(s, FPD_EBUSY, "fpd_take_beads: the ring reused the entry of step %lld during the copy",
                            (long long)n);
            return FPD_OK;
        }
        if ((spin & 1023) == 1023) {
            // the device has not written it yet: stop if the stream has run
            // dry (the step's bead phase cannot come), failed, or made no
            // progress for kTakeTimeoutS seconds
            if (spin == 1023) t_start = std::chrono::steady_clock::now();
            else if (std::chrono::steady_clock::now() - t_start > std::chrono::seconds(kTakeTimeoutS))
                return fail(s, FPD_ETIMEOUT, "fpd_take_beads: step %lld not written within %d s", (long long)n,
                            kTakeTimeoutS);
            const cudaError_t q = cudaStreamQuery(s->stream);
            if (q == cudaSuccess) {
                if (__atomic_load_n(hdr, __ATOMIC_ACQUIRE) == want) continue;
                return fail(s, FPD_EINVAL, "fpd_take_beads: the stream is idle and step %lld was not exported",
                            (long long)n);
            }
            if (q != cudaErrorNotReady) return cuda_fail(s, q, "fpd_take_beads");
        }
    }
}

int fpd_wait_read(fpd_sim *s, uint64_t ticket) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_wait_read: NULL handle");
    if (ticket >= s->read_seq) return fail(s, FPD_EINVAL, "fpd_wait_read: ticket %llu was not issued",
                                           (unsigned long long)ticket);
    // the slot holds this read or a later one on the same stream; either
    // completing means this read has completed
    const cudaError_t e = cudaEventSynchronize(s->read_ev[ticket % fpd_sim::kReadTickets]);
    return e == cudaSuccess ? FPD_OK : cuda_fail(s, e, "bead read");
}

namespace {

// Checkpoint file: header, the derived instance record, then the device
// blobs in this order: populations, bead tables, tile masks.
struct CkptHeader {
    char tag[8];
    uint32_t abi, inst_bytes;
    uint64_t pool_bytes, tab_bytes, mask_bytes;
    int64_t nstep;
};
constexpr char kCkptTag[8] = {'F', 'P', 'D', 'C', 'K', 'P', 'T', '1'};

}  // namespace

int fpd_save(fpd_sim *s, const char *path) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_save: NULL handle");
    if (!path) return fail(s, FPD_EINVAL, "fpd_save: NULL path");
    int rc = fpd_sync(s);
    if (rc) return rc;
    std::vector<char> pool(s->pool_bytes), tabs(s->tab_bytes), masks(s->mask_bytes);
    cudaError_t e = cudaMemcpy(pool.data(), s->pool, pool.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(tabs.data(), s->tabmem, tabs.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(masks.data(), s->masks[0], masks.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "fpd_save");
    CkptHeader h{};
    std::memcpy(h.tag, kCkptTag, sizeof h.tag);
    h.abi = FPD_ABI_VERSION;
    h.inst_bytes = (uint32_t)sizeof(fpd::Inst);
    h.pool_bytes = pool.size();
    h.tab_bytes = tabs.size();
    h.mask_bytes = masks.size();
    h.nstep = s->nstep;
    std::FILE *f = std::fopen(path, "wb");
    if (!f) return fail(s, FPD_EINVAL, "fpd_save: cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(&s->inst, sizeof(fpd::Inst), 1, f) == 1 &&
              std::fwrite(pool.data(), 1, pool.size(), f) == pool.size() &&
              std::fwrite(tabs.data(), 1, tabs.size(), f) == tabs.size() &&
              std::fwrite(masks.data(), 1, masks.size(), f) == masks.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(s, FPD_EINVAL, "fpd_save: writing %s failed", path);
    return FPD_OK;
}

int fpd_load(fpd_sim *s, const char *path) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_load: NULL handle");
    if (!path) return fail(s, FPD_EINVAL, "fpd_load: NULL path");
    std::FILE *f = std::fopen(path, "rb");
    if (!f) return fail(s, FPD_EINVAL, "fpd_load: cannot open %s", path);
    CkptHeader h{};
    fpd::Inst inst;
    std::vector<char> pool, tabs, masks;
    const char *why = nullptr;
    if (std::fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.tag, kCkptTag, sizeof h.tag) != 0) {
        why = "not a checkpoint of this format";
    } else if (h.abi != FPD_ABI_VERSION || h.inst_bytes != sizeof(fpd::Inst)) {
        why = "written by another ABI version";
    } else if (std::fread(&inst, sizeof inst, 1, f) != 1) {
        why = "truncated";
    } else if (std::memcmp(&inst, &s->inst, sizeof inst) != 0 || h.pool_bytes != s->pool_bytes ||
               h.tab_bytes != s->tab_bytes || h.mask_bytes != s->mask_bytes || h.nstep < 0) {
        why = "written with other parameters";
    } else {
        pool.resize(h.pool_bytes);
        tabs.resize(h.tab_bytes);
        masks.resize(h.mask_bytes);
        if (std::fread(pool.data(), 1, pool.size(), f) != pool.size() ||
            std::fread(tabs.data(), 1, tabs.size(), f) != tabs.size() ||
            std::fread(masks.data(), 1, masks.size(), f) != masks.size())
            why = "truncated";
        else if (std::fgetc(f) != EOF)
            why = "longer than a checkpoint";
    }
    std::fclose(f);
    if (why) return fail(s, FPD_EINVAL, "fpd_load: %s: %s", path, why);
    int rc = fpd_sync(s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(s->pool, pool.data(), pool.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->tabmem, tabs.data(), tabs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->masks[0], masks.data(), masks.size(), cudaMemcpyHostToDevice);
    // the status flags describe the replaced run: they start over
    if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(s, e, "fpd_load");
    s->nstep = h.nstep;
    s->watch_next = (s->nstep / fpd::kWatchSteps + 1) * fpd::kWatchSteps;
    // an active bead export restarts from the restored step count
    if (s->ex_ring) return fpd_export_beads(s, s->ex_slots);
    return FPD_OK;
}

int fpd_read_populations(fpd_sim *s, double *f) {
    if (!s || !f) return fail(s, FPD_EINVAL, "fpd_read_populations: NULL argument");
    const fpd::Inst &I = s->inst;
    const size_t n = 9 * (size_t)I.nx * I.ny;
    int rc = ensure_scratch(s, n * sizeof(double));
    if (rc) return rc;
    cudaError_t e = fpd::launch_read_pops(s->precision, s->inst_d, I, s->pool, (int)(s->nstep & 1), s->scratch,
                                          s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population read kernel");
    e = cudaMemcpyAsync(f, s->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy populations");
    return fpd_sync(s);
}

int fpd_write_populations(fpd_sim *s, const double *f) {
    if (!s || !f) return fail(s, FPD_EINVAL, "fpd_write_populations: NULL argument");
    const fpd::Inst &I = s->inst;
    const size_t n = 9 * (size_t)I.nx * I.ny;
    for (size_t i = 0; i < n; ++i)
        if (!is_fin(f[i])) return fail(s, FPD_EINVAL, "populations must be finite");
    int rc = ensure_scratch(s, n * sizeof(double));
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(s->scratch, f, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy populations");
    e = fpd::launch_write_pops(s->precision, s->inst_d, I, s->pool, (int)(s->nstep & 1), s->scratch, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population write kernel");
    return fpd_sync(s);
}

int fpd_diag(fpd_sim *s, double out[4]) {
    if (!s || !out) return fail(s, FPD_EINVAL, "fpd_diag: NULL argument");
    const fpd::Inst &I = s->inst;
    const int nb = fpd::diag_blocks(I);
    int rc = ensure_scratch(s, 4 * (size_t)nb * sizeof(double));
    if (rc) return rc;
    cudaError_t e = fpd::launch_diag(s->precision, s->inst_d, I, s->pool, (int)(s->nstep & 1), s->scratch, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "diagnostics kernel");
    std::vector<double> part(4 * (size_t)nb);
    e = cudaMemcpyAsync(part.data(), s->scratch, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy diagnostics");
    if ((rc = fpd_sync(s))) return rc;
    double m = 0, px = 0, py = 0, bad = 0;
    for (int b = 0; b < nb; ++b) {
        m += part[4 * b];
        px += part[4 * b + 1];
        py += part[4 * b + 2];
        bad += part[4 * b + 3];
    }
    out[0] = (double)I.nx * I.ny + m;  // sum of w_k over cells is 1 per cell
    out[1] = px;
    out[2] = py;
    out[3] = (double)s->nstep;
    if (bad > 0 || !is_fin(m) || !is_fin(px) || !is_fin(py))
        return fail(s, FPD_ENAN, "non-finite populations after %lld steps", (long long)s->nstep);
    return FPD_OK;
}

int fpd_derived(const fpd_sim *s, double out[8]) {
    if (!s || !out) return FPD_EINVAL;
    out[0] = s->nu_f;
    out[1] = s->k_s;
    out[2] = s->k_b;
    out[3] = s->k_ev;
    out[4] = s->inst.l0;
    out[5] = s->inst.rcut;
    out[6] = s->gamma_dot;
    out[7] = 18.0 * (double)s->elem;
    return FPD_OK;
}

int fpd_set_profiling(fpd_sim *s, int on) {
    if (!s) return fail(nullptr, FPD_EINVAL, "fpd_set_profiling: NULL handle");
    harvest(s);
    s->profiling = on != 0;
    if (on) {
        s->ms[0] = s->ms[1] = 0;
        s->launches[0] = s->launches[1] = 0;
    }
    return FPD_OK;
}

int fpd_kernel_times(fpd_sim *s, double out[4]) {
    if (!s || !out) return fail(s, FPD_EINVAL, "fpd_kernel_times: NULL argument");
    harvest(s);
    out[0] = s->ms[0];
    out[1] = s->launches[0];
    out[2] = s->ms[1];
    out[3] = s->launches[1];
    return FPD_OK;
}

const char *fpd_last_error(const fpd_sim *s) {
    if (!s) return g_create_error.c_str();
    return s->err.c_str();
}

int fpd_destroy(fpd_sim *s) {
    if (!s) return FPD_OK;
    cudaStreamSynchronize(s->stream);
    free_all(s);
    delete s;
    return FPD_OK;
}

}  // extern "C"
