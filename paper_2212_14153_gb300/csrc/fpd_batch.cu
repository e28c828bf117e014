// fpd_batch.cu -- many independent FPD instances advanced together.
//
// Every active instance (a sweep point or a serving request: its own
// lattice size, wall speeds, viscosity, fiber) lives in one device pool and
// is advanced by the same two launches per time step: one bead-phase launch
// over the beads of all instances and one lattice sweep over a packed list
// of the tiles of all instances.  Kernels never mix instances and reduce in
// a fixed order, so an instance's results do not depend on its companions.
//
// Instances join and leave between runs.  A newly admitted instance starts
// at local step 0 whatever the global step is: its step parity is the global
// parity XOR par_xor, and on its first step it skips the bead advance (its
// initial bead table is computed when the lists are rebuilt).  A run never
// advances an instance past its requested step count: a run is cut at the
// smallest remaining count, and finished instances stay readable until
// removed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "fpd_sim.h"

namespace {

// kFailed: the watchdog or the bead phase found a non-finite value in the
// instance; it is taken out of the running set at the next poll.
enum SlotState { kFree = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Slot {
    int state = kFree;
    bool fresh = false;     // admitted, initial bead table not yet built
    bool first = false;     // its next step is its local step 0
    bool reported = false;  // finished and returned by fpd_batch_poll
    fpd::Inst inst{};
    int64_t pop_len = 0;    // elements
    int bead_len = 0;
    int64_t steps_req = 0, steps_done = 0;
};

// First-fit allocator over [0, capacity) with coalescing free ranges.
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;  // offset -> length
    int64_t cap = 0;
    void reset(int64_t capacity) {
        cap = capacity;
        free_.clear();
        if (capacity > 0) free_[0] = capacity;
    }
    int64_t alloc(int64_t n, int64_t align) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const int64_t off = (it->first + align - 1) / align * align;
            const int64_t pad = off - it->first;
            if (it->second >= pad + n) {
                const int64_t start = it->first, len = it->second;
                free_.erase(it);
                if (pad > 0) free_[start] = pad;
                if (len - pad - n > 0) free_[off + n] = len - pad - n;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t n) {
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t used() const {
        int64_t f = 0;
        for (auto &kv : free_) f += kv.second;
        return cap - f;
    }
};

}  // namespace

struct fpd_batch {
    int precision = 1;
    size_t elem = 4;
    int max_slots = 0, max_beads = 0, mask_words = 1;
    cudaStream_t stream = nullptr;
    void *pool = nullptr;
    int64_t pool_elems = 0;
    RangeAlloc pop_alloc, bead_alloc;
    double *tabmem = nullptr;
    fpd::BeadTab tab[2]{};
    fpd::Inst *insts_d = nullptr;
    unsigned *counters = nullptr;
    unsigned *status = nullptr;  // sticky FPD_FLAG_* bits per slot (device)
    int64_t watch_next = fpd::kWatchSteps;  // global step of the next watchdog pass
    int2 *tiles_d = nullptr;
    int tiles_cap = 0, ntiles = 0;
    unsigned *masks = nullptr;  // kMaskBufs * tiles_cap * mask_words, in rotation by global step
    int2 *beads_all_d = nullptr, *beads_old_d = nullptr, *beads_fresh_d = nullptr;  // (slot, bead)
    int n_all = 0, n_old = 0, n_fresh = 0;
    std::vector<Slot> slots;
    std::vector<fpd::Inst> insts_h;
    int64_t gstep = 0;
    int64_t rebuild_gstep = -1;  // global step at which the masks were last reset
    double cell_updates = 0.0;
    bool dirty = true;
    int variant = 0;  // lattice sweep variant
    int any_mrt = 0;  // some resident instance uses constant Lallemand-Luo rates
    // captured chunks of kGraphSteps steps, one per starting mask buffer
    // (global step mod kMaskBufs); valid until the next rebuild or tuning change
    cudaGraphExec_t graph[fpd::kMaskBufs] = {};
    cudaStream_t cap_stream = nullptr;
    double *scratch = nullptr;
    size_t scratch_bytes = 0;
    std::string err;
};

namespace {

int bfail(fpd_batch *b, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

int bcuda(fpd_batch *b, cudaError_t e, const char *what) {
    return bfail(b, FPD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Destroys the captured step chunks (after the stream has drained them).
void drop_bgraphs(fpd_batch *b) {
    bool any = false;
    for (auto g : b->graph) any = any || g;
    if (!any) return;
    cudaStreamSynchronize(b->stream);
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

void free_batch(fpd_batch *b) {
    drop_bgraphs(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->pool);
    cudaFree(b->tabmem);
    cudaFree(b->insts_d);
    cudaFree(b->counters);
    cudaFree(b->status);
    cudaFree(b->tiles_d);
    cudaFree(b->masks);
    cudaFree(b->beads_all_d);
    cudaFree(b->beads_old_d);
    cudaFree(b->beads_fresh_d);
    cudaFree(b->scratch);
}

int ensure_bscratch(fpd_batch *b, size_t bytes) {
    if (b->scratch_bytes >= bytes) return FPD_OK;
    cudaFree(b->scratch);
    b->scratch = nullptr;
    b->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&b->scratch, bytes);
    if (e != cudaSuccess) return bfail(b, FPD_ENOMEM, "cudaMalloc of %zu scratch bytes: %s", bytes, cudaGetErrorString(e));
    b->scratch_bytes = bytes;
    return FPD_OK;
}

// Rebuild the packed tile list, the bead lists and the instance records
// after a membership change, clear the tile masks and build the initial
// bead tables of newly admitted instances.
int rebuild(fpd_batch *b) {
    cudaError_t e;
    // launch sizes and buffers change: captured chunks are stale
    drop_bgraphs(b);
    std::vector<int2> tiles;
    const int gp = (int)(b->gstep & 1);
    // words per tile mask: enough for the largest resident instance
    int W = 1;
    for (auto &sl : b->slots)
        if (sl.state == kActive) W = std::max(W, (sl.inst.nb + 31) / 32);
    if (W != b->mask_words) {
        b->mask_words = W;
        b->tiles_cap = 0;  // reallocate the masks below
    }
    for (int s = 0; s < b->max_slots; ++s) {
        Slot &sl = b->slots[s];
        if (sl.state != kActive) continue;
        fpd::Inst &I = sl.inst;
        I.mask_words = W;
        I.tile_base = (int)tiles.size();
        for (int by = 0; by < I.nty; ++by)
            for (int bx = 0; bx < I.ntx; ++bx) tiles.push_back(make_int2(s, (by << 16) | bx));
        if (sl.fresh) I.par_xor = gp;  // local step 0 happens at this global step
        b->insts_h[s] = I;
    }
    b->ntiles = (int)tiles.size();
    b->any_mrt = 0;
    for (auto &sl : b->slots)
        if (sl.state == kActive && sl.inst.collision == 1) b->any_mrt = 1;
    if (b->ntiles > b->tiles_cap || !b->masks) {
        cudaFree(b->tiles_d);
        cudaFree(b->masks);
        b->tiles_d = nullptr;
        b->masks = nullptr;
        const int cap = std::max(std::max(b->ntiles, 1), 2 * b->tiles_cap);
        if ((e = cudaMalloc(&b->tiles_d, cap * sizeof(int2))) != cudaSuccess) return bcuda(b, e, "cudaMalloc tiles");
        if ((e = cudaMalloc(&b->masks, fpd::kMaskBufs * (size_t)cap * b->mask_words * sizeof(unsigned))) !=
            cudaSuccess)
            return bcuda(b, e, "cudaMalloc masks");
        b->tiles_cap = cap;
    }
    if (b->ntiles > 0 &&
        (e = cudaMemcpyAsync(b->tiles_d, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice,
                             b->stream)) != cudaSuccess)
        return bcuda(b, e, "copy tiles");
    if ((e = cudaMemcpyAsync(b->insts_d, b->insts_h.data(), b->insts_h.size() * sizeof(fpd::Inst),
                             cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return bcuda(b, e, "copy instance records");
    if (b->tiles_cap > 0 &&
        (e = cudaMemsetAsync(b->masks, 0, fpd::kMaskBufs * (size_t)b->tiles_cap * b->mask_words * sizeof(unsigned),
                             b->stream)) !=
            cudaSuccess)
        return bcuda(b, e, "clear masks");
    // bead lists: (slot, global bead index) for every bead, for the beads of
    // instances past their first step, and for the newly admitted ones
    auto upload = [&](int2 *dst, int &n, int which) -> int {
        std::vector<int2> lst;
        for (int s = 0; s < b->max_slots; ++s) {
            Slot &sl = b->slots[s];
            if (sl.state != kActive) continue;
            const bool take = which == 0 || (which == 1 && !sl.first) || (which == 2 && sl.fresh);
            if (!take) continue;
            for (int q = 0; q < sl.inst.nb; ++q) lst.push_back(make_int2(s, sl.inst.bead_off + q));
        }
        n = (int)lst.size();
        if (n > 0) {
            cudaError_t e2 = cudaMemcpyAsync(dst, lst.data(), n * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
            // the copy must finish before lst goes out of scope
            if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(b->stream);
            if (e2 != cudaSuccess) return bcuda(b, e2, "copy bead lists");
        }
        return FPD_OK;
    };
    int rc;
    if ((rc = upload(b->beads_all_d, b->n_all, 0))) return rc;
    if ((rc = upload(b->beads_old_d, b->n_old, 1))) return rc;
    if ((rc = upload(b->beads_fresh_d, b->n_fresh, 2))) return rc;
    // initial bead tables of new instances (local parity 0 -> table 0)
    if (b->n_fresh > 0) {
        e = fpd::launch_beads(b->precision, b->insts_d, b->beads_fresh_d, b->n_fresh, b->pool, b->tab[0], b->tab[1],
                              b->masks + (size_t)(b->gstep % fpd::kMaskBufs) * b->tiles_cap * b->mask_words, gp, 0,
                              b->counters, 0, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "initial bead tables");
    }
    for (auto &sl : b->slots)
        if (sl.state == kActive) sl.fresh = false;
    b->dirty = false;
    b->rebuild_gstep = b->gstep;
    return FPD_OK;
}

}  // namespace

extern "C" {

int fpd_batch_create(int32_t precision, int32_t max_slots, int64_t pool_bytes, int32_t max_beads, void *stream,
                     fpd_batch **out) {
    if (!out) return FPD_EINVAL;
    *out = nullptr;
    if (precision < 0 || precision > 2 || max_slots < 1 || pool_bytes < 1 || max_beads < 0) return FPD_EINVAL;
    fpd_batch *b = new (std::nothrow) fpd_batch();
    if (!b) return FPD_ENOMEM;
    b->precision = precision;
    b->elem = precision == 0 ? 8 : (precision == 1 ? 4 : 2);
    b->max_slots = max_slots;
    b->max_beads = max_beads;
    b->mask_words = 1;
    b->stream = (cudaStream_t)stream;
    b->slots.assign(max_slots, Slot());
    b->insts_h.assign(max_slots, fpd::Inst{});
    b->pool_elems = pool_bytes / (int64_t)b->elem;
    b->pop_alloc.reset(b->pool_elems);
    b->bead_alloc.reset(max_beads);
    cudaError_t e;
    const int nbm = max_beads > 0 ? max_beads : 1;
    const size_t tab_bytes = (size_t)nbm * (fpd::kTabDoubles * sizeof(double) + fpd::kTabFloats * sizeof(float));
    if ((e = cudaMalloc(&b->pool, (size_t)b->pool_elems * b->elem)) != cudaSuccess ||
        (e = cudaMalloc(&b->tabmem, 2 * tab_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&b->insts_d, max_slots * sizeof(fpd::Inst))) != cudaSuccess ||
        (e = cudaMalloc(&b->counters, max_slots * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&b->status, max_slots * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&b->beads_all_d, nbm * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&b->beads_old_d, nbm * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&b->beads_fresh_d, nbm * sizeof(int2))) != cudaSuccess) {
        free_batch(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? FPD_ENOMEM : FPD_ECUDA;
    }
    cudaMemsetAsync(b->tabmem, 0, 2 * tab_bytes, b->stream);
    cudaMemsetAsync(b->counters, 0, max_slots * sizeof(unsigned), b->stream);
    cudaMemsetAsync(b->status, 0, max_slots * sizeof(unsigned), b->stream);
    for (int t = 0; t < 2; ++t) {
        double *d = (double *)((char *)b->tabmem + t * tab_bytes);
        float *f = (float *)(d + fpd::kTabDoubles * nbm);
        b->tab[t] = fpd::BeadTab{d,           d + nbm,     d + 2 * nbm, d + 3 * nbm, d + 4 * nbm,
                                 d + 5 * nbm, d + 6 * nbm, d + 7 * nbm, d + 8 * nbm, f,
                                 f + nbm,     f + 2 * nbm, f + 3 * nbm, f + 4 * nbm, f + 5 * nbm};
    }
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
        free_batch(b);
        delete b;
        return FPD_ECUDA;
    }
    *out = b;
    return FPD_OK;
}

int fpd_batch_add(fpd_batch *b, const fpd_params *p, int64_t n_steps, int32_t *slot) {
    if (!b || !p || !slot) return b ? bfail(b, FPD_EINVAL, "fpd_batch_add: NULL argument") : FPD_EINVAL;
    *slot = -1;
    if (p->precision != b->precision)
        return bfail(b, FPD_EINVAL, "instance precision %d differs from the batch's %d", p->precision, b->precision);
    if (n_steps < 0) return bfail(b, FPD_EINVAL, "n_steps must be >= 0");
    fpd_sim tmp;
    int rc = fpd::derive_params(&tmp, *p);
    if (rc != FPD_OK) return bfail(b, rc, "%s", fpd::create_error());
    fpd::Inst I = tmp.inst;
    int s = -1;
    for (int i = 0; i < b->max_slots; ++i)
        if (b->slots[i].state == kFree) {
            s = i;
            break;
        }
    if (s < 0) return bfail(b, FPD_EBUSY, "no free slot (%d in use)", b->max_slots);
    const int64_t pop_len = 2 * 9 * I.plane;  // two population buffers
    const int64_t off = b->pop_alloc.alloc(pop_len, (int64_t)(256 / b->elem));
    if (off < 0) return bfail(b, FPD_EBUSY, "no room for %lld population elements", (long long)pop_len);
    int boff = 0;
    if (I.nb > 0) {
        const int64_t bo = b->bead_alloc.alloc(I.nb, 1);
        if (bo < 0) {
            b->pop_alloc.release(off, pop_len);
            return bfail(b, FPD_EBUSY, "no room for %d beads", I.nb);
        }
        boff = (int)bo;
    }
    I.pop_off = off;
    I.bead_off = boff;
    Slot &sl = b->slots[s];
    sl = Slot();
    std::vector<double> Rx, Ry;
    if (I.nb > 0 && !fpd::initial_beads(*p, I.l0, Rx, Ry)) {
        b->pop_alloc.release(off, pop_len);
        b->bead_alloc.release(boff, I.nb);
        return bfail(b, FPD_EINVAL, "bead positions must be finite");
    }
    // the slot's status flags start clear (a removed instance may have left some)
    cudaError_t e = cudaMemsetAsync(b->status + s, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = fpd::launch_init(b->precision, nullptr, I, b->pool, p->init_couette, b->stream);
    if (e == cudaSuccess && I.nb > 0) {
        // initial positions into table 0 (V = 0); S, F, G follow at rebuild
        std::vector<double> zeros(I.nb, 0.0);
        e = cudaMemcpyAsync(b->tab[0].Rx + boff, Rx.data(), I.nb * sizeof(double), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->tab[0].Ry + boff, Ry.data(), I.nb * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->tab[0].Vx + boff, zeros.data(), I.nb * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->tab[0].Vy + boff, zeros.data(), I.nb * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e != cudaSuccess) {
        b->pop_alloc.release(off, pop_len);
        if (I.nb > 0) b->bead_alloc.release(boff, I.nb);
        return bcuda(b, e, "fpd_batch_add");
    }
    sl.state = n_steps > 0 ? kActive : kDone;
    sl.fresh = true;
    sl.first = true;
    sl.inst = I;
    sl.pop_len = pop_len;
    sl.bead_len = I.nb;
    sl.steps_req = n_steps;
    b->insts_h[s] = I;
    b->dirty = true;
    *slot = s;
    return FPD_OK;
}

namespace {

// The launches of global step gstep on stream st: the bead phase (all beads,
// or those of instances past their first step) and the batched sweep.
int enqueue_bstep(fpd_batch *b, cudaStream_t st, int64_t gstep, bool any_first) {
    const int gp = (int)(gstep & 1);
    const int2 *blist = any_first ? b->beads_old_d : b->beads_all_d;
    const int nbl = any_first ? b->n_old : b->n_all;
    constexpr int M = fpd::kMaskBufs;
    const size_t mstride = (size_t)b->tiles_cap * b->mask_words;
    unsigned *mw = b->masks + (size_t)(gstep % M) * mstride;
    // the previous buffer holds the previous bead phase's marks unless the
    // masks were reset before this step
    const fpd::SweepMasks mk{mw, b->masks + (size_t)((gstep + M - 1) % M) * mstride,
                             b->masks + (size_t)((gstep + 1) % M) * mstride, gstep > b->rebuild_gstep ? 1 : 0};
    cudaError_t e;
    if (nbl > 0) {
        e = fpd::launch_beads(b->precision, b->insts_d, blist, nbl, b->pool, b->tab[0], b->tab[1], mw, gp, 1,
                              b->counters, 1, st, fpd::BeadExport{}, b->status);
        if (e != cudaSuccess) return bcuda(b, e, "batched bead phase");
    }
    e = fpd::launch_lattice_batch(b->precision, b->insts_d, b->tiles_d, b->ntiles, b->pool, b->tab[0], b->tab[1], mk,
                                  gp, nbl > 0 ? 1 : 0, b->variant, b->any_mrt, st);
    if (e != cudaSuccess) return bcuda(b, e, "batched lattice sweep");
    return FPD_OK;
}

// Capture kGraphSteps steps starting at a global step g > rebuild_gstep with
// g % kMaskBufs == p (every instance past its first step) on a private
// stream; the graph replays on the batch's stream.
int capture_bchunk(fpd_batch *b, int p) {
    cudaError_t e;
    if (!b->cap_stream && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bcuda(b, e, "capture stream");
    // a start step with the same mask buffer and parity, past the last reset
    int64_t g0 = b->rebuild_gstep + 1;
    g0 += ((p - g0 % fpd::kMaskBufs) % fpd::kMaskBufs + fpd::kMaskBufs) % fpd::kMaskBufs;
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bcuda(b, e, "begin capture");
    int rc = FPD_OK;
    for (int i = 0; i < fpd::kGraphSteps && rc == FPD_OK; ++i) rc = enqueue_bstep(b, b->cap_stream, g0 + i, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc != FPD_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bcuda(b, e, "end capture");
    e = cudaGraphInstantiate(&b->graph[p], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[p] = nullptr;
        return bcuda(b, e, "graph instantiate");
    }
    return FPD_OK;
}

}  // namespace

int fpd_batch_run(fpd_batch *b, int64_t max_steps, int64_t *steps_done) {
    if (!b) return FPD_EINVAL;
    if (steps_done) *steps_done = 0;
    if (max_steps < 0) return bfail(b, FPD_EINVAL, "max_steps must be >= 0");
    int64_t chunk = max_steps;
    int nactive = 0;
    double cells = 0.0;
    for (auto &sl : b->slots)
        if (sl.state == kActive) {
            chunk = std::min(chunk, sl.steps_req - sl.steps_done);
            ++nactive;
            cells += (double)sl.inst.nx * sl.inst.ny;
        }
    if (nactive == 0 || chunk <= 0) return FPD_OK;
    int rc;
    if (b->dirty && (rc = rebuild(b)) != FPD_OK) return rc;
    // watchdog pass over every resident instance's populations (between
    // captured chunks, never inside one)
    auto watch = [b]() -> int {
        cudaError_t e = fpd::launch_watch(b->precision, b->insts_d, b->insts_h[0], b->tiles_d, b->ntiles, b->pool,
                                          (int)(b->gstep & 1), b->status, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "watchdog launch");
        b->watch_next = (b->gstep / fpd::kWatchSteps + 1) * fpd::kWatchSteps;
        return FPD_OK;
    };
    for (int64_t t = 0; t < chunk;) {
        if (b->gstep >= b->watch_next && (rc = watch()) != FPD_OK) return rc;
        // on the first step after admissions the new instances skip the
        // bead advance (their table is the initial one)
        const bool any_first = b->n_old != b->n_all;
        // whole chunks of steps with every instance past its first step and
        // the masks carried over from the previous step replay a captured
        // graph (launch sizes and pointers fixed until the next rebuild)
        if (!any_first && b->gstep > b->rebuild_gstep && chunk - t >= fpd::kGraphSteps) {
            const int p = (int)(b->gstep % fpd::kMaskBufs);
            if (!b->graph[p] && (rc = capture_bchunk(b, p)) != FPD_OK) return rc;
            cudaError_t e = cudaGraphLaunch(b->graph[p], b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "batched step graph");
            b->gstep += fpd::kGraphSteps;
            t += fpd::kGraphSteps;
            continue;
        }
        if ((rc = enqueue_bstep(b, b->stream, b->gstep, any_first)) != FPD_OK) return rc;
        b->gstep++;
        ++t;
        if (any_first) {
            for (auto &sl : b->slots)
                if (sl.state == kActive) sl.first = false;
            b->n_old = b->n_all;
        }
    }
    // and after the run, so that an instance reaching its count is checked
    // before it is reported finished
    if ((rc = watch()) != FPD_OK) return rc;
    b->cell_updates += cells * (double)chunk;
    for (auto &sl : b->slots)
        if (sl.state == kActive) {
            sl.steps_done += chunk;
            if (sl.steps_done >= sl.steps_req) {
                sl.state = kDone;
                b->dirty = true;
            }
        }
    if (steps_done) *steps_done = chunk;
    return FPD_OK;
}

int fpd_batch_set_tuning(fpd_batch *b, int32_t variant) {
    if (!b) return FPD_EINVAL;
    if (variant < 0 || variant >= fpd::kLatticeVariants)
        return bfail(b, FPD_EINVAL, "tuning variant must be in [0, %d)", fpd::kLatticeVariants);
    if (variant != b->variant) {
        drop_bgraphs(b);
        b->variant = variant;
    }
    return FPD_OK;
}

int fpd_batch_sync(fpd_batch *b) {
    if (!b) return FPD_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? FPD_OK : bcuda(b, e, "batch synchronize");
}

int fpd_batch_poll(fpd_batch *b, int32_t *done_slots, int32_t capacity, int32_t *n_done) {
    if (!b || !n_done) return FPD_EINVAL;
    int rc = fpd_batch_sync(b);
    if (rc) return rc;
    // instances with a non-finite value leave the running set as failed
    std::vector<unsigned> st(b->max_slots);
    cudaError_t e = cudaMemcpy(st.data(), b->status, st.size() * sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read status");
    for (int s = 0; s < b->max_slots; ++s) {
        Slot &sl = b->slots[s];
        if ((sl.state == kActive || (sl.state == kDone && !sl.reported)) && (st[s] & fpd::kFlagNonFinite)) {
            if (sl.state == kActive) b->dirty = true;
            sl.state = kFailed;
        }
    }
    int n = 0;
    for (int s = 0; s < b->max_slots && n < capacity; ++s) {
        Slot &sl = b->slots[s];
        if ((sl.state == kDone || sl.state == kFailed) && !sl.reported) {
            sl.reported = true;
            if (done_slots) done_slots[n] = s;
            ++n;
        }
    }
    *n_done = n;
    return FPD_OK;
}

int fpd_batch_slot_info(fpd_batch *b, int32_t slot, int64_t out[6]) {
    if (!b || !out || slot < 0 || slot >= b->max_slots) return b ? bfail(b, FPD_EINVAL, "bad slot") : FPD_EINVAL;
    const Slot &sl = b->slots[slot];
    out[0] = sl.inst.nx;
    out[1] = sl.inst.ny;
    out[2] = sl.inst.nb;
    out[3] = sl.steps_done;
    out[4] = sl.steps_req;
    out[5] = sl.state;
    return FPD_OK;
}

static int slot_ok(fpd_batch *b, int32_t slot);

int fpd_batch_slot_flags(fpd_batch *b, int32_t slot, uint32_t *flags) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    if (!flags) return bfail(b, FPD_EINVAL, "NULL output");
    if ((rc = fpd_batch_sync(b))) return rc;
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, b->status + slot, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read status");
    *flags = v;
    return FPD_OK;
}

static int slot_ok(fpd_batch *b, int32_t slot) {
    if (!b) return FPD_EINVAL;
    if (slot < 0 || slot >= b->max_slots || b->slots[slot].state == kFree)
        return bfail(b, FPD_EINVAL, "slot %d is not in use", slot);
    return FPD_OK;
}

int fpd_batch_read_fields(fpd_batch *b, int32_t slot, double *ux, double *uy, double *rho) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    const Slot &sl = b->slots[slot];
    const fpd::Inst &I = sl.inst;
    const size_t n = (size_t)I.nx * I.ny;
    if ((rc = ensure_bscratch(b, 3 * n * sizeof(double)))) return rc;
    const int64_t l = sl.steps_done;
    const int ct = l == 0 ? 0 : (int)((l - 1) & 1);
    cudaError_t e = fpd::launch_fields(b->precision, nullptr, I, b->pool, b->tab[ct], nullptr, (int)(l & 1),
                                       b->scratch, b->scratch + n, b->scratch + 2 * n, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "fields kernel");
    double *dst[3] = {ux, uy, rho};
    for (int i = 0; i < 3; ++i)
        if (dst[i] && (e = cudaMemcpyAsync(dst[i], b->scratch + i * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                                           b->stream)) != cudaSuccess)
            return bcuda(b, e, "copy fields");
    return fpd_batch_sync(b);
}

int fpd_batch_internal_flow(fpd_batch *b, int32_t slot, double *eps) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    if (!eps) return bfail(b, FPD_EINVAL, "NULL output");
    const Slot &sl = b->slots[slot];
    const fpd::Inst &I = sl.inst;
    if (I.nb == 0) return fpd_batch_sync(b);
    if ((rc = ensure_bscratch(b, 2 * (size_t)I.nb * sizeof(double)))) return rc;
    const int64_t l = sl.steps_done;
    const int ct = l == 0 ? 0 : (int)((l - 1) & 1);
    cudaError_t e = fpd::launch_internal_flow(b->precision, I, b->pool, b->tab[ct], (int)(l & 1), b->scratch,
                                              b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "internal-flow kernel");
    std::vector<double> h(2 * (size_t)I.nb);
    if ((e = cudaMemcpyAsync(h.data(), b->scratch, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream)) !=
        cudaSuccess)
        return bcuda(b, e, "copy internal flow");
    if ((rc = fpd_batch_sync(b))) return rc;
    for (int q = 0; q < I.nb; ++q) eps[q] = h[2 * q] / h[2 * q + 1];
    return FPD_OK;
}

int fpd_batch_read_populations(fpd_batch *b, int32_t slot, double *f) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    if (!f) return bfail(b, FPD_EINVAL, "NULL output");
    const Slot &sl = b->slots[slot];
    const fpd::Inst &I = sl.inst;
    const size_t n = 9 * (size_t)I.nx * I.ny;
    if ((rc = ensure_bscratch(b, n * sizeof(double)))) return rc;
    cudaError_t e = fpd::launch_read_pops(b->precision, nullptr, I, b->pool, (int)(sl.steps_done & 1), b->scratch,
                                          b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, b->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "read populations");
    return fpd_batch_sync(b);
}

int fpd_batch_read_beads(fpd_batch *b, int32_t slot, double *pos, double *vel, double *force, double *support) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    if ((rc = fpd_batch_sync(b))) return rc;
    const Slot &sl = b->slots[slot];
    const int nb = sl.inst.nb, off = sl.inst.bead_off;
    if (nb == 0) return FPD_OK;
    const int64_t l = sl.steps_done;
    const fpd::BeadTab &t = b->tab[l == 0 ? 0 : (int)((l - 1) & 1)];
    std::vector<double> a(nb), c(nb);
    auto pair = [&](double *dst, const double *dx, const double *dy) -> int {
        if (!dst) return FPD_OK;
        cudaError_t e = cudaMemcpy(a.data(), dx + off, nb * sizeof(double), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(c.data(), dy + off, nb * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bcuda(b, e, "copy beads");
        for (int i = 0; i < nb; ++i) {
            dst[2 * i] = a[i];
            dst[2 * i + 1] = c[i];
        }
        return FPD_OK;
    };
    if ((rc = pair(pos, t.Rx, t.Ry))) return rc;
    if ((rc = pair(vel, t.Vx, t.Vy))) return rc;
    if ((rc = pair(force, t.Fx, t.Fy))) return rc;
    if (support) {
        cudaError_t e = cudaMemcpy(support, t.S + off, nb * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bcuda(b, e, "copy support sums");
    }
    return FPD_OK;
}

int fpd_batch_remove(fpd_batch *b, int32_t slot) {
    int rc = slot_ok(b, slot);
    if (rc) return rc;
    if ((rc = fpd_batch_sync(b))) return rc;
    Slot &sl = b->slots[slot];
    b->pop_alloc.release(sl.inst.pop_off, sl.pop_len);
    if (sl.bead_len > 0) b->bead_alloc.release(sl.inst.bead_off, sl.bead_len);
    if (sl.state == kActive) b->dirty = true;
    sl = Slot();
    return FPD_OK;
}

int fpd_batch_stats(fpd_batch *b, double out[8]) {
    if (!b || !out) return FPD_EINVAL;
    double active = 0, cells = 0, done = 0;
    for (auto &sl : b->slots) {
        if (sl.state == kActive) {
            active += 1;
            cells += (double)sl.inst.nx * sl.inst.ny;
        } else if (sl.state == kDone) {
            done += 1;
        }
    }
    out[0] = active;
    out[1] = cells;
    out[2] = done;
    out[3] = (double)b->pop_alloc.used() * (double)b->elem;
    out[4] = (double)b->pool_elems * (double)b->elem;
    out[5] = (double)b->gstep;
    out[6] = b->cell_updates;
    out[7] = (double)b->bead_alloc.used();
    return FPD_OK;
}

const char *fpd_batch_last_error(const fpd_batch *b) { return b ? b->err.c_str() : ""; }

int fpd_batch_destroy(fpd_batch *b) {
    if (!b) return FPD_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return FPD_OK;
}

// Up to n steps of every active instance: fpd_batch_run repeated until n
// steps are done or no instance is active (each run stops where an instance
// reaches its requested count).
int fpd_batch_step(fpd_batch *b, int64_t n) {
    if (!b) return FPD_EINVAL;
    if (n < 0) return bfail(b, FPD_EINVAL, "n must be >= 0");
    for (int64_t done = 0; done < n;) {
        int64_t d = 0;
        const int rc = fpd_batch_run(b, n - done, &d);
        if (rc != FPD_OK) return rc;
        if (d == 0) break;
        done += d;
    }
    return FPD_OK;
}

// Velocity field and bead positions of one instance (any pointer may be
// NULL): fpd_batch_read_fields and fpd_batch_read_beads in one call.
int fpd_batch_read(fpd_batch *b, int32_t slot, double *ux, double *uy, double *pos) {
    if (!b) return FPD_EINVAL;
    int rc = FPD_OK;
    if ((ux || uy) && (rc = fpd_batch_read_fields(b, slot, ux, uy, nullptr)) != FPD_OK) return rc;
    if (pos && (rc = fpd_batch_read_beads(b, slot, pos, nullptr, nullptr, nullptr)) != FPD_OK) return rc;
    return FPD_OK;
}

}  // extern "C"
