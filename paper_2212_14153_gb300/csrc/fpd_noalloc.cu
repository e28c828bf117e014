// fpd_noalloc.cu -- fpd_diag_noalloc: the mass / momentum / non-finite check
// of fpd_diag without any device-memory allocation.
//
// fpd_diag reduces the populations into per-block partial sums held in the
// handle's scratch buffer, which it allocates with cudaMalloc the first time
// (or grows when a larger buffer is needed).  Some callers cannot allow a
// device allocation at the moment they want the check: a serving loop that
// has handed every byte of device memory to resident instances, code that
// runs while another thread captures or replays work on the device (a
// cudaMalloc may synchronise the device or be refused during capture), or an
// embedding application whose own allocator owns device memory.  This entry
// point keeps its scratch in a fixed file-scope device array instead.
//
// Scratch: g_diag_scratch, 4 * 1024 + 4 doubles (32 800 bytes) per device
// that loads the library, held until the process exits.  The reduction
// launches at most 1024 blocks (larger lattices are strided), which is the
// largest partial-sum count the array holds; the block count is checked and
// a larger one is refused with FPD_EINVAL.  Each call overwrites every slot
// it reads (partials of the blocks it launches, then the 4 totals), so no
// slot needs clearing between calls.  All calls on a device share the one
// array: calls whose device work overlaps (other streams, other handles on
// the same device, other host threads) race on it and must be serialised by
// the caller.
//
// The array's device address is looked up with cudaGetSymbolAddress once per
// device and CUDA context, and cached with the context's ID: an application
// that calls cudaDeviceReset gets a new primary context in which the library
// module, and with it the array, is loaded afresh at another address, so a
// cached address from the old context is never used in the new one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fpd_sim.h"

namespace {

constexpr int kNoAllocBlocks = 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_diag_scratch[4 * kNoAllocBlocks + 4];

std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};        // device address of g_diag_scratch per device
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // ID of the context that address belongs to

// ID of the calling thread's current context (driver entry points resolved
// through the runtime, so that no link to the driver library is needed).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
cudaError_t current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        get_current = (CtxGetCurrentFn)a;
        get_id = (CtxGetIdFn)b;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorContextIsDestroyed;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    return cudaSuccess;
}

// Sum the per-block partials in block order (the order fpd_diag sums them
// on the host) into the 4 slots after the partials.
__global__ void k_diag_finish(const double *__restrict__ partial, int nblocks, double *__restrict__ total) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double m = 0.0, px = 0.0, py = 0.0, bad = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        m += partial[4 * b];
        px += partial[4 * b + 1];
        py += partial[4 * b + 2];
        bad += partial[4 * b + 3];
    }
    total[0] = m;
    total[1] = px;
    total[2] = py;
    total[3] = bad;
}

int set_err(fpd_sim *s, int code, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[320];
    if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else std::snprintf(buf, sizeof buf, "%s", msg);
    s->err = buf;
    return code;
}

}  // namespace

extern "C" int fpd_diag_noalloc(fpd_sim *s, double out[4]) {
    if (!s || !out) {
        if (s) set_err(s, FPD_EINVAL, "fpd_diag_noalloc: NULL argument");
        return FPD_EINVAL;
    }
    const fpd::Inst &I = s->inst;
    const int nblocks = fpd::diag_blocks(I);
    if (nblocks > kNoAllocBlocks) return set_err(s, FPD_EINVAL, "fpd_diag_noalloc: reduction needs more than 1024 partial blocks");

    // the device that holds this handle's state
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, s->pool);
    if (e != cudaSuccess) return set_err(s, FPD_ECUDA, "fpd_diag_noalloc: cudaPointerGetAttributes", e);
    const int dev = attr.device;
    if (dev < 0 || dev >= kMaxDevices) return set_err(s, FPD_EINVAL, "fpd_diag_noalloc: device index out of range");
    int cur = -1;
    e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return set_err(s, FPD_ECUDA, "fpd_diag_noalloc: cudaGetDevice", e);
    if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
        return set_err(s, FPD_ECUDA, "fpd_diag_noalloc: cudaSetDevice", e);

    int rc = FPD_OK;
    double total[4] = {0.0, 0.0, 0.0, 0.0};
    double *scratch = nullptr;
    {
        // set-up, once per device and context, with that device current: the
        // host-side name g_diag_scratch is not a device address; ask the
        // runtime for it
        std::lock_guard<std::mutex> lock(g_setup_mu);
        unsigned long long ctx_id = 0;
        e = current_context_id(&ctx_id);
        if (e != cudaSuccess) {
            rc = set_err(s, FPD_ECUDA, "fpd_diag_noalloc: current context", e);
        } else if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx_id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_diag_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                rc = set_err(s, FPD_ECUDA, "fpd_diag_noalloc: cudaGetSymbolAddress", e);
            } else {
                g_scratch_addr[dev] = (double *)p;
                g_scratch_ctx[dev] = ctx_id;
            }
        }
        scratch = g_scratch_addr[dev];
    }
    if (rc == FPD_OK) {
        e = fpd::launch_diag(s->precision, s->inst_d, I, s->pool, (int)(s->nstep & 1), scratch, s->stream);
        if (e == cudaSuccess) {
            k_diag_finish<<<1, 1, 0, s->stream>>>(scratch, nblocks, scratch + 4 * kNoAllocBlocks);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(total, scratch + 4 * kNoAllocBlocks, sizeof total, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = set_err(s, FPD_ECUDA, "fpd_diag_noalloc: reduction", e);
    }
    if (cur != dev && cur >= 0) cudaSetDevice(cur);
    if (rc != FPD_OK) return rc;

    out[0] = (double)I.nx * I.ny + total[0];  // sum of w_k over cells is 1 per cell
    out[1] = total[1];
    out[2] = total[2];
    out[3] = (double)s->nstep;
    if (total[3] > 0 || !std::isfinite(total[0]) || !std::isfinite(total[1]) || !std::isfinite(total[2])) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "non-finite populations after %lld steps", (long long)s->nstep);
        return set_err(s, FPD_ENAN, buf);
    }
    return FPD_OK;
}
