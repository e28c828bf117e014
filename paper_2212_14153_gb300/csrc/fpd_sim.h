// fpd_sim.h -- the state behind an fpd_sim handle (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/fpd.h"
#include "fpd_kernels.h"

struct fpd_sim {
    fpd_params p{};
    fpd::Inst inst{};
    fpd::Inst *inst_d = nullptr;
    int precision = 0;
    size_t elem = 8;
    void *state = nullptr;          // one block holding pool, tables, masks, counters, instance record
    bool owns_state = true;         // false: caller workspace (fpd_create_ex), never freed here
    void *pool = nullptr;           // 9 planes of pitch * ny elements
    size_t pool_bytes = 0, tab_bytes = 0, mask_bytes = 0;  // sizes of pool, both tables, all masks
    double *tabmem = nullptr;       // two bead tables
    fpd::BeadTab tab[2]{};
    unsigned *counters = nullptr;   // one per instance (bead-phase last-block)
    unsigned *status = nullptr;     // sticky FPD_FLAG_* bits of the instance (device word)
    unsigned *masks[fpd::kMaskBufs] = {};  // per-tile bead masks, in rotation by step (t % kMaskBufs)
    double *scratch = nullptr;      // fields / populations / diagnostics
    size_t scratch_bytes = 0;
    cudaStream_t stream = nullptr;
    int64_t nstep = 0;
    double nu_f = 0, k_s = 0, k_b = 0, k_ev = 0, gamma_dot = 0;
    std::string err;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Rec> recs;
    double ms[2] = {0, 0};
    double launches[2] = {0, 0};
    // captured step chunks, one per starting parity (see fpd_step)
    bool use_graphs = true;
    double *host_stage = nullptr;  // pinned staging for bead reads (7 nb doubles)
    // completion events of stream-ordered bead reads, by ticket % kReadTickets
    static constexpr int kReadTickets = 8;
    cudaEvent_t read_ev[kReadTickets] = {};
    uint64_t read_seq = 0;  // tickets issued so far
    // per-step bead export (fpd_export_beads): mapped page-locked ring, its
    // device alias, slot count and stride (doubles), the device-side export
    // counter (in the state block) and the step count of export 0
    double *ex_ring = nullptr, *ex_ring_d = nullptr;
    int ex_slots = 0, ex_stride = 0;
    unsigned long long *ex_count = nullptr;
    int64_t ex_first = 0;
    bool early_cold = true;  // unmarked tiles update before the bead phase ends (same results)
    // bytes the staged sweep's copies are told to expect beyond what they
    // move (FPD_TEST_COPY_SHORTFALL=1: 16), so that its bounded wait runs
    // out in a failure-handling test; 0 otherwise
    unsigned copy_shortfall = 0;
    int64_t watch_next = fpd::kWatchSteps;  // step count at which the next watchdog pass runs
    int variant = 0;  // lattice sweep variant (see launch_lattice)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph[fpd::kMaskBufs] = {};  // captured step chunks, by first step % kMaskBufs
};

namespace fpd {
// Validate p and fill s->inst and the derived constants of s (no device
// work).  On error the text is available from create_error().
int derive_params(fpd_sim *s, const fpd_params &p);
const char *create_error();
// Initial bead positions of p (false if any is not finite).
bool initial_beads(const fpd_params &p, double l0, std::vector<double> &Rx, std::vector<double> &Ry);
}  // namespace fpd
