// fpd_kernels.h -- host-side launch wrappers of the FPD kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "fpd_device.cuh"

namespace fpd {

constexpr int kTileX = 32;       // lattice tile: 32 x 8 cells, one thread each
constexpr int kTileY = 8;
constexpr int kMaxBeads = 256;   // beads per instance (shared-memory tables)
constexpr int kBeadThreads = 128;  // per bead CTA: more beads resident at once (batched sweep +9 %)
constexpr int kBeadThreadsFew = 256;  // per bead CTA when the beads fit on the SMs one per SM
constexpr int kBeadLanes = 256;  // virtual lanes of the per-bead sums (any CTA size gives the same bits)
static_assert(kBeadLanes % kBeadThreads == 0 && kBeadLanes % kBeadThreadsFew == 0 &&
                  kBeadLanes / kBeadThreads <= 2 && kBeadLanes / kBeadThreadsFew <= 2,
              "a bead thread holds one or two virtual lanes");
constexpr int kGraphSteps = 32;  // time steps per captured graph chunk
// Tile-mask buffers, used in rotation: the bead phase of step t marks buffer
// t % kMaskBufs; the sweep of step t reads it (hot tiles) and buffer
// (t - 1) % kMaskBufs (tiles it may update without waiting), and zeroes
// buffer (t + 1) % kMaskBufs for the next bead phase.  kGraphSteps is a
// multiple of kMaskBufs, so a captured chunk depends on t % kMaskBufs only.
constexpr int kMaskBufs = 4;
static_assert(kGraphSteps % kMaskBufs == 0, "graph chunks must keep the mask rotation");

// The masks one sweep uses.  early_cold = 1 lets tiles that no bead marked
// in the previous bead phase (read) update without waiting for the current
// one; valid when `prev` holds that phase's marks (not after the masks were
// reset) and the sweep follows the bead phase as a programmatic dependent.
struct SweepMasks {
    const unsigned *read;  // this step's marks
    const unsigned *prev;  // the previous bead phase's marks
    unsigned *clear;       // zeroed for the next bead phase
    int early_cold;
    unsigned *status = nullptr;  // the instance's status word (staged sweep)
    unsigned copy_shortfall = 0;  // test only: extra bytes the staged copies expect (their waits run out)
};

// Sticky per-instance status bits, set on the device (values of the
// FPD_FLAG_* constants of fpd.h).  kFlagFastBead: a bead phase found a bead
// velocity component of magnitude >= kFastBead cells per step (or a
// non-finite one); that phase and every later one then mark all tiles of the
// instance, so that no sweep updates a tile early any more (that path
// assumes a bead moves less than a cell per step).  kFlagNonFinite: a
// non-finite bead velocity, or a non-finite population found by the
// watchdog.  kFlagCopyTimeout: a CTA of the staged sweep gave up waiting
// for the bulk copy of its block (bounded wait) and left the block unwritten.
constexpr unsigned kFlagFastBead = 1u;
constexpr unsigned kFlagNonFinite = 2u;
constexpr unsigned kFlagCopyTimeout = 4u;
constexpr double kFastBead = 0.5;
// Steps between two watchdog passes over the populations (a multiple of
// kGraphSteps, so that the passes fall between captured chunks).
constexpr int kWatchSteps = 1024;

// One fused collide-stream-bounce-back sweep of a single instance (Sec. 2.3
// item (2) with the item-(1) overlay of Eqs. 1, 2, 4 evaluated in hot tiles),
// with the tile masks of SweepMasks.
// after_beads = 1 when the previous launch on the stream is the bead phase
// of the same step: the sweep is then launched as a programmatic dependent
// of it and loads its populations before waiting for it.
// variant: 0 = one cell per thread (32 x 8 threads), 1 = two cells per
// thread along x, adjacent (FP32, FP16 storage) or 16 apart (FP64) (16 x 8
// threads), 2 = lattice_vec_width(precision) cells per
// thread along x with vector loads and stores ((32 / width) x 8 threads;
// needs nx % width == 0, otherwise variant 0 runs), 3 and 4 = variant 1's
// threads on blocks of 2 or 4 (FP32) / 4 or 8 (FP16) tiles stacked in y,
// whose populations a bulk copy stages in shared memory (FP32 and FP16
// storage with masks.status set; otherwise, and in batches, variant 1
// runs); same tiles, same results.
constexpr int kLatticeVariants = 5;
// Kernel attributes of the staged sweep on the current device (once per
// instance creation, outside any stream capture).
cudaError_t prepare_lattice_kernels();
inline int lattice_vec_width(int precision) { return precision == 0 ? 2 : 4; }
cudaError_t launch_lattice(int precision, const Inst *inst_d, const Inst &inst_h, void *pool, BeadTab tab,
                           const SweepMasks &masks, int parity, int after_beads, int variant, cudaStream_t st);

// Bead phase (items (3) then (1)): one CTA per bead of any instance
// (blist[i] = (instance slot, global bead index); NULL = instance 0, bead i;
// every bead of an instance must be in the same launch).  With the instance's
// step parity p = gparity ^ par_xor it reads table p ^ 1 and writes table p
// (tab0 / tab1); advance = 0 only computes S and F of table p from its own R
// (initialisation).  Every bead ORs its bit into the mask of each lattice
// tile its support reaches (mask_write, zeroed beforehand).
// pdl = 1 launches the bead phase as a programmatic dependent of the
// previous sweep: it waits for that sweep first thing and releases the next
// sweep at once, so the next sweep's unmarked tiles overlap the whole phase.
// Per-step export of a single instance's finished bead table to host
// memory (ring == nullptr: none): the instance's last CTA writes R_x, R_y,
// V_x, V_y, F_x, F_y, S (nb doubles each) after kExportHeader doubles into
// slot k % slots of the ring (stride doubles a slot, device address of
// mapped page-locked memory), then k + 1 into the slot's first 64-bit word,
// and increments *count (k: the exports before this one).
constexpr int kExportHeader = 8;
struct BeadExport {
    double *ring = nullptr;
    unsigned long long *count = nullptr;
    int slots = 0;
    int stride = 0;
};
// status: per-instance status words (indexed by instance slot), where the
// instance's last CTA sets kFlagFastBead (and kFlagNonFinite) when a bead
// velocity component reaches kFastBead in magnitude (or is not finite), and
// marks every tile of a flagged instance in mask_write; NULL: not checked.
cudaError_t launch_beads(int precision, const Inst *inst_d, const int2 *blist, int nb_total,
                         const void *pool, BeadTab tab0, BeadTab tab1, unsigned *mask_write, int gparity,
                         int advance, unsigned *counters, int pdl, cudaStream_t st, BeadExport ex = BeadExport{},
                         unsigned *status = nullptr);

// Watchdog: sets kFlagNonFinite in status[slot] of every instance holding a
// non-finite population at its current step.  Batch form: tiles[t] =
// (slot, by << 16 | bx) over insts (device records, each at its parity
// gparity ^ par_xor); single form (tiles == NULL): every tile of inst_h at
// parity gparity, status[0].
cudaError_t launch_watch(int precision, const Inst *insts, const Inst &inst_h, const int2 *tiles, int ntiles,
                         const void *pool, int gparity, unsigned *status, cudaStream_t st);

// Batched sweep over a packed tile list of many instances (tiles[t] =
// (slot, by << 16 | bx)); each instance at its own parity.  Under variant 2
// the tiles of an instance whose nx is not a multiple of the vector width
// run with that many cells per thread along y on the same threads.
// any_mrt = 1 when some instance uses constant Lallemand-Luo rates
// (collision 1): the sweep then runs variant 0 with both collision forms.
// A single instance with collision 1 runs variant 0 as well.
cudaError_t launch_lattice_batch(int precision, const Inst *insts, const int2 *tiles, int ntiles, void *pool,
                                 BeadTab tab0, BeadTab tab1, const SweepMasks &masks, int gparity, int after_beads,
                                 int variant, int any_mrt, cudaStream_t st);

cudaError_t launch_init(int precision, const Inst *inst_d, const Inst &inst_h, void *pool, int couette,
                        cudaStream_t st);

cudaError_t launch_fields(int precision, const Inst *inst_d, const Inst &inst_h, const void *pool, BeadTab tab,
                          const unsigned *mask, int parity, double *ux, double *uy, double *rho, cudaStream_t st);

// eps_v numerator and denominator of every bead of the instance (Sec. 3.2):
// out[2 q] = sum_x phi_q |u - V_q|^2, out[2 q + 1] = sum_x phi_q, FP64.
cudaError_t launch_internal_flow(int precision, const Inst &inst_h, const void *pool, BeadTab tab, int parity,
                                 double *out, cudaStream_t st);

cudaError_t launch_read_pops(int precision, const Inst *inst_d, const Inst &inst_h, const void *pool,
                             int parity, double *f, cudaStream_t st);
cudaError_t launch_write_pops(int precision, const Inst *inst_d, const Inst &inst_h, void *pool, int parity,
                              const double *f, cudaStream_t st);

// FP64 partial sums (mass, px, py, non-finite count) per block into
// partial[4 * nblocks]; returns the number of blocks used.
int diag_blocks(const Inst &inst_h);
cudaError_t launch_diag(int precision, const Inst *inst_d, const Inst &inst_h, const void *pool, int parity,
                        double *partial, cudaStream_t st);

}  // namespace fpd
