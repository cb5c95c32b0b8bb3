// Internal declarations shared by the CUDA translation units of libpotts_lr.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace plr {

constexpr int kSweepThreads = 256;  // threads of one sweep CTA (one CTA per slot)
constexpr int kSiteBlock = 32;      // sites decided by one warp between field updates
constexpr int kAuxThreads = 256;    // threads of the init / measure / rebuild CTAs
constexpr int kMaxQ = 16;           // largest q (4-bit packed spins)
constexpr int kMaxL = 65536;        // largest L (16-bit positions in the direct rebuild)
constexpr int kChunk = 128;         // K sites per chunk of the tensor-core rebuild
constexpr int kMeasMaxParts = 32;   // largest split of one slot's measurement over CTAs
constexpr int kNearLogCap = 256;    // near-tie events logged per job (all are counted)
// default bounds of the device waits (potts_lr_set_wait_limits)
constexpr unsigned long long kTcWaitNs = 4000000000ull;  // each pipeline wait of the tensor-core rebuild: 4 s
constexpr unsigned long long kSchedWaitNs = 50000;       // sweep CTAs waiting for the others' first claims
// precision modes (JobDev::precision, the C ABI's POTTS_LR_FP64 / FP32 / FX64)
constexpr int kPrecFP64 = 0;        // FP64 fields
constexpr int kPrecFP32 = 1;        // FP32 fields, tensor-core rebuilds
constexpr int kPrecFX64 = 2;        // 64-bit fixed-point fields: exact integer updates

// Everything a kernel needs to know about one job, resident in device memory.
// Arrays indexed by "replica" follow the configuration; arrays indexed by
// "slot" belong to a temperature.  map[slot] = replica currently at that slot.
struct JobDev {
    int L, q, Lpad, W, R, c, precision;
    int recompute_every;  // FP32 mode: longest interval K between field rebuilds (0 = on request only)
    int h_smem, j_smem;   // sweep kernel: fields / coupling table staged in shared memory
    int rf;               // register-resident sweep configuration (0 = none; FP32 mode 1..8, FX64 mode 1..6)
    int cl;               // CTAs of the cluster that shares a slot's fields in shared memory (0 = none; 2, 4, 8)
    int rc;               // CTAs of the cluster that holds a slot's fields in registers (0 = none; 2, 4, 8)
    int random_sites;     // direct sweep: attempt m at a site drawn from Philox counter (m, slot, sweep, 3)
    uint32_t key0, key1;  // Philox key (seed low, high)
    double jtot;          // sum_r J*(r)
    const double* J64d;   // doubled table: J64d[m] = J*(m mod L), m = 0..2L-1
    const float* J32d;    // the same in FP32
    const long long* Jfxd;  // FX64 mode: the same rounded to the field grid, llrint(J*(m mod L) 2^F)
    double fx_scale;        // FX64 mode: 2^-F, the value of one field unit
    uint32_t* spins;      // [replica][W] packed, 4 bits per spin, spin i at bits 4(i%8) of word i/8
    void* fields;         // [replica][q][Lpad], double (FP64), float (FP32) or long long (FX64, units of 2^-F)
    double* E;            // running energy per replica
    int* map;             // slot -> replica
    const double* beta;   // per slot
    uint32_t* nsweep;     // sweeps done, per slot
    uint32_t* nexch;      // exchange steps done [1]
    unsigned long long* acc_flip;  // per slot
    unsigned long long* acc_swap;  // per pair (t, t+1), R entries
    unsigned long long* near;      // [2]: Metropolis, exchange near ties
    int4* near_log;                // [kNearLogCap]: {kind | decision << 1, slot or pair, sweep or exchange
                                   // index, attempt or stage} of the first near ties (near_tie.cuh)
    unsigned* near_log_n;          // near ties logged since create (the log keeps the first kNearLogCap)
    double* meas_E;       // per slot, written by the measure kernel
    double* meas_M;
    double* meas_part;    // [slot][kMeasMaxParts]: the measure kernel's partial energy sums
    int* meas_ticket;     // per slot: parts of the running measurement done (0 between launches)
    int meas_parts;       // CTAs per slot of the measure kernel (measure_parts(L))
    unsigned long long* err_bits;  // fields_error result (double bits, max)
    const uint16_t* Jhank;         // FP32 mode: BF16 parts hi, mid, lo of J* as Hankel core matrices,
                                   // [3][hank_cores][8][8] (the tensor-core rebuild's A operand)
    uint16_t* Xoh;                 // FP32 mode: one-hot spins, the rebuild's B operand,
                                   // [Lc / kChunk][NG][16][8][8] (Lc: L rounded up to kChunk)
    int hank_cores;                // core matrices per part of Jhank: Lc / 4 - 1
    int NG;                        // 8-row groups of the B operand: q R rounded up to 128, / 8
    int* status;                   // 0 ok; 1 a bounded device wait expired
    unsigned long long tc_wait_ns; // bound of each pipeline wait of the tensor-core rebuild (kTcWaitNs)
    int* sched;                    // FP32 rebuild schedule: [0] current interval k, [1] sweep of the next rebuild,
                                   // [2] rebuilds done (policy updates), [3] sweep of the last energy anchor
    unsigned long long* drift_bits;  // max |h_before - h_rebuilt| / Jtot (double bits): [0] of the rebuild
                                     // running now, [1] of the last completed one
    int tc_parts;                  // BF16 parts of J* the rebuild multiplies: 3 (hi, mid, lo), 2 (hi, mid) or
                                   // 0 = automatic (default; rebuild_parts)
};

// FP32 drift control: after each rebuild the measured drift d of the period
// halves the interval if d > kDriftHigh, doubles it (up to recompute_every)
// if d < kDriftLow; drift grows like the square root of the interval, so the
// field error stays below 1e-5 of Jtot.
constexpr double kDriftHigh = 7e-6;
constexpr double kDriftLow = 3.5e-6;

__device__ __forceinline__ bool rebuild_due(const JobDev& jb)
{
    return jb.recompute_every > 0 && jb.nsweep[0] >= (uint32_t)jb.sched[1];
}

// The exact energy that re-anchors the running FP32 energy at a scheduled
// rebuild is taken once at least kAnchorSweeps sweeps have passed since the
// last one: long chains rebuild every sweep or two, and the O(L^2) energy
// costs a quarter of their rebuild.  In between, the running energy carries
// the FP32 fields' error in the energy changes it sums (measured about 3e-5
// of Jtot per sweep, so at most about 2.4e-4 Jtot; in the exchange exponent
// that is the size of the FP32 Metropolis decisions' own error).  Explicit
// rebuilds always re-anchor.  The policy kernel, which runs after the
// measurement, moves sched[3].
constexpr int kAnchorSweeps = 8;
__device__ __forceinline__ bool anchor_due(const JobDev& jb)
{
    return jb.nsweep[0] - (uint32_t)jb.sched[3] >= (uint32_t)kAnchorSweeps;
}

// BF16 parts of a rebuild: as set, or automatically two where scheduled
// rebuilds come every sweep (there the sweep's own drift, 4e-6 to 9e-6 of Jtot,
// dwarfs the two-part split's 3e-7, and the interval cannot shrink further)
// and three elsewhere (at longer intervals the split's error would enter the
// measured drift that lets the interval grow)
__device__ __forceinline__ int rebuild_parts(const JobDev& jb)
{
    if (jb.tc_parts) return jb.tc_parts;
    return (jb.recompute_every > 0 && jb.sched[0] <= 1) ? 2 : 3;
}

// Placement of the work items of one sweep launch on the SMs.  The field
// updates of a slot cost about (accepted flips per sweep) x L, which varies
// many-fold along a temperature ladder, and the CTAs resident on one SM share
// its FP64 (or FP32) pipe; hardware placement ignores that.  A plan kernel
// orders the items by that estimate (from the slot counters) and deals the
// heaviest nsm * occ of them to (SM, resident CTA) places in serpentine order;
// sweep CTAs claim their place by SM id, then take the remaining items, in
// order, from the list (every item is claimed exactly once, wherever the
// CTAs land, so placement changes the timing only, never the results).
constexpr int kSchedMaxOcc = 8;    // resident sweep CTAs per SM that a plan can address
struct SweepSched {
    int* order;   // [n] item indices, heaviest first
    int2* sorted; // [n] the items themselves in that order (cluster launches)
    int* bins;    // [nsm * occ] item of each (SM, resident CTA) place, -1 for none
    int* claim;   // [n] 0 until an item is taken
    int* ctr;     // [nsm + 2]: arrivals per SM, next list position, CTAs past their claim
    int n, nsm, occ;
    unsigned long long wait_ns;  // longest wait for the other CTAs' first claims (kSchedWaitNs)
};
size_t sweep_sched_bytes(int n, int nsm);
// carve a SweepSched for n items out of device memory at base (sweep_sched_bytes long)
void sweep_sched_carve(char* base, int n, int nsm, SweepSched* s);
// device SM count (cached per device)
int device_sm_count();
// the plan kernel (one CTA); weights from jobs[work[i].x] counters
cudaError_t launch_sweep_plan(const JobDev* jobs_dev, const int2* work, const SweepSched& s, cudaStream_t st);
// Placement of a cluster launch (cfg: its grid, CTA size, shared memory and
// cluster attribute): when its nwork clusters are more than can be resident
// at once, the plan kernel (on st) writes the items heaviest first to
// sched->sorted and *items points there, so that the clusters dispatched
// first take the heaviest items and the light ones fill the last wave;
// otherwise *items is left as it is.
cudaError_t cluster_plan(const void* kernel, const cudaLaunchConfig_t& cfg, int nwork, const SweepSched* sched,
                         const JobDev* jobs_dev, const int2* work, const int2** items, cudaStream_t st);

// ---- host-side helpers (jstar.cpp) ----
void jstar_table(int L, double sigma, double* out);

// ---- launchers (each returns the cudaError_t of the launch) ----
// work[i] = {job index, slot}
cudaError_t launch_init_spins(const JobDev* jobs_dev, int job, int L, int W, int R, cudaStream_t st);
// the kernel variant (precision, fields in smem, table in smem) is uniform per launch
// sched: placement buffers for this work list (nullptr: one CTA per item, in order)
cudaError_t launch_sweep(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, int precision,
                         int h_smem, int j_smem, size_t smem_bytes, const SweepSched* sched, cudaStream_t st);
cudaError_t launch_exchange(const JobDev* jobs_dev, int njobs, cudaStream_t st);
// "cond" arguments: when nonzero the kernel does nothing unless the job's
// rebuild is due (rebuild_due: its sweep counter has reached the next rebuild
// of its schedule), which lets a captured CUDA graph carry the rebuild every
// step.
// anchor: 0 = measure only, 1 = measure and re-anchor the running energy.
// max_parts: the largest meas_parts among the work items' jobs.
cudaError_t launch_measure(const JobDev* jobs_dev, const int2* work, int nwork, int anchor, int cond,
                           size_t smem_bytes, int max_parts, cudaStream_t st);
int measure_parts(int L);  // CTAs per slot of the measure kernel for chain length L
// FP64 direct rebuild of the fields of every replica of job jobs_dev[0]
// (grid over element tiles x replicas).  mode 0: write fields; mode 1: compare
// with the stored fields and fold max |diff| / jtot into err_bits.
cudaError_t launch_fields_direct(const JobDev* job_dev, int L, int R, int mode, int cond, size_t smem_bytes,
                                 cudaStream_t st);
// FP32 mode: the split-BF16 tensor-core rebuild H = C . onehot(S): a one-hot
// kernel writes the B operand of the listed jobs (jobs_dev[idx[i]], i < njobs;
// idx null: jobs_dev[i]) on a grid of onehot_blocks x njobs CTAs, then the
// persistent tensor-core kernel (one CTA per SM) walks a tile table of
// (job index, first row, first column) 128 x tn output tiles (any mix of
// jobs).  tn: output tile width, 64 or 128 (tc_tile_width picks it from the
// tile counts).
cudaError_t launch_fields_tc(const JobDev* jobs_dev, const int* idx, int njobs, int onehot_blocks,
                             const int4* tiles, int ntiles, int cond, int tn, cudaStream_t st);
void tc_tiles(int job, int L, int q, int R, int tn, std::vector<int4>& out);
void tc_order_tiles(std::vector<int4>& tiles);  // full-width tiles first (the rebuild's round-robin)
long long tc_tile_count(int L, int q, int R, int tn);
int tc_tile_width(long long tiles64, long long tiles128, int nsm);
int tc_onehot_blocks(int L, int q, int R);  // one-hot grid width for one job of this shape
int tc_ng(int q, int R);                     // JobDev::NG of this shape
long long tc_hank_cores(int L);              // JobDev::hank_cores of this shape
size_t tc_hank_bytes(int L);                 // bytes of the Jhank table
size_t tc_onehot_bytes(int L, int q, int R); // bytes of the Xoh operand
// the Jhank table from the split table ([3][Lpad], part sp of J*(r) at sp Lpad + r)
void tc_hank_table(const std::vector<double>& J, const uint16_t* split, int Lpad, std::vector<uint16_t>& out);
// after a rebuild: adapt the FP32 rebuild interval of jobs[idx[i]] to the
// measured drift (one thread per job)
cudaError_t launch_rebuild_policy(const JobDev* jobs_dev, const int* idx, int njobs, int cond, cudaStream_t st);

size_t sweep_smem_bytes(const JobDev& j);

// Direct sweep (sweep_direct.cu): the paper's O(L)-per-attempt scheme, FP64,
// no fields; one CTA per work item.
size_t direct_sweep_smem_bytes(int L, int Lpad);
cudaError_t launch_sweep_direct(const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps, size_t smem,
                                cudaStream_t st);

// Cluster sweep (sweep_cluster.cu): a slot's fields (FP32, FP64 or FX64)
// spread over the shared memory of a cluster of C = 2, 4 or 8 CTAs.
size_t cluster_sweep_smem(int L, int q, int C, int precision);
int cluster_size_for(int L, int q, size_t budget, int precision);  // smallest C whose share fits (0: none)
cudaError_t launch_sweep_cluster(int C, int precision, const JobDev* jobs_dev, const int2* work, int nwork,
                                 int nsweeps, size_t smem, const SweepSched* sched, cudaStream_t st);

// Register-resident FP32 sweep (sweep_rf.cuh): configuration 1..8 =
// (E sites per update thread, update warps) = (1, 7), (2, 7), (5, 7) for
// L <= 224, 448, 1120; (5, 15) with q <= 10 for L <= 2400; (9, 15) with
// q <= 8 for L <= 4320;
// (16, 15) with q <= 5 for L <= 7680; (26, 15) with q <= 3 for L <= 12480;
// (35, 15) with q = 2 for L <= 16800; 0 if the shape does not fit in registers.
int rf_config(int L, int q);
bool rf_fits(int cfg, int L, int q);  // configuration cfg (1..8) holds L sites of q states
size_t rf_smem_bytes(int cfg, int q, int L, int Lpad);
cudaError_t launch_sweep_rf(int cfg, int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                            size_t smem, const SweepSched* sched, cudaStream_t st);
cudaError_t launch_sweep_rf_a(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_b(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_c(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_d(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_e(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_f(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_g(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
cudaError_t launch_sweep_rf_h(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                             cudaStream_t);
// Register-resident FX64 sweep (sweep_rf.cuh with 64-bit integer fields):
// configuration 1..6 = (E, update warps) = (1, 7), (2, 7), (4, 8), (5, 7),
// (5, 15), (9, 15) for L <= 224, 448, 1024, 1120, 2400, 4320 with q at most
// 16, 16, 8, 8, 5, 3; rfx_config: 4 where it fits, else the fewest sites per
// thread that hold the chain, 0 if none does.
int rfx_config(int L, int q);
bool rfx_fits(int cfg, int L, int q);
int rfx_threads(int cfg);  // threads per CTA of configuration cfg
size_t rfx_smem_bytes(int cfg, int q, int L, int Lpad);
cudaError_t launch_sweep_rfx(int cfg, int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                             size_t smem, const SweepSched* sched, cudaStream_t st);
#define PLR_RFX_DECL(tag)                                                                                    \
    cudaError_t launch_sweep_rfx_##tag(int q, const JobDev*, const int2*, int, int, size_t, const SweepSched*, \
                                       cudaStream_t);                                                          \
    size_t sweep_rfx_smem_##tag(int q, int L, int Lpad);
PLR_RFX_DECL(a)
PLR_RFX_DECL(b)
PLR_RFX_DECL(c)
PLR_RFX_DECL(d)
PLR_RFX_DECL(e)
PLR_RFX_DECL(f)
#undef PLR_RFX_DECL
// Register-resident cluster sweep (sweep_rfc.cuh): a slot's fields in the
// registers of a cluster of C = 2, 4 or 8 CTAs (FP32: 9 sites per update
// thread, q <= 8, L <= 4320 C, or 5 sites, q <= 12, L <= 2400 C; FX64: 5
// sites, q <= 7, L <= 2400 C).
bool rfc_fits(int precision, int C, int L, int q);
int rfc_cluster_for(int precision, int L, int q);  // smallest C that holds the chain (0: none)
size_t rfc_smem_bytes(int precision, int q, int C, int L);
cudaError_t launch_sweep_rfc(int precision, int C, int q, const JobDev* jobs_dev, const int2* work, int nwork,
                             int nsweeps, size_t smem, const SweepSched* sched, cudaStream_t st);
cudaError_t launch_sweep_rfc_f(int q, int C, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                               cudaStream_t);
cudaError_t launch_sweep_rfc_x(int q, int C, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                               cudaStream_t);
size_t sweep_rfc_smem_f(int q, int C, int L);
cudaError_t launch_sweep_rfc_fq(int q, int C, const JobDev*, const int2*, int, int, size_t, const SweepSched*,
                                cudaStream_t);
size_t sweep_rfc_smem_fq(int q, int C, int L);
size_t sweep_rfc_smem_x(int q, int C, int L);
size_t sweep_rf_smem_a(int q, int L, int Lpad);
size_t sweep_rf_smem_b(int q, int L, int Lpad);
size_t sweep_rf_smem_c(int q, int L, int Lpad);
size_t sweep_rf_smem_d(int q, int L, int Lpad);
size_t sweep_rf_smem_e(int q, int L, int Lpad);
size_t sweep_rf_smem_f(int q, int L, int Lpad);
size_t sweep_rf_smem_g(int q, int L, int Lpad);
size_t sweep_rf_smem_h(int q, int L, int Lpad);
size_t sweep_smem_bytes_for(int precision, int L, int Lpad, int q, int h_smem, int j_smem);
size_t direct_smem_bytes(int L, int q);

}  // namespace plr
