// Dispatch of the register-resident sweeps over their configurations
// (sweep_rf.cuh; one translation unit per configuration): FP32 fields and
// FX64 fields (64-bit integers, two registers per value).
#include "potts_internal.h"

namespace plr {

namespace {
// capacity of each register configuration: largest L (E x 32 x update warps) and q
constexpr int kRfMaxL[9] = {0, 224, 448, 1120, 2400, 4320, 7680, 12480, 16800};
constexpr int kRfMaxQ[9] = {0, 16, 16, 16, 10, 8, 5, 3, 2};
// FX64 configurations 1..6: (E, NU) = (1, 7), (2, 7), (4, 8), (5, 7), (5, 15), (9, 15)
constexpr int kRfxMaxL[7] = {0, 224, 448, 1024, 1120, 2400, 4320};
constexpr int kRfxMaxQ[7] = {0, 16, 16, 8, 8, 5, 3};
}  // namespace

bool rfx_fits(int cfg, int L, int q) { return cfg >= 1 && cfg <= 6 && L <= kRfxMaxL[cfg] && q <= kRfxMaxQ[cfg]; }

int rfx_config(int L, int q)
{
    // configuration 4 (5 sites x 7 warps) wherever it holds the chain: timed
    // on GB300 the fastest, or within 2% of it, from L = 128 to 1024 (q <= 8);
    // else the fewest sites per thread that hold it
    if (rfx_fits(4, L, q)) return 4;
    for (int cfg = 1; cfg <= 6; ++cfg)
        if (rfx_fits(cfg, L, q)) return cfg;
    return 0;
}

int rfx_threads(int cfg) { return cfg == 3 ? 288 : (cfg >= 5 ? 512 : 256); }

size_t rfx_smem_bytes(int cfg, int q, int L, int Lpad)
{
    switch (cfg) {
    case 1: return sweep_rfx_smem_a(q, L, Lpad);
    case 2: return sweep_rfx_smem_b(q, L, Lpad);
    case 3: return sweep_rfx_smem_c(q, L, Lpad);
    case 4: return sweep_rfx_smem_d(q, L, Lpad);
    case 5: return sweep_rfx_smem_e(q, L, Lpad);
    case 6: return sweep_rfx_smem_f(q, L, Lpad);
    default: return 0;
    }
}

cudaError_t launch_sweep_rfx(int cfg, int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                             size_t smem, const SweepSched* sched, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    switch (cfg) {
    case 1: return launch_sweep_rfx_a(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 2: return launch_sweep_rfx_b(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 3: return launch_sweep_rfx_c(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 4: return launch_sweep_rfx_d(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 5: return launch_sweep_rfx_e(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 6: return launch_sweep_rfx_f(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    default: return cudaErrorNotSupported;
    }
}

bool rf_fits(int cfg, int L, int q) { return cfg >= 1 && cfg <= 8 && L <= kRfMaxL[cfg] && q <= kRfMaxQ[cfg]; }

int rf_config(int L, int q)
{
    for (int cfg = 1; cfg <= 8; ++cfg)  // the fewest sites per thread that hold the chain
        if (rf_fits(cfg, L, q)) return cfg;
    return 0;
}

size_t rf_smem_bytes(int cfg, int q, int L, int Lpad)
{
    switch (cfg) {
    case 1: return sweep_rf_smem_a(q, L, Lpad);
    case 2: return sweep_rf_smem_b(q, L, Lpad);
    case 3: return sweep_rf_smem_c(q, L, Lpad);
    case 4: return sweep_rf_smem_d(q, L, Lpad);
    case 5: return sweep_rf_smem_e(q, L, Lpad);
    case 6: return sweep_rf_smem_f(q, L, Lpad);
    case 7: return sweep_rf_smem_g(q, L, Lpad);
    case 8: return sweep_rf_smem_h(q, L, Lpad);
    default: return 0;
    }
}

cudaError_t launch_sweep_rf(int cfg, int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                            size_t smem, const SweepSched* sched, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    switch (cfg) {
    case 1: return launch_sweep_rf_a(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 2: return launch_sweep_rf_b(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 3: return launch_sweep_rf_c(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 4: return launch_sweep_rf_d(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 5: return launch_sweep_rf_e(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 6: return launch_sweep_rf_f(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 7: return launch_sweep_rf_g(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    case 8: return launch_sweep_rf_h(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace plr

namespace plr {

// Register-resident cluster sweep (sweep_rfc.cuh): FP32 fields 9 sites per
// update thread (q <= 8), FX64 fields 5 (q <= 7); 15 update warps per CTA;
// a cluster of C = 2, 4 or 8 CTAs holds 480 C E sites.
bool rfc_fits(int precision, int C, int L, int q)
{
    if (C != 2 && C != 4 && C != 8) return false;
    if (L <= kSiteBlock || q < 2) return false;  // at least two blocks of sites
    if (precision == kPrecFP32) return q <= 8 ? L <= C * 9 * 480 : (q <= 12 && L <= C * 5 * 480);
    if (precision == kPrecFX64) return q <= 7 && L <= C * 5 * 480;
    return false;
}

int rfc_cluster_for(int precision, int L, int q)
{
    for (int C = 2; C <= 8; C *= 2)
        if (rfc_fits(precision, C, L, q)) return C;
    return 0;
}

size_t rfc_smem_bytes(int precision, int q, int C, int L)
{
    return precision == kPrecFP32   ? (q <= 8 ? sweep_rfc_smem_f(q, C, L) : sweep_rfc_smem_fq(q, C, L))
           : precision == kPrecFX64 ? sweep_rfc_smem_x(q, C, L)
                                    : 0;
}

cudaError_t launch_sweep_rfc(int precision, int C, int q, const JobDev* jobs_dev, const int2* work, int nwork,
                             int nsweeps, size_t smem, const SweepSched* sched, cudaStream_t st)
{
    if (nwork <= 0 || nsweeps <= 0) return cudaSuccess;
    if (precision == kPrecFP32)
        return q <= 8 ? launch_sweep_rfc_f(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st)
                      : launch_sweep_rfc_fq(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    if (precision == kPrecFX64) return launch_sweep_rfc_x(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
    return cudaErrorNotSupported;
}

}  // namespace plr
