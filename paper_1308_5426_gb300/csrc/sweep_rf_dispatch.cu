// Dispatch of the register-resident FP32 sweep over its configurations
// (sweep_rf.cuh; one translation unit per configuration).
#include "potts_internal.h"

namespace plr {

namespace {
// capacity of each register configuration: largest L (E x 32 x update warps) and q
constexpr int kRfMaxL[9] = {0, 224, 448, 1120, 2400, 4320, 7680, 12480, 16800};
constexpr int kRfMaxQ[9] = {0, 16, 16, 16, 8, 8, 5, 3, 2};
}  // namespace

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
