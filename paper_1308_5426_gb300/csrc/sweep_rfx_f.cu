// Register-resident FX64 sweep: E = 9 sites per update thread, 15 update warps
// + 1 decision warp per CTA, q <= 3 (chains up to L = 4320).
#include "sweep_rf.cuh"

namespace plr {

cudaError_t launch_sweep_rfx_f(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                                 size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rf::launch_rf_q<long long, 9, 15, 3>(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfx_smem_f(int q, int L, int Lpad) { return rf::rf_smem_q<long long, 9, 15>(q, L, Lpad); }

}  // namespace plr
