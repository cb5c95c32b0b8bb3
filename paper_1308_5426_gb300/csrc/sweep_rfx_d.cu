// Register-resident FX64 sweep: E = 5 sites per update thread, 7 update warps
// + 1 decision warp per CTA, q <= 8 (chains up to L = 1120).
#include "sweep_rf.cuh"

namespace plr {

cudaError_t launch_sweep_rfx_d(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                                 size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rf::launch_rf_q<long long, 5, 7, 8>(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfx_smem_d(int q, int L, int Lpad) { return rf::rf_smem_q<long long, 5, 7>(q, L, Lpad); }

}  // namespace plr
