// Register-resident FX64 sweep: E = 1 sites per update thread, 7 update warps
// + 1 decision warp per CTA, q <= 16 (chains up to L = 224).
#include "sweep_rf.cuh"

namespace plr {

cudaError_t launch_sweep_rfx_a(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                                 size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rf::launch_rf_q<long long, 1, 7, 16>(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfx_smem_a(int q, int L, int Lpad) { return rf::rf_smem_q<long long, 1, 7>(q, L, Lpad); }

}  // namespace plr
