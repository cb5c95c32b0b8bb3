// Register-resident FP32 sweep: E = 35 sites per update thread, 15 update warps
// + 1 decision warp per CTA, q <= 2 (chains up to L = 16800).
#include "sweep_rf.cuh"

namespace plr {

cudaError_t launch_sweep_rf_h(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                               size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rf::launch_rf_q<float, 35, 15, 2>(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rf_smem_h(int q, int L, int Lpad) { return rf::rf_smem_q<float, 35, 15>(q, L, Lpad); }

}  // namespace plr
