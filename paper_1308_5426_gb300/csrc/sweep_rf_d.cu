// Register-resident FP32 sweep: E = 5 sites per update thread, 15 update warps
// + 1 decision warp per CTA, q <= 10 (chains up to L = 2400; 128 registers at q = 10,
// no spills).
#include "sweep_rf.cuh"

namespace plr {

cudaError_t launch_sweep_rf_d(int q, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                               size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rf::launch_rf_q<float, 5, 15, 10>(q, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rf_smem_d(int q, int L, int Lpad) { return rf::rf_smem_q<float, 5, 15>(q, L, Lpad); }

}  // namespace plr
