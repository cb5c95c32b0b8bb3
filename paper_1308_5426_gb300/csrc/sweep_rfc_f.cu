// Register-resident cluster sweep, FP32 fields: E = 9 sites per update thread,
// 15 update warps + 1 decision warp per CTA, q <= 8, clusters of 2, 4 or 8 CTAs.
#include "sweep_rfc.cuh"

namespace plr {

cudaError_t launch_sweep_rfc_f(int q, int C, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                               size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rfc::launch_rfc_qc<float, 9, 2, 8>(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfc_smem_f(int q, int C, int L) { return rfc::rfc_smem_q<float, 9, 2, 8>(q, C, L); }

}  // namespace plr
