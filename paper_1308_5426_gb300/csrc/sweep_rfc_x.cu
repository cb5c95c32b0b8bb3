// Register-resident cluster sweep, FX64 fields: E = 5 sites per update thread,
// 15 update warps + 1 decision warp per CTA, q <= 7, clusters of 2, 4 or 8 CTAs.
#include "sweep_rfc.cuh"

namespace plr {

cudaError_t launch_sweep_rfc_x(int q, int C, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                               size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rfc::launch_rfc_qc<long long, 5, 2, 7>(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfc_smem_x(int q, int C, int L) { return rfc::rfc_smem_q<long long, 5, 2, 7>(q, C, L); }

}  // namespace plr
