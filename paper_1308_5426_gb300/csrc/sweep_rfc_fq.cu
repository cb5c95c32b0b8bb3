// Register-resident cluster sweep, FP32 fields of q = 9..12 states: E = 5 sites
// per update thread (60 field registers at q = 12, no spills; 9 sites would not
// fit), 15 update warps + 1 decision warp per CTA, clusters of 2, 4 or 8 CTAs.
#include "sweep_rfc.cuh"

namespace plr {

cudaError_t launch_sweep_rfc_fq(int q, int C, const JobDev* jobs_dev, const int2* work, int nwork, int nsweeps,
                                size_t smem, const SweepSched* sched, cudaStream_t st)
{
    return rfc::launch_rfc_qc<float, 5, 9, 12>(q, C, jobs_dev, work, nwork, nsweeps, smem, sched, st);
}

size_t sweep_rfc_smem_fq(int q, int C, int L) { return rfc::rfc_smem_q<float, 5, 9, 12>(q, C, L); }

}  // namespace plr
