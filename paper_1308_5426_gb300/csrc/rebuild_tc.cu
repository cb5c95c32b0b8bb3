// FP32-mode field rebuild H = C . onehot(S) on the tensor cores (written next).
#include "potts_internal.h"

namespace plr {

cudaError_t launch_fields_tc(const JobDev* job_dev, int L, int q, int R, int cond, cudaStream_t st)
{
    (void)job_dev; (void)L; (void)q; (void)R; (void)cond; (void)st;
    return cudaErrorNotSupported;
}

}  // namespace plr
