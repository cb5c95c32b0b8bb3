// Host side and plan kernel of the sweep placement (SweepSched in
// potts_internal.h).
#include <cmath>
#include <mutex>

#include "potts_internal.h"

namespace plr {

namespace {

constexpr int kPlanThreads = 1024;
constexpr int kBuckets = 256;  // eighth-octave buckets of the work estimate

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Expected cost of one sweep of item (job, slot): L x (accepted flips per
// sweep so far + 16), 16 standing for the per-site decision work; L^2 / 4
// flips before the slot's first sweep.  Returned as its eighth-octave bucket.
__device__ __forceinline__ int plan_bucket(const JobDev* jobs, int2 wk)
{
    const JobDev& jb = jobs[wk.x];
    const uint32_t ns = jb.nsweep[wk.y];
    const float L = (float)jb.L;
    const float fps = ns ? (float)jb.acc_flip[wk.y] / (float)ns : 0.25f * L;
    const float w = L * (fps + 16.0f);
    const int b = (int)(8.0f * log2f(w));
    return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

// One CTA: reset the claim state, bucket-sort the items by decreasing
// estimate, deal the first nsm * occ of the order to SM places in serpentine
// order (pass p over the SMs runs forwards for even p, backwards for odd p).
__global__ void __launch_bounds__(kPlanThreads) sweep_plan_kernel(const JobDev* __restrict__ jobs,
                                                                   const int2* __restrict__ work, SweepSched s)
{
    __shared__ int hist[kBuckets];
    __shared__ int start[kBuckets];
    const int tid = threadIdx.x;
    const int nplace = s.nsm * s.occ;
    for (int i = tid; i < kBuckets; i += kPlanThreads) hist[i] = 0;
    for (int i = tid; i < nplace; i += kPlanThreads) s.bins[i] = -1;
    for (int i = tid; i < s.n; i += kPlanThreads) s.claim[i] = 0;
    for (int i = tid; i < s.nsm + 2; i += kPlanThreads) s.ctr[i] = 0;
    __syncthreads();
    for (int i = tid; i < s.n; i += kPlanThreads) atomicAdd(&hist[plan_bucket(jobs, work[i])], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            start[b] = acc;
            acc += hist[b];
        }
    }
    __syncthreads();
    for (int i = tid; i < s.n; i += kPlanThreads) s.order[atomicAdd(&start[plan_bucket(jobs, work[i])], 1)] = i;
    __syncthreads();
    for (int p = tid; p < s.n; p += kPlanThreads) s.sorted[p] = work[s.order[p]];
    const int ndeal = s.n < nplace ? s.n : nplace;
    for (int p = tid; p < ndeal; p += kPlanThreads) {
        const int pass = p / s.nsm, idx = p - pass * s.nsm;
        const int sm = (pass & 1) ? s.nsm - 1 - idx : idx;
        s.bins[sm * s.occ + pass] = s.order[p];
    }
}

}  // namespace

size_t sweep_sched_bytes(int n, int nsm)
{
    return a256((size_t)n * 4) * 2 + a256((size_t)n * 8) + a256((size_t)nsm * kSchedMaxOcc * 4) +
           a256((size_t)(nsm + 2) * 4);
}

void sweep_sched_carve(char* base, int n, int nsm, SweepSched* s)
{
    size_t off = 0;
    s->order = (int*)(base + off);
    off += a256((size_t)n * 4);
    s->claim = (int*)(base + off);
    off += a256((size_t)n * 4);
    s->sorted = (int2*)(base + off);
    off += a256((size_t)n * 8);
    s->bins = (int*)(base + off);
    off += a256((size_t)nsm * kSchedMaxOcc * 4);
    s->ctr = (int*)(base + off);
    s->n = n;
    s->nsm = nsm;
    s->occ = 0;  // set per launch from the kernel's occupancy
    s->wait_ns = kSchedWaitNs;
}

int device_sm_count()
{
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

cudaError_t launch_sweep_plan(const JobDev* jobs_dev, const int2* work, const SweepSched& s, cudaStream_t st)
{
    sweep_plan_kernel<<<1, kPlanThreads, 0, st>>>(jobs_dev, work, s);
    return cudaGetLastError();
}

cudaError_t cluster_plan(const void* kernel, const cudaLaunchConfig_t& cfg, int nwork, const SweepSched* sched,
                         const JobDev* jobs_dev, const int2* work, const int2** items, cudaStream_t st)
{
    if (!sched || sched->nsm <= 0 || nwork <= 1) return cudaSuccess;
    int resident = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&resident, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (resident <= 0 || nwork <= resident) return cudaSuccess;
    SweepSched sc = *sched;
    sc.n = nwork;
    sc.occ = 0;  // no places dealt: the plan only orders the items
    if ((e = launch_sweep_plan(jobs_dev, work, sc, st)) != cudaSuccess) return e;
    *items = sc.sorted;
    return cudaSuccess;
}

}  // namespace plr
