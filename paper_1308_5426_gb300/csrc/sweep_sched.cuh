// Device side of the sweep placement (SweepSched in potts_internal.h): how a
// persistent sweep CTA finds its work items.
#pragma once
#include <cstdint>

#include "potts_internal.h"

namespace plr {

__device__ __forceinline__ unsigned sched_smid()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned long long sched_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First claim (one thread per CTA): the item dealt to this CTA's place on
// its SM, or -1.  Counts the CTA as arrived either way.
__device__ __forceinline__ int sched_claim_home(const SweepSched& s)
{
    int item = -1;
    const unsigned sm = sched_smid();
    if (sm < (unsigned)s.nsm) {
        const int r = atomicAdd(&s.ctr[sm], 1);
        if (r < s.occ) {
            const int c = s.bins[sm * s.occ + r];
            if (c >= 0 && atomicExch(&s.claim[c], 1) == 0) item = c;
        }
    }
    __threadfence();
    atomicAdd(&s.ctr[s.nsm + 1], 1);
    return item;
}

// Later claims (one thread per CTA): the next unclaimed item of the ordered
// list, or -1 when none is left.  Before its first such claim a CTA waits,
// for at most s.wait_ns, until every CTA of the grid has made its first
// claim, so that no item is taken from the SM it was dealt to; the wait only
// shapes placement (every item is claimed once whatever happens), so its
// expiry is not an error.
__device__ __forceinline__ int sched_claim_next(const SweepSched& s, bool& waited)
{
    if (!waited) {
        waited = true;
        const unsigned long long t0 = sched_clock_ns();
        const volatile int* arrived = s.ctr + s.nsm + 1;
        while (*arrived < (int)gridDim.x && sched_clock_ns() - t0 < s.wait_ns) __nanosleep(256);
    }
    for (;;) {
        const int p = atomicAdd(&s.ctr[s.nsm], 1);
        if (p >= s.n) return -1;
        const int c = s.order[p];
        if (atomicExch(&s.claim[c], 1) == 0) return c;
    }
}

}  // namespace plr
