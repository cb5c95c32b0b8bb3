// Near-tie log of a job (Eq. 8, Eq. 9): decisions whose FP64 margin
// |beta dE + ln u| (Metropolis) or |D - ln u| (exchange) is below 1e-9, where
// two correct FP64 implementations may decide differently because their exp
// and log round differently.  Each is counted (JobDev::near) and the first
// kNearLogCap are logged, so that a checker can compare where the ties fell
// and adopt the decisions taken here.
#pragma once
#include <cstdint>

#include "potts_internal.h"

namespace plr {

constexpr double kNearTie = 1e-9;

// Where a decision's near tie is logged: the job's log and the slot and sweep
// (Metropolis) of the decisions being taken.
struct NearSink {
    int4* log;
    unsigned* count;
    int t;
    uint32_t n;
};

// Append {kind | decision << 1, slot or pair, sweep or exchange index,
// attempt or stage}; kind 0 = Metropolis, 1 = exchange.  Past the capacity
// the event is counted only.
__device__ __forceinline__ void near_tie_log(int4* log, unsigned* count, int kind, int t, uint32_t index,
                                             int attempt, bool accepted)
{
    if (!log) return;
    const unsigned i = atomicAdd(count, 1u);
    if (i < (unsigned)kNearLogCap) log[i] = make_int4(kind | (accepted ? 2 : 0), t, (int)index, attempt);
}

}  // namespace plr
