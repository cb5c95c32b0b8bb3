// Host side of the potts_lr C ABI: argument checks, the device arena of a job,
// launch sequencing, checkpoints and graph-captured batching.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <unordered_set>
#include <vector>

#include "../../include/potts_lr.h"
#include "measure_body.cuh"
#include "potts_internal.h"

using namespace plr;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(POTTS_LR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define PLR_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

constexpr size_t kSmemBudget = 220 * 1024;  // dynamic shared memory a sweep CTA may take
constexpr size_t kClusterFieldBytes = 88 * 1024;   // FP32 fields above this go to a cluster (see create)
constexpr size_t kClusterFieldBytes8 = 64 * 1024;  // FP64 and FX64 fields above this (see create)
constexpr uint32_t kStateMagic = 0x31524c50u; // "PLR1"
constexpr uint32_t kStateVersion = 4;          // header + the job's checkpoint block

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Checkpoint header: what a restored state must share with the handle for
// the run to continue as the uninterrupted run would (72 bytes).
struct StateHeader {
    uint32_t magic, version;
    int32_t L, q, R, precision, c, Lpad;
    uint64_t seed;
    uint32_t nsweep, nexch;
    uint64_t sigma_bits;  // bit pattern of sigma (the couplings, Eq. 4-6)
    uint64_t temps_hash;  // FNV-1a of the bit patterns of the R inverse temperatures
    int32_t fx_bits;      // FX64 mode: F of the field grid 2^-F (0 otherwise)
    int32_t reserved;
};
static_assert(sizeof(StateHeader) == 72, "checkpoint header layout");

// FNV-1a (64-bit) over the bytes of n doubles
uint64_t fnv1a(const double* v, size_t n)
{
    uint64_t hsh = 0xcbf29ce484222325ull;
    const unsigned char* p = (const unsigned char*)v;
    for (size_t i = 0; i < n * sizeof(double); ++i) {
        hsh ^= p[i];
        hsh *= 0x100000001b3ull;
    }
    return hsh;
}

}  // namespace

struct potts_lr {
    int L, q, R, W, Lpad, precision, K, c;
    double sigma, jtot;
    uint64_t seed;
    int fx_bits;                  // FX64 mode: F of the field grid (0 otherwise)
    uint64_t temps_hash;          // fnv1a of the inverse temperatures (checkpoint check)
    cudaStream_t stream;
    bool own_stream;
    void* arena;
    size_t wsize;                 // field word size
    JobDev hj;                    // host copy of the device descriptor
    JobDev* dj;                   // device descriptor
    int2* dwork;                  // {0, t}, t = 0..R-1
    uint32_t nsweep, nexch;       // host mirrors of the counters
    size_t sweep_smem, measure_smem, direct_smem;
    double* pinned;               // 2R doubles of pinned host memory for measure
    int4* dtiles;                 // FP32: tensor-core rebuild tiles of this job (job index 0)
    int ntiles;
    int tc_tn;                    // their width (64 or 128 columns)
    int onehot_blocks;            // FP32: grid width of the rebuild's one-hot kernel
    SweepSched sched;             // placement of the R slots on the SMs
    bool direct;                  // sweeps by the direct O(L) sum: fields are rebuilt on demand
    bool cl_auto;                 // the cluster sweep was chosen automatically (not asked for)
    int cl_min;                   // the smallest cluster whose shares fit (j.cl may be larger)
    size_t state_off, state_len;  // the checkpointed arrays: one block of the arena
};

struct potts_lr_batch {
    std::vector<potts_lr_t*> jobs;
    cudaStream_t stream;
    bool own_stream;
    JobDev* djobs;
    void* arena;
    struct Group {
        int key;  // sweep kernel variant
        int2* dwork;
        int nwork;
        size_t smem;
        SweepSched sched;
        cudaStream_t stream;  // its own stream when the batch has several groups
        cudaEvent_t done;     // recorded on it after the group's sweep
    };
    std::vector<Group> groups;
    cudaEvent_t fork;             // the batch stream's point where the groups' sweeps start
    std::vector<int> fp32_jobs;  // jobs that need the conditional rebuild
    int4* dtc_tiles;             // their rebuild tiles (job index into djobs)
    int ntc_tiles;
    int tc_tn;                   // tile width (64 or 128 columns)
    int onehot_blocks;           // grid width of their one-hot kernel (the largest job's)
    int2* dfp_work;              // (job, slot) of their slots, for the energy re-anchor
    int nfp_work;
    size_t fp_meas_smem;
    int fp_meas_parts;           // the largest measure split among them
    int* dfp_idx;                // their job indices, for the schedule policy
    int2* dmeas;                 // (job, slot) of every slot, job order
    int nmeas;
    size_t meas_smem;
    int meas_parts;              // the largest measure split among the jobs
    double* meas_buf;            // device staging: 2 * nmeas doubles
    std::vector<int> meas_off;   // first row of each job
    cudaGraphExec_t exec;
    int exec_steps;
    cudaEvent_t ev;
};

namespace {

uint16_t to_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
    return (uint16_t)(u >> 16);
}

double from_bf16(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

int check_opts(const potts_lr_opts* o)
{
    if (o->precision != POTTS_LR_FP64 && o->precision != POTTS_LR_FP32 && o->precision != POTTS_LR_FX64)
        return fail(POTTS_LR_EINVAL, "precision must be POTTS_LR_FP64, POTTS_LR_FP32 or POTTS_LR_FX64");
    if (o->pair_factor != 1 && o->pair_factor != 2) return fail(POTTS_LR_EINVAL, "pair_factor must be 1 or 2");
    if (o->recompute_every < 0) return fail(POTTS_LR_EINVAL, "recompute_every must be >= 0");
    if (o->sweep_variant < 0 || (o->sweep_variant > 6 && (o->sweep_variant < 17 || o->sweep_variant > 24)))
        return fail(POTTS_LR_EINVAL, "sweep_variant must be 0..6 or 17..24");
    if (o->sweep_variant == 6 && o->precision == POTTS_LR_FP64)
        return fail(POTTS_LR_EINVAL, "the register-resident cluster sweep (sweep_variant 6) holds FP32 or FX64 fields");
    if (o->sweep_variant == 4 && o->precision != POTTS_LR_FP64)
        return fail(POTTS_LR_EINVAL, "the direct sweep (sweep_variant 4) runs in FP64 mode only");
    if (o->site_order != 0 && o->site_order != 1) return fail(POTTS_LR_EINVAL, "site_order must be 0 or 1");
    if (o->site_order == 1 && (o->precision != POTTS_LR_FP64 || (o->sweep_variant != 0 && o->sweep_variant != 4)))
        return fail(POTTS_LR_EINVAL, "random site order runs on the direct sweep: FP64, sweep_variant 0 or 4");
    return POTTS_LR_OK;
}

// Field rebuild of one job: FP32 mode on the tensor cores, FP64 mode by
// direct sums, FX64 mode by direct integer sums (which reproduce the swept
// fields bit for bit); then the energies are re-anchored from the spins.  job_dev is the
// job's descriptor in device memory (its own, or its entry in a batch table).
cudaError_t rebuild_launch(const potts_lr_t* h, const JobDev* job_dev, int cond, cudaStream_t st)
{
    cudaError_t e;
    if (h->precision == POTTS_LR_FP32)
        e = launch_fields_tc(job_dev, nullptr, 1, h->onehot_blocks, h->dtiles, h->ntiles, cond, h->tc_tn, st);
    else
        e = launch_fields_direct(job_dev, h->L, h->R, 0, cond, h->direct_smem, st);
    if (e != cudaSuccess) return e;
    e = launch_measure(job_dev, h->dwork, h->R, 1, cond, h->measure_smem, h->hj.meas_parts, st);
    if (e != cudaSuccess || h->precision != POTTS_LR_FP32) return e;
    return launch_rebuild_policy(job_dev, nullptr, 1, cond, st);
}

// the sweep kernel variant of a job: register-resident (per configuration and
// q) or memory-resident (per precision and shared-memory residency)
// keys: memory kernel 0..11 (precision, fields and table residency), direct
// sweep 99, FP32 register kernel 100 + 32 configuration + q (132..372), FX64
// register kernel kRfxKey + 32 configuration + q (432..608), cluster kernel
// kClusterKey + 16 precision + cluster size
constexpr int kDirectKey = 99;
constexpr int kRfxKey = 400;
constexpr int kClusterKey = 1000;
constexpr int kRfcKey = 3000;  // register-resident cluster: + 1024 precision + 64 cluster size + q

int variant_key(const potts_lr_t* h)
{
    if (h->direct) return kDirectKey;
    if (h->hj.rc) return kRfcKey + 1024 * h->precision + 64 * h->hj.rc + h->q;
    if (h->hj.cl) return kClusterKey + 16 * h->precision + h->hj.cl;
    if (h->hj.rf) return (h->precision == POTTS_LR_FX64 ? kRfxKey : 100) + h->hj.rf * 32 + h->q;
    return h->precision * 4 + h->hj.h_smem * 2 + h->hj.j_smem;
}

cudaError_t launch_variant(int key, const JobDev* jobs, const int2* work, int nwork, int nsweeps, size_t smem,
                           const SweepSched* sched, cudaStream_t st)
{
    if (key >= kRfcKey) {
        const int r = key - kRfcKey;
        return launch_sweep_rfc(r / 1024, (r % 1024) / 64, r % 64, jobs, work, nwork, nsweeps, smem, sched, st);
    }
    if (key > kClusterKey)
        return launch_sweep_cluster((key - kClusterKey) % 16, (key - kClusterKey) / 16, jobs, work, nwork, nsweeps,
                                    smem, sched, st);
    if (key >= kRfxKey)
        return launch_sweep_rfx((key - kRfxKey) / 32, (key - kRfxKey) % 32, jobs, work, nwork, nsweeps, smem, sched,
                                st);
    if (key >= 100)
        return launch_sweep_rf((key - 100) / 32, (key - 100) % 32, jobs, work, nwork, nsweeps, smem, sched, st);
    if (key == kDirectKey) return launch_sweep_direct(jobs, work, nwork, nsweeps, smem, st);
    return launch_sweep(jobs, work, nwork, nsweeps, key >> 2, (key >> 1) & 1, key & 1, smem, sched, st);
}

// the direct sweep keeps no fields: rebuild them (FP64, exact) before they are read
int fresh_fields(potts_lr_t* h)
{
    if (!h->direct) return POTTS_LR_OK;
    cudaError_t e = launch_fields_direct(h->dj, h->L, h->R, 0, 0, h->direct_smem, h->stream);
    return e == cudaSuccess ? POTTS_LR_OK : cuda_fail(e, "field rebuild");
}

int rebuild(potts_lr_t* h)
{
    cudaError_t e = rebuild_launch(h, h->dj, 0, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "field rebuild");
    return POTTS_LR_OK;
}

// after a stream synchronisation: report (and clear) an expired device wait
int check_status(potts_lr_t* h)
{
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, h->hj.status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st) {
        cudaMemset(h->hj.status, 0, 4);
        return fail(POTTS_LR_ETIMEOUT, "a bounded device wait expired (tensor-core rebuild); fields are invalid");
    }
    return POTTS_LR_OK;
}

}  // namespace

extern "C" {

const char* potts_lr_last_error(void) { return g_err; }

int potts_lr_default_opts(potts_lr_opts* opts)
{
    if (!opts) return fail(POTTS_LR_EINVAL, "opts is NULL");
    opts->precision = POTTS_LR_FP64;
    opts->recompute_every = 100;
    opts->pair_factor = 2;
    opts->cuda_stream = nullptr;
    opts->sweep_variant = 0;
    opts->site_order = 0;
    return POTTS_LR_OK;
}

int potts_lr_jstar(int L, double sigma, double* out)
{
    if (L < 2 || L > kMaxL) return fail(POTTS_LR_EINVAL, "L must be in [2, %d]", kMaxL);
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(POTTS_LR_EINVAL, "sigma must be positive and finite");
    if (!out) return fail(POTTS_LR_EINVAL, "out is NULL");
    jstar_table(L, sigma, out);
    return POTTS_LR_OK;
}

void potts_lr_destroy(potts_lr_t* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->arena) cudaFree(h->arena);
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int potts_lr_create(int L, int q, double sigma, const double* temps, int R, uint64_t seed,
                    const potts_lr_opts* opts, potts_lr_t** out)
{
    if (!out) return fail(POTTS_LR_EINVAL, "out is NULL");
    *out = nullptr;
    potts_lr_opts o;
    potts_lr_default_opts(&o);
    if (opts) o = *opts;
    int rc = check_opts(&o);
    if (rc) return rc;
    if (L < 2 || L > kMaxL) return fail(POTTS_LR_EINVAL, "L must be in [2, %d]", kMaxL);
    if (q < 2 || q > kMaxQ) return fail(POTTS_LR_EINVAL, "q must be in [2, %d]", kMaxQ);
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(POTTS_LR_EINVAL, "sigma must be positive and finite");
    if (R < 1 || R > 4096) return fail(POTTS_LR_EINVAL, "R must be in [1, 4096]");
    if (!temps) return fail(POTTS_LR_EINVAL, "temps is NULL");
    for (int t = 0; t < R; ++t)
        if (!(temps[t] > 0.0) || !std::isfinite(temps[t]))
            return fail(POTTS_LR_EINVAL, "temperature %d is not positive and finite", t);

    potts_lr_t* h = new (std::nothrow) potts_lr();
    if (!h) return fail(POTTS_LR_ENOMEM, "host allocation failed");
    h->L = L;
    h->q = q;
    h->R = R;
    h->W = (L + 7) / 8;
    h->Lpad = (L + 31) & ~31;
    h->precision = o.precision;
    h->K = o.precision == POTTS_LR_FP32 ? o.recompute_every : 0;
    h->c = o.pair_factor;
    h->sigma = sigma;
    h->seed = seed;
    h->wsize = o.precision == POTTS_LR_FP32 ? 4 : 8;
    if (o.cuda_stream) {
        h->stream = (cudaStream_t)o.cuda_stream;
        h->own_stream = false;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        h->own_stream = true;
    }

    // host tables
    std::vector<double> J(L);
    jstar_table(L, sigma, J.data());
    double jt = 0.0;
    for (int r = 1; r < L; ++r) jt += J[r];
    h->jtot = jt;
    // FX64 field grid 2^-F: F = 61 - e with Jtot < 2^e, so every field, being
    // at most Jtot (+ L/2 units of rounding), stays below 2^62 units
    const bool fx = h->precision == POTTS_LR_FX64;
    int fx_bits = 0;
    if (fx) {
        int e2 = 0;
        std::frexp(jt, &e2);  // jt = m 2^e2, m in [0.5, 1)
        fx_bits = 61 - std::max(e2, 0);
        if (fx_bits < 24) {
            potts_lr_destroy(h);
            return fail(POTTS_LR_EINVAL, "sigma too small for FX64 fields (sum of couplings %g)", jt);
        }
    }
    std::vector<long long> Jfxd(fx ? 2 * (size_t)h->Lpad : 0, 0);
    for (int m = 0; fx && m < 2 * L; ++m) Jfxd[m] = std::llrint(std::ldexp(J[m % L], fx_bits));
    std::vector<double> J64d(2 * (size_t)h->Lpad, 0.0);
    std::vector<float> J32d(2 * (size_t)h->Lpad, 0.0f);
    for (int m = 0; m < 2 * L; ++m) {
        J64d[m] = J[m % L];
        J32d[m] = (float)J[m % L];
    }
    // BF16 parts hi + mid + lo of J* for the tensor-core rebuild (FP32 mode)
    std::vector<uint16_t> split(3 * (size_t)h->Lpad, 0);
    for (int r = 0; r < L; ++r) {
        const uint16_t hi = to_bf16((float)J[r]);
        const double r1 = J[r] - from_bf16(hi);
        const uint16_t mid = to_bf16((float)r1);
        const double r2 = r1 - from_bf16(mid);
        split[r] = hi;
        split[h->Lpad + r] = mid;
        split[2 * (size_t)h->Lpad + r] = to_bf16((float)r2);
    }
    // the same parts as the Hankel core matrices the rebuild copies (its A operand)
    std::vector<uint16_t> hank;
    if (h->precision == POTTS_LR_FP32) tc_hank_table(J, split.data(), h->Lpad, hank);
    std::vector<double> beta(R);
    for (int t = 0; t < R; ++t) beta[t] = 1.0 / temps[t];
    h->fx_bits = fx_bits;
    h->temps_hash = fnv1a(beta.data(), (size_t)R);
    // first FP32 rebuild interval: short for long chains with few states (the
    // drift grows with the field updates per element, ~L/q per sweep); the
    // device doubles it while the measured drift stays small
    int sched0[4] = {0, 0, 0, 0};
    if (h->K > 0) {
        const int k0 = (int)std::max(1.0, std::min((double)h->K, 2500.0 * q / (double)L));
        sched0[0] = k0;
        sched0[1] = k0;
    }
    std::vector<int> map(R);
    std::vector<int2> work(R);
    for (int t = 0; t < R; ++t) {
        map[t] = t;
        work[t] = make_int2(0, t);
    }

    // arena layout
    const size_t Lp = (size_t)h->Lpad;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off += align256(bytes);
        return o2;
    };
    const size_t o_J64 = take(2 * Lp * 8), o_J32 = take(2 * Lp * 4), o_Jfx = take(fx ? 2 * Lp * 8 : 0);
    // the checkpointed arrays, contiguous in checkpoint order (a checkpoint is
    // a host header and one copy of this block)
    size_t sb = 0;
    auto in_block = [&](size_t bytes) {
        size_t o2 = sb;
        sb += align256(bytes);
        return o2;
    };
    const size_t r_map = in_block((size_t)R * 4), r_E = in_block((size_t)R * 8);
    const size_t r_spins = in_block((size_t)R * h->W * 4), r_fields = in_block((size_t)R * q * Lp * h->wsize);
    const size_t r_nsw = in_block((size_t)R * 4), r_accf = in_block((size_t)R * 8), r_accs = in_block((size_t)R * 8);
    const size_t r_near = in_block(16), r_sched = in_block(16), r_drift = in_block(16), r_nex = in_block(4);
    const size_t o_state = take(sb);
    h->state_off = o_state;
    h->state_len = sb;
    const size_t o_map = o_state + r_map, o_E = o_state + r_E, o_spins = o_state + r_spins;
    const size_t o_fields = o_state + r_fields, o_nsw = o_state + r_nsw, o_accf = o_state + r_accf;
    const size_t o_accs = o_state + r_accs, o_near = o_state + r_near, o_sched = o_state + r_sched;
    const size_t o_drift = o_state + r_drift, o_nex = o_state + r_nex;
    const size_t o_beta = take((size_t)R * 8);
    const size_t o_mE = take((size_t)R * 8), o_mM = take((size_t)R * 8), o_err = take(8);
    const size_t o_mpart = take((size_t)R * kMeasMaxParts * 8), o_mtick = take((size_t)R * 4);
    const size_t o_job = take(sizeof(JobDev)), o_work = take((size_t)R * sizeof(int2));
    const bool tc = h->precision == POTTS_LR_FP32;  // tensor-core rebuild operands
    const size_t o_hank = take(tc ? tc_hank_bytes(L) : 0), o_xoh = take(tc ? tc_onehot_bytes(L, q, R) : 0);
    const size_t o_status = take(4);
    const size_t o_nlog = take((size_t)kNearLogCap * sizeof(int4)), o_nlogn = take(4);
    std::vector<int4> tiles;
    h->tc_tn = tc_tile_width(tc_tile_count(L, q, R, 64), tc_tile_count(L, q, R, 128), device_sm_count());
    if (h->precision == POTTS_LR_FP32) {
        tc_tiles(0, L, q, R, h->tc_tn, tiles);
        tc_order_tiles(tiles);
    }
    const size_t o_tiles = take(tiles.size() * sizeof(int4) + 16);
    const int nsm = device_sm_count();
    const size_t o_plan = take(sweep_sched_bytes(R, nsm));
    cudaError_t e = cudaMalloc(&h->arena, off);
    if (e != cudaSuccess) {
        potts_lr_destroy(h);
        return fail(e == cudaErrorMemoryAllocation ? POTTS_LR_ENOMEM : POTTS_LR_ECUDA, "cudaMalloc(%zu): %s", off,
                    cudaGetErrorString(e));
    }
    e = cudaMallocHost((void**)&h->pinned, 2 * (size_t)R * sizeof(double));
    if (e != cudaSuccess) {
        potts_lr_destroy(h);
        return fail(POTTS_LR_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    char* base = (char*)h->arena;
    JobDev& j = h->hj;
    std::memset(&j, 0, sizeof(j));
    j.L = L;
    j.q = q;
    j.Lpad = h->Lpad;
    j.W = h->W;
    j.R = R;
    j.c = h->c;
    j.precision = h->precision;
    j.recompute_every = h->K;
    j.key0 = (uint32_t)(seed & 0xffffffffu);
    j.key1 = (uint32_t)(seed >> 32);
    j.jtot = jt;
    j.J64d = (const double*)(base + o_J64);
    j.J32d = (const float*)(base + o_J32);
    j.Jfxd = fx ? (const long long*)(base + o_Jfx) : nullptr;
    j.fx_scale = std::ldexp(1.0, -fx_bits);
    j.spins = (uint32_t*)(base + o_spins);
    j.fields = (void*)(base + o_fields);
    j.E = (double*)(base + o_E);
    j.map = (int*)(base + o_map);
    j.beta = (const double*)(base + o_beta);
    j.nsweep = (uint32_t*)(base + o_nsw);
    j.nexch = (uint32_t*)(base + o_nex);
    j.acc_flip = (unsigned long long*)(base + o_accf);
    j.acc_swap = (unsigned long long*)(base + o_accs);
    j.near = (unsigned long long*)(base + o_near);
    j.near_log = (int4*)(base + o_nlog);
    j.near_log_n = (unsigned*)(base + o_nlogn);
    j.meas_E = (double*)(base + o_mE);
    j.meas_M = (double*)(base + o_mM);
    j.meas_part = (double*)(base + o_mpart);
    j.meas_ticket = (int*)(base + o_mtick);
    j.meas_parts = measure_parts(L);
    j.err_bits = (unsigned long long*)(base + o_err);
    j.Jhank = tc ? (const uint16_t*)(base + o_hank) : nullptr;
    j.Xoh = tc ? (uint16_t*)(base + o_xoh) : nullptr;
    j.hank_cores = (int)tc_hank_cores(L);
    j.NG = tc_ng(q, R);
    h->onehot_blocks = tc_onehot_blocks(L, q, R);
    j.status = (int*)(base + o_status);
    j.tc_wait_ns = kTcWaitNs;
    j.tc_parts = 0;  // automatic (rebuild_parts)
    j.sched = (int*)(base + o_sched);
    h->dtiles = (int4*)(base + o_tiles);
    h->ntiles = (int)tiles.size();
    sweep_sched_carve(base + o_plan, R, nsm, &h->sched);
    j.drift_bits = (unsigned long long*)(base + o_drift);
    // residency of the sweep kernel's working set: fields and table in shared
    // memory when they fit, else fields first, else the table, else neither
    {
        const int opts_hs[4] = {1, 1, 0, 0}, opts_js[4] = {1, 0, 1, 0};
        for (int v = o.sweep_variant == 3 ? 2 : 0; v < 4; ++v) {  // variant 3: fields in global memory
            if (sweep_smem_bytes_for(h->precision, L, h->Lpad, q, opts_hs[v], opts_js[v]) <= kSmemBudget) {
                j.h_smem = opts_hs[v];
                j.j_smem = opts_js[v];
                break;
            }
        }
    }
    if (o.sweep_variant == 0 || o.sweep_variant == 2)
        j.rf = h->precision == POTTS_LR_FP32 ? rf_config(L, q) : h->precision == POTTS_LR_FX64 ? rfx_config(L, q) : 0;
    if (o.sweep_variant >= 17) {  // one register configuration, chosen by the caller (a tuner)
        const int cfg = o.sweep_variant - 16;
        const bool ok = h->precision == POTTS_LR_FP32   ? rf_fits(cfg, L, q)
                        : h->precision == POTTS_LR_FX64 ? rfx_fits(cfg, L, q)
                                                        : false;
        if (!ok) {
            potts_lr_destroy(h);
            return fail(POTTS_LR_EINVAL, "register configuration %d does not hold L = %d, q = %d in this precision",
                        cfg, L, q);
        }
        j.rf = cfg;
    }
    if (o.sweep_variant == 2 && !j.rf) {
        potts_lr_destroy(h);
        return fail(POTTS_LR_EINVAL, "register-resident sweep needs FP32 and L <= 1120, or L <= 2400 with q <= 10, "
                                     "L <= 4320 with q <= 8 (7680 with q <= 5, 12480 with q <= 3, 16800 with q = 2), "
                                     "or FX64 and L <= 448, "
                                     "or L <= 1120 with q <= 8 (2400 with q <= 5, 4320 with q <= 3)");
    }
    h->dj = (JobDev*)(base + o_job);
    h->dwork = (int2*)(base + o_work);
    h->sweep_smem = !j.rf                              ? sweep_smem_bytes(j)
                    : h->precision == POTTS_LR_FX64 ? rfx_smem_bytes(j.rf, q, L, h->Lpad)
                                                    : rf_smem_bytes(j.rf, q, L, h->Lpad);
    // Fields that fit no registers: a cluster of CTAs shares them when they
    // fit no single CTA's shared memory, or when they are large (FP32: fill
    // most of one CTA, which then sweeps the slot alone with few update warps;
    // FP64, FX64: more than 64 KB, so that a hot slot's 8-byte updates keep
    // one SM busy) while the job's clusters fit on the GPU at once; or when
    // asked for (variant 5).  Measured, one job of 64 slots: FP32 2-2.6x
    // faster; FP64 at equilibrium L = 2048, q = 5 2.13 -> 0.85 ms per sweep,
    // L = 4096, q = 5 7.96 -> 2.36, L = 8192, q = 3 29.6 -> 5.37; on a GPU
    // already filled by many jobs' slots about even (see the batch rule).
    // First, FP32 and FX64 chains that no single CTA's registers hold go to the
    // registers of a cluster where one holds them (measured on GB300 2-3x
    // faster than the shared-memory cluster: L = 16384, q = 5, R = 64, FP32
    // 4.07 against 11.68 ms per sweep; L = 8192, q = 5: 1.41 against 3.01).
    if (!j.rf && o.sweep_variant == 0 && h->precision != POTTS_LR_FP64) {
        const int C = rfc_cluster_for(h->precision, L, q);
        if (C && rfc_smem_bytes(h->precision, q, C, L) <= kSmemBudget) {
            j.rc = C;
            h->sweep_smem = rfc_smem_bytes(h->precision, q, C, L);
        }
    }
    if (!j.rf && !j.rc && (o.sweep_variant == 0 || o.sweep_variant == 5)) {
        const int C = cluster_size_for(L, q, kSmemBudget, h->precision);
        const bool fp32 = h->precision == POTTS_LR_FP32;
        const bool big = fp32 ? (size_t)q * h->Lpad * 4 > kClusterFieldBytes
                              : (size_t)q * h->Lpad * 8 > kClusterFieldBytes8;
        const bool fits_gpu = (long long)R * C <= (long long)std::max(1, device_sm_count());
        if (o.sweep_variant == 5 || (C && (!j.h_smem || (big && fits_gpu)))) {
            if (!C) {
                potts_lr_destroy(h);
                return fail(POTTS_LR_EINVAL, "the cluster sweep holds at most 8 x %zu bytes of fields and spins",
                            kSmemBudget);
            }
            j.cl = C;
            h->cl_min = C;
            h->cl_auto = o.sweep_variant == 0;
            // FP64 and FX64 chosen automatically: a larger cluster while the
            // job's CTAs still fit four per SM and each CTA keeps at least
            // C * 128 sites.  A hot slot's rank-1 updates (8-byte adds) then
            // spread over more SMs; they set the sweep's length on a ladder
            // with slots above the transition, against a per-block cost of the
            // cluster (flip lists to C CTAs, one cluster barrier) that does
            // not shrink with C.  Measured at equilibrium, FP64 (ms per sweep,
            // C = 2 / 4 / 8): L = 1024, q = 8, R = 64 0.437 / 0.417 / 0.790;
            // L = 2048, q = 5 1.28 / 0.851 / 1.32; L = 4096, q = 5 4.20 /
            // 2.36 / 2.65; L = 8192, q = 3 14.7 / 7.99 / 5.37; L = 4096, q = 8,
            // R = 128 4.78 / 2.69 / 3.65 (FX64 1.82 / 1.49 / 3.32); L = 16384,
            // q = 5, R = 64 - / 34.9 / 29.5.
            if (h->cl_auto && !fp32)
                while (j.cl < 8 && (long long)R * 2 * j.cl <= 4LL * std::max(1, device_sm_count()) &&
                       4 * j.cl * j.cl * 128 <= L)
                    j.cl *= 2;
            h->sweep_smem = cluster_sweep_smem(L, q, j.cl, h->precision);
        }
    }
    if (o.sweep_variant == 6) {  // the slot's fields in the registers of a cluster of CTAs
        const int C = rfc_cluster_for(h->precision, L, q);
        if (!C || rfc_smem_bytes(h->precision, q, C, L) > kSmemBudget) {
            potts_lr_destroy(h);
            return fail(POTTS_LR_EINVAL, "the register-resident cluster sweep holds FP32 chains of q <= 8 and L <= "
                                         "34560 or q <= 12 and L <= 19200, FX64 chains of q <= 7 and L <= 19200 (and "
                                         "more than 32 sites)");
        }
        j.rc = C;
        j.rf = 0;
        j.cl = 0;
        h->sweep_smem = rfc_smem_bytes(h->precision, q, C, L);
    }
    j.random_sites = o.site_order;
    if (o.sweep_variant == 4 || o.site_order == 1) {
        h->direct = true;
        h->cl_auto = false;  // the direct sweep keeps its kernel in every batch
        h->sweep_smem = direct_sweep_smem_bytes(L, h->Lpad);
        if (h->sweep_smem > kSmemBudget) {
            potts_lr_destroy(h);
            return fail(POTTS_LR_EINVAL, "the direct sweep keeps the spins of its slot in shared memory: L too large");
        }
    }
    h->measure_smem = measure_smem_bytes(L, q);
    h->direct_smem = direct_smem_bytes(L, q);

    cudaStream_t st = h->stream;
    int rc2 = POTTS_LR_OK;
    do {
        if ((e = cudaMemsetAsync(h->arena, 0, off, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync((void*)j.J64d, J64d.data(), 2 * Lp * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync((void*)j.J32d, J32d.data(), 2 * Lp * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if (fx && (e = cudaMemcpyAsync((void*)j.Jfxd, Jfxd.data(), 2 * Lp * 8, cudaMemcpyHostToDevice, st)) !=
                      cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync((void*)j.beta, beta.data(), (size_t)R * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(j.map, map.data(), (size_t)R * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(h->dj, &j, sizeof(JobDev), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(h->dwork, work.data(), (size_t)R * sizeof(int2), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if (tc && (e = cudaMemcpyAsync((void*)j.Jhank, hank.data(), hank.size() * 2, cudaMemcpyHostToDevice, st)) !=
                      cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(j.sched, sched0, 16, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
        if (!tiles.empty() &&
            (e = cudaMemcpyAsync(h->dtiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st)) !=
                cudaSuccess)
            break;
        if ((e = launch_init_spins(h->dj, 0, L, h->W, R, st)) != cudaSuccess) break;
        if ((e = launch_fields_direct(h->dj, L, R, 0, 0, h->direct_smem, st)) != cudaSuccess) break;
        if ((e = launch_measure(h->dj, h->dwork, R, 1, 0, h->measure_smem, j.meas_parts, st)) != cudaSuccess) break;
        e = cudaStreamSynchronize(st);
    } while (0);
    if (e != cudaSuccess) rc2 = cuda_fail(e, "potts_lr_create");
    if (rc2) {
        potts_lr_destroy(h);
        return rc2;
    }
    h->nsweep = 0;
    h->nexch = 0;
    *out = h;
    return POTTS_LR_OK;
}

int potts_lr_sweep(potts_lr_t* h, int n)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    if (n < 0) return fail(POTTS_LR_EINVAL, "n must be >= 0");
    if (n == 0) return POTTS_LR_OK;
    const int key = variant_key(h);
    if (h->K <= 0) {
        cudaError_t e = launch_variant(key, h->dj, h->dwork, h->R, n, h->sweep_smem, &h->sched, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel");
        h->nsweep += (uint32_t)n;
        return POTTS_LR_OK;
    }
    // FP32 mode with automatic rebuilds: the schedule lives on the device, so
    // every sweep is followed by the conditional rebuild
    for (int s = 0; s < n; ++s) {
        cudaError_t e = launch_variant(key, h->dj, h->dwork, h->R, 1, h->sweep_smem, &h->sched, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel");
        h->nsweep += 1u;
        e = rebuild_launch(h, h->dj, 1, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "field rebuild");
    }
    return POTTS_LR_OK;
}

int potts_lr_exchange(potts_lr_t* h)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    cudaError_t e = launch_exchange(h->dj, 1, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "exchange kernel");
    h->nexch++;
    return POTTS_LR_OK;
}

int potts_lr_measure_device(potts_lr_t* h, double* E, double* M)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    cudaError_t e = launch_measure(h->dj, h->dwork, h->R, 0, 0, h->measure_smem, h->hj.meas_parts, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "measure kernel");
    const size_t b = (size_t)h->R * sizeof(double);
    if (E) PLR_CUDA(cudaMemcpyAsync(E, h->hj.meas_E, b, cudaMemcpyDeviceToDevice, h->stream));
    if (M) PLR_CUDA(cudaMemcpyAsync(M, h->hj.meas_M, b, cudaMemcpyDeviceToDevice, h->stream));
    return POTTS_LR_OK;
}

int potts_lr_measure(potts_lr_t* h, double* E, double* M)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    cudaError_t e = launch_measure(h->dj, h->dwork, h->R, 0, 0, h->measure_smem, h->hj.meas_parts, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "measure kernel");
    const size_t b = (size_t)h->R * sizeof(double);
    PLR_CUDA(cudaMemcpyAsync(h->pinned, h->hj.meas_E, b, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaMemcpyAsync(h->pinned + h->R, h->hj.meas_M, b, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    if (E) std::memcpy(E, h->pinned, b);
    if (M) std::memcpy(M, h->pinned + h->R, b);
    return check_status(h);
}

int potts_lr_fields_recompute(potts_lr_t* h)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    return rebuild(h);
}

int potts_lr_fields_error(potts_lr_t* h, double* max_err)
{
    if (!h || !max_err) return fail(POTTS_LR_EINVAL, "NULL argument");
    if (int rc = fresh_fields(h)) return rc;
    PLR_CUDA(cudaMemsetAsync(h->hj.err_bits, 0, 8, h->stream));
    cudaError_t e = launch_fields_direct(h->dj, h->L, h->R, 1, 0, h->direct_smem, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fields check");
    unsigned long long bits = 0;
    PLR_CUDA(cudaMemcpyAsync(&bits, h->hj.err_bits, 8, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    std::memcpy(max_err, &bits, 8);
    return check_status(h);
}

int potts_lr_sync(potts_lr_t* h)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    return check_status(h);
}

int potts_lr_counters(potts_lr_t* h, uint32_t* nsweep, uint32_t* nexch)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    if (nsweep) *nsweep = h->nsweep;
    if (nexch) *nexch = h->nexch;
    return POTTS_LR_OK;
}

static size_t state_bytes(const potts_lr_t* h) { return sizeof(StateHeader) + h->state_len; }

// Checkpoint of one job: a StateHeader, then the job's checkpoint block as it
// sits in device memory -- map, E, spins, fields, sweep counters, flip / swap /
// near-tie counters, rebuild schedule, drift and the exchange counter, each at
// a 256-byte aligned offset in that order (state_bytes(h) bytes in all).  The
// *_enqueue helpers only issue asynchronous copies on stream st; the caller
// synchronises.
static int state_out_enqueue(potts_lr_t* h, char* p, cudaStream_t st)
{
    if (h->direct) {  // the direct sweep keeps no fields: rebuild them (FP64, exact) first
        cudaError_t e = launch_fields_direct(h->dj, h->L, h->R, 0, 0, h->direct_smem, st);
        if (e != cudaSuccess) return cuda_fail(e, "field rebuild");
    }
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    hd.magic = kStateMagic;
    hd.version = kStateVersion;
    hd.L = h->L;
    hd.q = h->q;
    hd.R = h->R;
    hd.precision = h->precision;
    hd.c = h->c;
    hd.Lpad = h->Lpad;
    hd.seed = h->seed;
    hd.nsweep = h->nsweep;
    hd.nexch = h->nexch;
    std::memcpy(&hd.sigma_bits, &h->sigma, 8);
    hd.temps_hash = h->temps_hash;
    hd.fx_bits = h->fx_bits;
    std::memcpy(p, &hd, sizeof(hd));
    PLR_CUDA(cudaMemcpyAsync(p + sizeof(hd), (const char*)h->arena + h->state_off, h->state_len,
                             cudaMemcpyDeviceToHost, st));
    return POTTS_LR_OK;
}

// a checkpoint of len bytes at p fits job h (size, shape, a permutation as slot map)
static int state_in_check(const potts_lr_t* h, const char* p, size_t len)
{
    if (len != state_bytes(h)) return fail(POTTS_LR_ESTATE, "checkpoint size %zu does not match %zu", len, state_bytes(h));
    StateHeader hd;
    std::memcpy(&hd, p, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != kStateVersion)
        return fail(POTTS_LR_ESTATE, "not a checkpoint of this format (version %u, expected %u)", hd.version,
                    kStateVersion);
    if (hd.L != h->L || hd.q != h->q || hd.R != h->R || hd.precision != h->precision || hd.Lpad != h->Lpad)
        return fail(POTTS_LR_ESTATE, "checkpoint does not match this job's L, q, R or precision");
    uint64_t sb;
    std::memcpy(&sb, &h->sigma, 8);
    if (hd.sigma_bits != sb || hd.fx_bits != h->fx_bits)
        return fail(POTTS_LR_ESTATE, "checkpoint was made with other couplings (sigma or the FX64 grid differ)");
    if (hd.seed != h->seed) return fail(POTTS_LR_ESTATE, "checkpoint was made with another seed");
    if (hd.c != h->c) return fail(POTTS_LR_ESTATE, "checkpoint was made with another pair factor c");
    if (hd.temps_hash != h->temps_hash)
        return fail(POTTS_LR_ESTATE, "checkpoint was made with another temperature grid");
    const size_t R = h->R;
    std::vector<int> map(R);
    std::memcpy(map.data(), p + sizeof(hd), R * 4);
    std::vector<char> seen(R, 0);
    for (size_t t = 0; t < R; ++t) {
        if (map[t] < 0 || (size_t)map[t] >= R || seen[map[t]]) return fail(POTTS_LR_ESTATE, "corrupt slot map");
        seen[map[t]] = 1;
    }
    return POTTS_LR_OK;
}

// copies of a checked checkpoint into job h (p must stay valid until st has run them)
static int state_in_enqueue(potts_lr_t* h, const char* p, cudaStream_t st)
{
    StateHeader hd;
    std::memcpy(&hd, p, sizeof(hd));
    PLR_CUDA(cudaMemcpyAsync((char*)h->arena + h->state_off, p + sizeof(hd), h->state_len, cudaMemcpyHostToDevice,
                             st));
    h->nsweep = hd.nsweep;
    h->nexch = hd.nexch;
    return POTTS_LR_OK;
}

int potts_lr_get_state(potts_lr_t* h, void* buf, size_t* len)
{
    if (!h || !len) return fail(POTTS_LR_EINVAL, "NULL argument");
    const size_t need = state_bytes(h);
    if (!buf) {
        *len = need;
        return POTTS_LR_OK;
    }
    if (*len < need) return fail(POTTS_LR_ESTATE, "checkpoint buffer too small (%zu < %zu)", *len, need);
    if (int rc = state_out_enqueue(h, (char*)buf, h->stream)) return rc;
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    *len = need;
    return POTTS_LR_OK;
}

int potts_lr_set_state(potts_lr_t* h, const void* buf, size_t len)
{
    if (!h || !buf) return fail(POTTS_LR_EINVAL, "NULL argument");
    if (int rc = state_in_check(h, (const char*)buf, len)) return rc;
    if (int rc = state_in_enqueue(h, (const char*)buf, h->stream)) return rc;
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    return POTTS_LR_OK;
}

int potts_lr_get_spins(potts_lr_t* h, uint8_t* out)
{
    if (!h || !out) return fail(POTTS_LR_EINVAL, "NULL argument");
    std::vector<uint32_t> packed((size_t)h->R * h->W);
    std::vector<int> map(h->R);
    PLR_CUDA(cudaMemcpyAsync(packed.data(), h->hj.spins, packed.size() * 4, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaMemcpyAsync(map.data(), h->hj.map, (size_t)h->R * 4, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < h->R; ++t) {
        const uint32_t* w = packed.data() + (size_t)map[t] * h->W;
        for (int i = 0; i < h->L; ++i) out[(size_t)t * h->L + i] = (uint8_t)((w[i >> 3] >> (4 * (i & 7))) & 15u);
    }
    return POTTS_LR_OK;
}

int potts_lr_get_fields(potts_lr_t* h, double* out)
{
    if (!h || !out) return fail(POTTS_LR_EINVAL, "NULL argument");
    if (int rc = fresh_fields(h)) return rc;
    const size_t per = (size_t)h->q * h->Lpad;
    std::vector<char> raw((size_t)h->R * per * h->wsize);
    std::vector<int> map(h->R);
    PLR_CUDA(cudaMemcpyAsync(raw.data(), h->hj.fields, raw.size(), cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaMemcpyAsync(map.data(), h->hj.map, (size_t)h->R * 4, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < h->R; ++t)
        for (int x = 0; x < h->q; ++x)
            for (int i = 0; i < h->L; ++i) {
                const size_t src = (size_t)map[t] * per + (size_t)x * h->Lpad + i;
                out[((size_t)t * h->q + x) * h->L + i] =
                    h->precision == POTTS_LR_FP64   ? ((const double*)raw.data())[src]
                    : h->precision == POTTS_LR_FX64 ? (double)((const long long*)raw.data())[src] * h->hj.fx_scale
                                                    : (double)((const float*)raw.data())[src];
            }
    return POTTS_LR_OK;
}

int potts_lr_get_energy(potts_lr_t* h, double* E)
{
    if (!h || !E) return fail(POTTS_LR_EINVAL, "NULL argument");
    std::vector<double> Er(h->R);
    std::vector<int> map(h->R);
    PLR_CUDA(cudaMemcpyAsync(Er.data(), h->hj.E, (size_t)h->R * 8, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaMemcpyAsync(map.data(), h->hj.map, (size_t)h->R * 4, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < h->R; ++t) E[t] = Er[map[t]];
    return POTTS_LR_OK;
}

int potts_lr_stats(potts_lr_t* h, uint64_t* acc_flip, uint64_t* acc_swap, uint64_t* near_ties)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    const size_t b = (size_t)h->R * 8;
    if (acc_flip) PLR_CUDA(cudaMemcpyAsync(acc_flip, h->hj.acc_flip, b, cudaMemcpyDeviceToHost, h->stream));
    if (acc_swap) PLR_CUDA(cudaMemcpyAsync(acc_swap, h->hj.acc_swap, b, cudaMemcpyDeviceToHost, h->stream));
    if (near_ties) PLR_CUDA(cudaMemcpyAsync(near_ties, h->hj.near, 16, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    return POTTS_LR_OK;
}

int potts_lr_sweep_info(potts_lr_t* h, int32_t* info, int n)
{
    if (!h || !info || n < 1) return fail(POTTS_LR_EINVAL, "bad argument");
    const JobDev& j = h->hj;
    const int kind = h->direct ? 3 : j.rc ? 4 : j.cl ? 2 : j.rf ? 1 : 0;
    // threads per CTA of each kernel: register configurations 1-3 run 7 update
    // warps, 4-8 run 15, plus the decision warp; the direct sweep one warp
    const int threads = kind == 3 ? 32
                        : kind == 2 || kind == 4 ? 512
                        : kind == 1 ? (h->precision == POTTS_LR_FX64 ? rfx_threads(j.rf) : (j.rf <= 3 ? 256 : 512))
                                    : (j.h_smem ? 256 : 512);
    const int32_t v[7] = {kind, kind == 0 ? j.h_smem : 0, kind == 0 ? j.j_smem : 0, j.rf, j.rc ? j.rc : j.cl, threads,
                          (int32_t)h->sweep_smem};
    for (int i = 0; i < n && i < 7; ++i) info[i] = v[i];
    return POTTS_LR_OK;
}

int potts_lr_set_rebuild_split(potts_lr_t* h, int parts)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    if (h->precision != POTTS_LR_FP32) return fail(POTTS_LR_EINVAL, "the split-BF16 rebuild is FP32 mode's");
    if (parts != 0 && parts != 2 && parts != 3) return fail(POTTS_LR_EINVAL, "parts must be 0, 2 or 3");
    h->hj.tc_parts = parts;
    PLR_CUDA(cudaMemcpyAsync(h->dj, &h->hj, sizeof(JobDev), cudaMemcpyHostToDevice, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    return POTTS_LR_OK;
}

int potts_lr_rebuild_info(potts_lr_t* h, int32_t* interval, uint32_t* rebuilds, double* last_drift)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    int sched[4] = {0, 0, 0, 0};
    unsigned long long drift[2] = {0ull, 0ull};
    PLR_CUDA(cudaMemcpyAsync(sched, h->hj.sched, 16, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaMemcpyAsync(drift, h->hj.drift_bits, 16, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    if (interval) *interval = sched[0];
    if (rebuilds) *rebuilds = (uint32_t)sched[2];
    if (last_drift) std::memcpy(last_drift, &drift[1], 8);
    return POTTS_LR_OK;
}

int potts_lr_set_wait_limits(potts_lr_t* h, uint64_t rebuild_ns, uint64_t plan_ns)
{
    if (!h) return fail(POTTS_LR_EINVAL, "handle is NULL");
    h->hj.tc_wait_ns = rebuild_ns;
    h->sched.wait_ns = plan_ns;
    PLR_CUDA(cudaMemcpyAsync(h->dj, &h->hj, sizeof(JobDev), cudaMemcpyHostToDevice, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    return POTTS_LR_OK;
}

int potts_lr_near_log(potts_lr_t* h, int32_t* events, int cap, int* n)
{
    if (!h || !n || cap < 0 || (cap > 0 && !events)) return fail(POTTS_LR_EINVAL, "bad argument");
    std::vector<int4> log(kNearLogCap);
    unsigned cnt = 0;
    PLR_CUDA(cudaMemcpyAsync(log.data(), h->hj.near_log, log.size() * sizeof(int4), cudaMemcpyDeviceToHost,
                             h->stream));
    PLR_CUDA(cudaMemcpyAsync(&cnt, h->hj.near_log_n, 4, cudaMemcpyDeviceToHost, h->stream));
    PLR_CUDA(cudaStreamSynchronize(h->stream));
    const int keep = std::min<int>(std::min<unsigned>(cnt, (unsigned)kNearLogCap), cap);
    for (int i = 0; i < keep; ++i) {
        int32_t* e = events + 5 * (size_t)i;
        e[0] = log[i].x & 1;         // kind
        e[1] = log[i].y;             // slot or pair
        e[2] = log[i].z;             // sweep or exchange index
        e[3] = log[i].w;             // attempt or stage
        e[4] = (log[i].x >> 1) & 1;  // decision
    }
    *n = (int)std::min<unsigned>(cnt, 0x7fffffffu);
    return POTTS_LR_OK;
}

// ---------------------------------------------------------------- batching

void potts_lr_batch_destroy(potts_lr_batch_t* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto& g : b->groups) {
        if (g.done) cudaEventDestroy(g.done);
        if (g.stream) cudaStreamDestroy(g.stream);
    }
    if (b->arena) cudaFree(b->arena);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int potts_lr_batch_create(potts_lr_t* const* jobs, int n, void* cuda_stream, potts_lr_batch_t** out)
{
    if (!out) return fail(POTTS_LR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!jobs || n < 1) return fail(POTTS_LR_EINVAL, "need at least one job");
    std::unordered_set<const void*> seen;
    for (int i = 0; i < n; ++i) {
        if (!jobs[i]) return fail(POTTS_LR_EINVAL, "job %d is NULL", i);
        if (!seen.insert(jobs[i]).second) return fail(POTTS_LR_EINVAL, "job %d listed twice", i);
    }
    potts_lr_batch_t* b = new (std::nothrow) potts_lr_batch();
    if (!b) return fail(POTTS_LR_ENOMEM, "host allocation failed");
    b->jobs.assign(jobs, jobs + n);
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        b->own_stream = true;
    }
    cudaError_t e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        potts_lr_batch_destroy(b);
        return cuda_fail(e, "cudaEventCreate");
    }
    // work tables per sweep kernel variant, longest slots first
    std::vector<JobDev> hjobs(n);
    std::map<int, std::vector<int2>> works;
    std::map<int, size_t> smem;
    // A batch whose slots fill the GPU many times over is bound by per-SM
    // throughput, not by the latency of single slots: there jobs that took the
    // cluster sweep automatically although their fields fit one CTA's shared
    // memory sweep with one CTA per slot (measured: about even per SM, and
    // fewer CTAs; identical results either way), and automatic clusters larger
    // than their fields need go back to the smallest.  8-byte fields, whose
    // clusters serve to spread the hot slots' updates, do so from four slots
    // per SM on: there every SM already holds a share of the hot slots.
    long long total_slots = 0;
    for (int i = 0; i < n; ++i) total_slots += jobs[i]->R;
    const long long nsm_b = std::max(1, device_sm_count());
    for (int i = 0; i < n; ++i) {
        hjobs[i] = jobs[i]->hj;
        int key = variant_key(jobs[i]);
        size_t sm = jobs[i]->sweep_smem;
        const bool crowded =
            !jobs[i]->direct && total_slots > (jobs[i]->precision == POTTS_LR_FP32 ? 16 : 4) * nsm_b;
        if (crowded && jobs[i]->cl_auto && jobs[i]->hj.h_smem) {
            hjobs[i].cl = 0;
            key = jobs[i]->precision * 4 + 2 + jobs[i]->hj.j_smem;
            sm = sweep_smem_bytes(hjobs[i]);
        } else if (crowded && jobs[i]->cl_auto && jobs[i]->hj.cl > jobs[i]->cl_min) {
            hjobs[i].cl = jobs[i]->cl_min;
            key = kClusterKey + 16 * jobs[i]->precision + jobs[i]->cl_min;
            sm = cluster_sweep_smem(jobs[i]->L, jobs[i]->q, jobs[i]->cl_min, jobs[i]->precision);
        }
        for (int t = 0; t < jobs[i]->R; ++t) works[key].push_back(make_int2(i, t));
        smem[key] = std::max(smem[key], sm);
        if (jobs[i]->precision == POTTS_LR_FP32 && jobs[i]->K > 0) b->fp32_jobs.push_back(i);
    }
    for (auto& kv : works)
        std::stable_sort(kv.second.begin(), kv.second.end(), [&](const int2& x, const int2& y) {
            const potts_lr_t* a = jobs[x.x];
            const potts_lr_t* c = jobs[y.x];
            return (long long)a->L * (a->q + 8) > (long long)c->L * (c->q + 8);
        });
    std::vector<int2> mwork;
    for (int i = 0; i < n; ++i) {
        b->meas_off.push_back((int)mwork.size());
        for (int t = 0; t < jobs[i]->R; ++t) mwork.push_back(make_int2(i, t));
        b->meas_smem = std::max(b->meas_smem, jobs[i]->measure_smem);
        b->meas_parts = std::max(b->meas_parts, jobs[i]->hj.meas_parts);
    }
    b->nmeas = (int)mwork.size();
    std::vector<int4> btiles;
    std::vector<int2> fwork;
    long long t64 = 0, t128 = 0;
    for (int i : b->fp32_jobs) {
        t64 += tc_tile_count(jobs[i]->L, jobs[i]->q, jobs[i]->R, 64);
        t128 += tc_tile_count(jobs[i]->L, jobs[i]->q, jobs[i]->R, 128);
    }
    b->tc_tn = tc_tile_width(t64, t128, device_sm_count());
    for (int i : b->fp32_jobs) {
        const potts_lr_t* h = jobs[i];
        tc_tiles(i, h->L, h->q, h->R, b->tc_tn, btiles);
        for (int t = 0; t < h->R; ++t) fwork.push_back(make_int2(i, t));
        b->onehot_blocks = std::max(b->onehot_blocks, h->onehot_blocks);
        b->fp_meas_smem = std::max(b->fp_meas_smem, h->measure_smem);
        b->fp_meas_parts = std::max(b->fp_meas_parts, h->hj.meas_parts);
    }
    tc_order_tiles(btiles);
    b->ntc_tiles = (int)btiles.size();
    b->nfp_work = (int)fwork.size();
    size_t bytes = align256(n * sizeof(JobDev));
    std::map<int, size_t> ow, osch;
    const int nsm = device_sm_count();
    for (auto& kv : works) {
        ow[kv.first] = bytes;
        bytes += align256(kv.second.size() * sizeof(int2) + 8);
        osch[kv.first] = bytes;
        bytes += align256(sweep_sched_bytes((int)kv.second.size(), nsm));
    }
    const size_t o_m = bytes;
    bytes += align256(mwork.size() * sizeof(int2));
    const size_t o_mb = bytes;
    bytes += align256(2 * mwork.size() * sizeof(double));
    const size_t o_bt = bytes;
    bytes += align256(btiles.size() * sizeof(int4) + 16);
    const size_t o_fw = bytes;
    bytes += align256(fwork.size() * sizeof(int2) + 8);
    const size_t o_fi = bytes;
    bytes += align256(b->fp32_jobs.size() * sizeof(int) + 4);
    e = cudaMalloc(&b->arena, bytes);
    if (e != cudaSuccess) {
        potts_lr_batch_destroy(b);
        return fail(POTTS_LR_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    b->djobs = (JobDev*)b->arena;
    b->dmeas = (int2*)((char*)b->arena + o_m);
    b->meas_buf = (double*)((char*)b->arena + o_mb);
    b->dtc_tiles = (int4*)((char*)b->arena + o_bt);
    b->dfp_work = (int2*)((char*)b->arena + o_fw);
    b->dfp_idx = (int*)((char*)b->arena + o_fi);
    for (auto& kv : works) {
        potts_lr_batch_t::Group g;
        g.key = kv.first;
        g.dwork = (int2*)((char*)b->arena + ow[kv.first]);
        g.nwork = (int)kv.second.size();
        g.smem = smem[kv.first];
        sweep_sched_carve((char*)b->arena + osch[kv.first], g.nwork, nsm, &g.sched);
        for (const int2& w : kv.second) g.sched.wait_ns = std::min(g.sched.wait_ns, jobs[w.x]->sched.wait_ns);
        g.stream = nullptr;
        g.done = nullptr;
        b->groups.push_back(g);
        e = cudaMemcpyAsync(g.dwork, kv.second.data(), kv.second.size() * sizeof(int2), cudaMemcpyHostToDevice,
                            b->stream);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && b->groups.size() > 1) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (auto& g : b->groups) {
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->djobs, hjobs.data(), n * sizeof(JobDev), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->dmeas, mwork.data(), mwork.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !btiles.empty())
        e = cudaMemcpyAsync(b->dtc_tiles, btiles.data(), btiles.size() * sizeof(int4), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !fwork.empty())
        e = cudaMemcpyAsync(b->dfp_work, fwork.data(), fwork.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !b->fp32_jobs.empty())
        e = cudaMemcpyAsync(b->dfp_idx, b->fp32_jobs.data(), b->fp32_jobs.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        potts_lr_batch_destroy(b);
        return cuda_fail(e, "potts_lr_batch_create");
    }
    *out = b;
    return POTTS_LR_OK;
}

static cudaError_t batch_enqueue_sweeps(potts_lr_batch_t* b)
{
    cudaError_t e;
    if (b->groups.size() == 1) {
        const auto& g = b->groups[0];
        if ((e = launch_variant(g.key, b->djobs, g.dwork, g.nwork, 1, g.smem, &g.sched, b->stream)) != cudaSuccess)
            return e;
    } else {
        // the kernel-variant groups hold different jobs: sweep them concurrently,
        // each on its own stream (fork / join through events, which a graph
        // capture turns into parallel branches), so that groups smaller than
        // the GPU share it instead of running one after another
        if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess) return e;
        for (const auto& g : b->groups) {
            if ((e = cudaStreamWaitEvent(g.stream, b->fork, 0)) != cudaSuccess) return e;
            if ((e = launch_variant(g.key, b->djobs, g.dwork, g.nwork, 1, g.smem, &g.sched, g.stream)) != cudaSuccess)
                return e;
            if ((e = cudaEventRecord(g.done, g.stream)) != cudaSuccess) return e;
        }
        for (const auto& g : b->groups)
            if ((e = cudaStreamWaitEvent(b->stream, g.done, 0)) != cudaSuccess) return e;
    }
    if (b->fp32_jobs.empty()) return cudaSuccess;
    // the rebuilds that fall due, for all FP32 jobs at once: tensor-core fields,
    // energy re-anchor, schedule update
    if ((e = launch_fields_tc(b->djobs, b->dfp_idx, (int)b->fp32_jobs.size(), b->onehot_blocks, b->dtc_tiles,
                              b->ntc_tiles, 1, b->tc_tn, b->stream)) != cudaSuccess)
        return e;
    if ((e = launch_measure(b->djobs, b->dfp_work, b->nfp_work, 1, 1, b->fp_meas_smem, b->fp_meas_parts,
                            b->stream)) != cudaSuccess)
        return e;
    return launch_rebuild_policy(b->djobs, b->dfp_idx, (int)b->fp32_jobs.size(), 1, b->stream);
}

static cudaError_t batch_enqueue_step(potts_lr_batch_t* b)
{
    cudaError_t e = batch_enqueue_sweeps(b);
    if (e != cudaSuccess) return e;
    return launch_exchange(b->djobs, (int)b->jobs.size(), b->stream);
}

static int batch_begin(potts_lr_batch_t* b)
{
    for (potts_lr_t* h : b->jobs) {
        if (h->stream == b->stream) continue;
        PLR_CUDA(cudaEventRecord(b->ev, h->stream));
        PLR_CUDA(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
    return POTTS_LR_OK;
}

static int batch_end(potts_lr_batch_t* b)
{
    PLR_CUDA(cudaEventRecord(b->ev, b->stream));
    for (potts_lr_t* h : b->jobs)
        if (h->stream != b->stream) PLR_CUDA(cudaStreamWaitEvent(h->stream, b->ev, 0));
    return POTTS_LR_OK;
}

int potts_lr_batch_sweep(potts_lr_batch_t* b, int n)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    if (n < 0) return fail(POTTS_LR_EINVAL, "n must be >= 0");
    int rc = batch_begin(b);
    if (rc) return rc;
    for (int s = 0; s < n; ++s) {
        cudaError_t e = batch_enqueue_sweeps(b);
        if (e != cudaSuccess) return cuda_fail(e, "batch sweep");
    }
    for (potts_lr_t* h : b->jobs) h->nsweep += (uint32_t)n;
    return batch_end(b);
}

int potts_lr_batch_exchange(potts_lr_batch_t* b)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    int rc = batch_begin(b);
    if (rc) return rc;
    cudaError_t e = launch_exchange(b->djobs, (int)b->jobs.size(), b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch exchange");
    for (potts_lr_t* h : b->jobs) h->nexch += 1u;
    return batch_end(b);
}

// measure every slot of every job into meas_E / meas_M of each job, then
// gather them into E / M (device arrays, job order)
static int batch_measure_enqueue(potts_lr_batch_t* b, double* E, double* M, cudaMemcpyKind kind)
{
    int rc = batch_begin(b);
    if (rc) return rc;
    cudaError_t e = launch_measure(b->djobs, b->dmeas, b->nmeas, 0, 0, b->meas_smem, b->meas_parts, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch measure");
    for (size_t i = 0; i < b->jobs.size(); ++i) {
        const potts_lr_t* h = b->jobs[i];
        const size_t bytes = (size_t)h->R * sizeof(double);
        if (E) PLR_CUDA(cudaMemcpyAsync(E + b->meas_off[i], h->hj.meas_E, bytes, kind, b->stream));
        if (M) PLR_CUDA(cudaMemcpyAsync(M + b->meas_off[i], h->hj.meas_M, bytes, kind, b->stream));
    }
    return batch_end(b);
}

int potts_lr_batch_measure_device(potts_lr_batch_t* b, double* E, double* M)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    return batch_measure_enqueue(b, E, M, cudaMemcpyDeviceToDevice);
}

int potts_lr_batch_measure(potts_lr_batch_t* b, double* E, double* M)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    int rc = batch_measure_enqueue(b, b->meas_buf, b->meas_buf + b->nmeas, cudaMemcpyDeviceToDevice);
    if (rc) return rc;
    const size_t bytes = (size_t)b->nmeas * sizeof(double);
    std::vector<double> host(2 * (size_t)b->nmeas);
    PLR_CUDA(cudaMemcpyAsync(host.data(), b->meas_buf, 2 * bytes, cudaMemcpyDeviceToHost, b->stream));
    PLR_CUDA(cudaStreamSynchronize(b->stream));
    if (E) std::memcpy(E, host.data(), bytes);
    if (M) std::memcpy(M, host.data() + b->nmeas, bytes);
    return POTTS_LR_OK;
}

int potts_lr_batch_run(potts_lr_batch_t* b, int nsteps, int steps_per_graph)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(POTTS_LR_EINVAL, "nsteps must be >= 0");
    if (steps_per_graph <= 0) steps_per_graph = 10;
    int rc = batch_begin(b);  // order after each job's pending work
    if (rc) return rc;
    if (nsteps >= steps_per_graph && (!b->exec || b->exec_steps != steps_per_graph)) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        PLR_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < steps_per_graph && e == cudaSuccess; ++s) e = batch_enqueue_step(b);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e, "batch capture");
        }
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        b->exec_steps = steps_per_graph;
    }
    int left = nsteps;
    while (left >= steps_per_graph) {
        PLR_CUDA(cudaGraphLaunch(b->exec, b->stream));
        left -= steps_per_graph;
    }
    for (; left > 0; --left) {
        cudaError_t e = batch_enqueue_step(b);
        if (e != cudaSuccess) return cuda_fail(e, "batch step");
    }
    for (potts_lr_t* h : b->jobs) {
        h->nsweep += (uint32_t)nsteps;
        h->nexch += (uint32_t)nsteps;
    }
    return batch_end(b);
}

int potts_lr_batch_state_size(potts_lr_batch_t* b, size_t* len)
{
    if (!b || !len) return fail(POTTS_LR_EINVAL, "NULL argument");
    size_t n = 0;
    for (const potts_lr_t* h : b->jobs) n += state_bytes(h);
    *len = n;
    return POTTS_LR_OK;
}

int potts_lr_batch_get_state(potts_lr_batch_t* b, void* buf, size_t len)
{
    if (!b || !buf) return fail(POTTS_LR_EINVAL, "NULL argument");
    size_t need = 0;
    for (const potts_lr_t* h : b->jobs) need += state_bytes(h);
    if (len != need) return fail(POTTS_LR_ESTATE, "batch checkpoint size %zu does not match %zu", len, need);
    if (int rc = batch_begin(b)) return rc;
    char* p = (char*)buf;
    for (potts_lr_t* h : b->jobs) {
        if (int rc = state_out_enqueue(h, p, b->stream)) return rc;
        p += state_bytes(h);
    }
    PLR_CUDA(cudaStreamSynchronize(b->stream));
    return POTTS_LR_OK;
}

int potts_lr_batch_set_state(potts_lr_batch_t* b, const void* buf, size_t len)
{
    if (!b || !buf) return fail(POTTS_LR_EINVAL, "NULL argument");
    size_t need = 0;
    for (const potts_lr_t* h : b->jobs) need += state_bytes(h);
    if (len != need) return fail(POTTS_LR_ESTATE, "batch checkpoint size %zu does not match %zu", len, need);
    // every job's part checked before any device memory changes
    const char* p = (const char*)buf;
    for (const potts_lr_t* h : b->jobs) {
        if (int rc = state_in_check(h, p, state_bytes(h))) return rc;
        p += state_bytes(h);
    }
    if (int rc = batch_begin(b)) return rc;
    p = (const char*)buf;
    for (potts_lr_t* h : b->jobs) {
        if (int rc = state_in_enqueue(h, p, b->stream)) return rc;
        p += state_bytes(h);
    }
    PLR_CUDA(cudaStreamSynchronize(b->stream));
    return POTTS_LR_OK;
}

int potts_lr_batch_sync(potts_lr_batch_t* b)
{
    if (!b) return fail(POTTS_LR_EINVAL, "batch is NULL");
    PLR_CUDA(cudaStreamSynchronize(b->stream));
    for (potts_lr_t* h : b->jobs) {
        int rc = check_status(h);
        if (rc) return rc;
    }
    return POTTS_LR_OK;
}

}  // extern "C"
