/*
 * potts_lr -- parallel-tempering Metropolis simulation of the one-dimensional
 * q-state Potts chain with long-range periodic couplings, on one GB300 GPU
 * (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * The model (A. Boer, arXiv:1308.5426):
 *   spins s_i in {0..q-1}, i = 0..L-1                       (Sec. 2, Eq. 1; the
 *                                                             paper's 1..q minus one)
 *   H = -(c/2) sum_{i != j} J*(|i-j|) delta(s_i, s_j)       (Eq. 2; pair factor c:
 *        c = 2 is the ordered double sum as printed, c = 1 counts each pair once
 *        as the paper's energy listing of Sec. 4.2 does)
 *   J*(r) = r^-s + L^-s [zeta(s, 1 + r/L) + zeta(s, 1 - r/L)],  s = 1 + sigma
 *                                                            (Eq. 5-7), J*(0) = 0
 *   Metropolis: sites k = 0..L-1 in order, proposal uniform over the other q-1
 *     states, accept iff dE <= 0 or u < exp(-beta dE)          (Eq. 8, Sec. 4.2)
 *   exchange: stage 0 pairs (t, t+1) with t even, then stage 1 with t odd;
 *     D = (beta_t - beta_{t+1})(E_t - E_{t+1}), accept iff D >= 0 or u < exp(D)
 *                                                            (Eq. 9, Sec. 4.2)
 *   M = (q N_max / L - 1) / (q - 1)                            (Eq. 10)
 * Temperature slots t = 0..R-1 keep their temperatures; configurations move
 * between slots on accepted exchanges.  All outputs are in slot order.
 *
 * Random numbers: Philox4x32-10 with key (seed_lo, seed_hi) and counters
 * (i, t, 0, 0) for the initial spins, (k, t, n, 1) for the Metropolis draw of
 * site k in slot t at absolute sweep n, (t, stage, m, 2) for exchange m.  A job
 * is therefore a pure function of its arguments and its call sequence, the
 * same alone or batched with others, and resumable bit-exactly.
 *
 * Precision modes:
 *   POTTS_LR_FP64 -- local fields h[x][i] = sum_{j != i} J*(|i-j|) delta(x, s_j)
 *     in FP64; every accept decision is the FP64 decision (decided in FP32
 *     where the FP32 margin is provably large enough, else in FP64).
 *   POTTS_LR_FP32 -- fields in FP32, decisions in FP32, running energy in FP64;
 *     at most every recompute_every sweeps the fields are rebuilt as
 *     H = C . onehot(S) on the tensor cores (C = J*(|i-j|) split into BF16
 *     hi + mid + lo parts, FP32 accumulation) and the energy is re-anchored
 *     from the spins.  Each rebuild measures the drift of the period it ends,
 *     max |h_fp32 - h_rebuilt| / Jtot; the interval halves when that exceeds
 *     7e-6 and doubles (up to recompute_every) when it is below 3.5e-6, so the
 *     fields stay within 1e-5 Jtot of exact.  The first interval is
 *     min(recompute_every, max(1, 2500 q / L)).  The schedule lives on the
 *     device, is part of the checkpoint and is the same alone or batched.
 *   POTTS_LR_FX64 -- fields as 64-bit integers in units of 2^-F, F = 61 - e
 *     where Jtot < 2^e (F = 58 for Jtot in [4, 8)), built from the couplings
 *     rounded to that grid, Jx(r) = round(J*(r) 2^F), |Jx(r) 2^-F - J*(r)| <=
 *     2^-(F+1).  Every field update is an exact integer add, so the fields
 *     never drift: they are, bit for bit, the direct sums of the rounded
 *     couplings (potts_lr_fields_recompute leaves them unchanged), and any
 *     energy difference is within L 2^-(F+1) <= L 2^-61 Jtot of the FP64
 *     couplings' (below 3e-14 Jtot at L = 65536).  Decisions follow FP64
 *     mode's rule, the exact difference converted to FP64 once, so
 *     trajectories equal FP64 mode's except where |beta dE + ln u| is within
 *     rounding of zero (counted as near ties).  Same memory as FP64 mode; the updates run on the integer pipes
 *     instead of GB300's narrow FP64 pipe.  sweep_variant 0 to 3 or 5 (0 keeps
 *     the fields in registers where a register configuration holds them).  EINVAL if
 *     sigma is so small that F would fall below 24.  Energies and fields come
 *     out in FP64 (fields converted from field units).
 *
 * Errors: every int-returning call returns POTTS_LR_OK (0) or one of the codes
 * below; potts_lr_last_error() gives a message for the calling thread.  A call
 * that fails leaves the handle unchanged unless its description says otherwise.
 *
 * Ownership and threads: a handle owns all of its device memory; arrays passed
 * in are copied (or read before the call returns).  A handle must not be used
 * from two threads at once; distinct handles are independent.
 */
#ifndef POTTS_LR_H
#define POTTS_LR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define POTTS_LR_OK 0
#define POTTS_LR_EINVAL 1   /* argument out of range */
#define POTTS_LR_ENOMEM 2   /* device or host allocation failed */
#define POTTS_LR_ECUDA 3    /* CUDA runtime error (message has the detail) */
#define POTTS_LR_ETIMEOUT 4 /* a bounded device wait expired; results invalid */
#define POTTS_LR_ESTATE 5   /* checkpoint buffer does not match the handle */

#define POTTS_LR_FP64 0
#define POTTS_LR_FP32 1
#define POTTS_LR_FX64 2

#define POTTS_LR_MAX_Q 16
#define POTTS_LR_NEAR_LOG_CAP 256 /* near-tie events kept per job (potts_lr_near_log) */

typedef struct potts_lr potts_lr_t;

typedef struct {
    int precision;       /* POTTS_LR_FP64 (default), POTTS_LR_FP32 or POTTS_LR_FX64 */
    int recompute_every; /* FP32 mode: longest interval K between tensor-core field
                            rebuilds (default 100; 0 = only on explicit request) */
    int pair_factor;     /* c in Eq. 2: 2 (default) or 1 */
    void* cuda_stream;   /* cudaStream_t to run on; NULL = a stream the handle creates */
    int sweep_variant;   /* 0 = automatic (default); FP32 mode: 1 = fields in shared or
                            global memory, 2 = fields in registers (EINVAL if the shape
                            does not fit: L <= 1120, or L <= 2400 with q <= 10, L <= 4320
                            with q <= 8, L <= 7680 with q <= 5, L <= 12480 with q <= 3,
                            L <= 16800 with q = 2);
                            either mode: 3 = fields in global memory even where they fit
                            in shared memory (FX64 mode: 0, 1, 2, 3 and 5; 2 = the FX64 fields
                            in registers, EINVAL unless L <= 448, or L <= 1120 with q <= 8,
                            L <= 2400 with q <= 5, L <= 4320 with q <= 3); FP64 mode:
                            4 = the direct sweep of the
                            paper (Sec. 4.2: every proposal sums its O(L) interaction,
                            no fields; same decisions up to rounding of the sum; L up to
                            about 27000); any mode: 5 = the slot's fields spread over
                            the shared memory of a cluster of 2, 4 or 8 CTAs (the
                            smallest that holds them; EINVAL if 8 do not; chosen by 0
                            where the fields fit no registers and fit no single
                            CTA's shared memory, and also where they take more than
                            88 KB of it (FP32) or more than 64 KB (FP64, FX64) with
                            R x C at most the SM count; chosen by 0 in FP64 and FX64
                            modes, C is then the largest of 2, 4, 8 with R x C at
                            most 4 x the SM count and C^2 <= L / 128, at least the
                            smallest that holds them; a batch with more than 16
                            (FP32) or 4 (FP64, FX64) slots per SM gives such jobs the
                            smallest C, or one CTA per slot where the fields fit one
                            CTA); FP32 and FX64 modes: 6 = the slot's fields in the
                            registers of a cluster of 2, 4 or 8 CTAs (FP32: q <= 8, L <=
                            4320 C, or q <= 12, L <= 2400 C; FX64: q <= 7, L <= 2400 C;
                            the smallest C that holds them; EINVAL beyond L = 34560 or
                            19200; chosen by 0 where
                            no single CTA's registers hold the chain and this does,
                            before either shared-memory placement); FP32 mode:
                            16 + c (c = 1..8) = register
                            configuration c (E sites per update thread x update warps:
                            1x7, 2x7, 5x7, 5x15, 9x15, 16x15, 26x15, 35x15; q at most
                            16, 16, 16, 10, 8, 5, 3, 2; EINVAL if L > 32 x E x warps or q
                            too large); FX64 mode: 16 + c (c = 1..6) = FX64 register
                            configuration c (1x7, 2x7, 4x8, 5x7, 5x15, 9x15; q at most 16,
                            16, 8, 8, 5, 3).  All variants of a precision give identical
                            results. */
    int site_order;      /* 0 = sites 0..L-1 in order (default); 1 = random sites: attempt
                            m of a sweep at site floor(x3 L / 2^32) of Philox counter
                            (m, slot, sweep, 3) -- the other reading of Sec. 4.2; runs
                            on the direct sweep (FP64, sweep_variant 0 or 4, else EINVAL) */
} potts_lr_opts;

/* Fill *opts with the defaults above. */
int potts_lr_default_opts(potts_lr_opts* opts);

/*
 * Create a job: R temperature slots of an L-site chain with q states, coupling
 * exponent sigma (Eq. 4-6), absolute temperatures temps[0..R-1] (k_B = 1,
 * Sec. 3; host array, copied), Philox seed.  Draws the initial spins, builds the
 * FP64 J* table and the exact local fields, and computes the initial energies.
 * Errors: EINVAL for L < 2, L > 65536, q < 2, q > 16, sigma <= 0 or not finite,
 * R < 1 or R > 4096, a non-positive or non-finite temperature, pair_factor not
 * 1 or 2, unknown precision; ENOMEM; ECUDA.  On error *out is set to NULL.
 */
int potts_lr_create(int L, int q, double sigma, const double* temps, int R, uint64_t seed,
                    const potts_lr_opts* opts, potts_lr_t** out);

/* n full Metropolis sweeps of every slot (L attempts per slot per sweep, Eq. 8),
 * asynchronous on the handle's stream.  In FP32 mode the tensor-core field
 * rebuild runs after the sweeps at which the schedule above makes it due.
 * n >= 0. */
int potts_lr_sweep(potts_lr_t* h, int n);

/* One exchange step (Eq. 9): stage 0 then stage 1, asynchronous. */
int potts_lr_exchange(potts_lr_t* h);

/* Energy (Eq. 2) and magnetisation (Eq. 10) of every slot, computed on the GPU
 * from the packed spins (energy = -(c/2) sum_r J*(r) N_r, N_r the number of
 * sites i with s_i = s_{(i+r) mod L}).  E and M are caller-owned host arrays
 * of R doubles (either may be NULL).  Synchronises the handle's stream. */
int potts_lr_measure(potts_lr_t* h, double* E, double* M);

/* As potts_lr_measure, but E and M are device arrays of R doubles and the call
 * is asynchronous (usable inside a captured CUDA graph). */
int potts_lr_measure_device(potts_lr_t* h, double* E, double* M);

/* Rebuild the local fields from the spins: FP32 mode -- split-BF16 tensor-core
 * product H = C . onehot(S) with FP32 accumulation; FP64 mode -- direct FP64
 * sums; FX64 mode -- direct integer sums of the rounded couplings (identical,
 * bit for bit, to the swept fields).  Re-anchors the running energies from
 * the spins.  Asynchronous. */
int potts_lr_fields_recompute(potts_lr_t* h);

/* Largest |h - h_exact| / Jtot over all fields of all slots, h_exact the FP64
 * direct rebuild of the current spins (the FP32 drift measure).  Synchronises. */
int potts_lr_fields_error(potts_lr_t* h, double* max_err);

/* Checkpoint.  With buf == NULL sets *len to the size needed.  Otherwise
 * writes the complete state (spins, fields, energies, slot map, counters) into
 * buf (*len bytes available, *len set to bytes written); ESTATE if too small.
 * Synchronises. */
int potts_lr_get_state(potts_lr_t* h, void* buf, size_t* len);

/* Restore a checkpoint written by potts_lr_get_state of a handle created with
 * the same L, q, sigma, temperatures, R, seed, precision and pair factor;
 * ESTATE if any of them differs (the checkpoint's header records them), or
 * the size, format version or slot map is wrong.  Continuing from a restored
 * state reproduces the uninterrupted run bit for bit. */
int potts_lr_set_state(potts_lr_t* h, const void* buf, size_t len);

/* Spins of every slot, out[t*L + i] in 0..q-1 (host array of R*L bytes). Syncs. */
int potts_lr_get_spins(potts_lr_t* h, uint8_t* out);

/* Local fields of every slot as doubles, out[(t*q + x)*L + i] (host array of
 * R*q*L doubles; FX64 mode: field units times 2^-F, exact). Syncs. */
int potts_lr_get_fields(potts_lr_t* h, double* out);

/* Running energies (the value the exchange step uses) of every slot. Syncs. */
int potts_lr_get_energy(potts_lr_t* h, double* E);

/* Counters since create, host arrays (any may be NULL): acc_flip[R] accepted
 * Metropolis flips per slot; acc_swap[R] accepted exchanges of pair (t, t+1)
 * (entry R-1 is 0); near_ties[2] = {Metropolis, exchange} decisions whose FP64
 * margin |beta dE + ln u| (resp. |D - ln u|) was below 1e-9. Syncs. */
int potts_lr_stats(potts_lr_t* h, uint64_t* acc_flip, uint64_t* acc_swap, uint64_t* near_ties);

/* Log of the near ties counted by potts_lr_stats, so that a checker whose
 * exp and log round differently can see where they fell and adopt the
 * decisions taken here (the re-synchronisation reading of Eq. 8 and Eq. 9).
 * events: host array of cap rows of 5 int32 {kind (0 = Metropolis, 1 =
 * exchange), slot t (exchange: pair (t, t+1)), sweep index n (exchange:
 * exchange index m), attempt within the sweep (the site k in sequential
 * order; exchange: stage 0 or 1), decision (1 = accepted)}.  The rows are
 * the first POTTS_LR_NEAR_LOG_CAP near ties since create in the order the
 * device recorded them (the order between slots of one launch is not
 * fixed); min(cap, *n, POTTS_LR_NEAR_LOG_CAP) rows are written.  *n = near
 * ties logged since create (more than the capacity are counted, not kept).
 * The log is not part of a checkpoint.  Only the FP64 rule logs (FP64 and
 * FX64 modes, the exchange of any mode).  EINVAL for a NULL handle or n, cap
 * < 0, or events NULL with cap > 0.  Synchronises. */
int potts_lr_near_log(potts_lr_t* h, int32_t* events, int cap, int* n);

/* Bounds of the handle's device waits (the paper has no counterpart), in ns:
 *   rebuild_ns -- each pipeline wait of the FP32 tensor-core rebuild (default
 *     4e9).  When one expires, the rebuild stops, lets its own copies and
 *     tensor-core operations finish, frees its tensor memory and returns; the
 *     fields are then invalid, and the next synchronising call on the handle
 *     (or on a batch holding it) returns ETIMEOUT.  The next
 *     potts_lr_fields_recompute under a sufficient bound makes them valid.
 *   plan_ns -- how long sweep CTAs wait for the other CTAs' first claims
 *     under the SM placement plan (default 50000).  Expiry only changes which
 *     SM sweeps which slot, never a result.
 * Small values exist to test the expiry paths.  They apply to the handle's
 * own calls and to batches created afterwards (a batch group takes the
 * smallest plan_ns of its jobs).  Synchronises.  EINVAL for a NULL handle. */
int potts_lr_set_wait_limits(potts_lr_t* h, uint64_t rebuild_ns, uint64_t plan_ns);

/* FP32 mode: how many BF16 parts of J* the tensor-core rebuild multiplies
 * (the paper has no counterpart): 3 (hi + mid + lo, representation error
 * about 2^-25 of each coupling), 2 (hi + mid, about 2^-17, two thirds of the
 * tensor-core work) or 0 (the default: 2 while the automatic schedule rebuilds
 * every sweep, where the sweep's drift is an order of magnitude larger than
 * the split's error, else 3).  Applies to the handle's own
 * rebuilds and to batches created afterwards.  EINVAL for a NULL handle, a
 * job not in FP32 mode, or parts other than 0, 2 and 3.  Synchronises.
 * (Scheduled rebuilds re-anchor the running energy from the spins once at
 * least 8 sweeps have passed since the last anchor; explicit ones always.) */
int potts_lr_set_rebuild_split(potts_lr_t* h, int parts);

/* FP32 mode's rebuild schedule (any argument may be NULL): *interval = the
 * current interval between rebuilds in sweeps (it halves or doubles with the
 * measured drift, up to recompute_every), *rebuilds = automatic rebuilds done
 * since create (0 in the other modes), *last_drift = max |h_fp32 -
 * h_rebuilt| / Jtot measured by the last of them.  Synchronises. */
int potts_lr_rebuild_info(potts_lr_t* h, int32_t* interval, uint32_t* rebuilds, double* last_drift);

/* Sweep and exchange counts since create. */
int potts_lr_counters(potts_lr_t* h, uint32_t* nsweep, uint32_t* nexch);

/* Wait for all work queued on the handle's stream. */
int potts_lr_sync(potts_lr_t* h);

void potts_lr_destroy(potts_lr_t* h);

/* Message of the last failed call on this thread ("" if none). */
const char* potts_lr_last_error(void);

/* The FP64 coupling table of Eq. 6 (Hurwitz zeta by Euler-Maclaurin):
 * out[r] = J*(r) for r = 0..L-1, out[0] = 0; host array of L doubles. */
int potts_lr_jstar(int L, double sigma, double* out);

/*
 * Batching: run many jobs (any mix of L, q, sigma, R, precision) together.  One
 * batch step is one sweep of every slot of every job followed by one exchange
 * step of every job (the FP32 rebuild runs for each job on its own schedule).
 * The steps are launched as one CUDA graph per chunk of steps, captured on the
 * first run and replayed afterwards.  Each job's results are bit-identical to
 * running it alone with the same call sequence.  The jobs must outlive the
 * batch and must not be used on their own while a batch run is in flight.
 */
typedef struct potts_lr_batch potts_lr_batch_t;

/* jobs: host array of n handles (copied). Errors: EINVAL (n < 1, NULL job,
 * a job listed twice), ENOMEM, ECUDA. */
int potts_lr_batch_create(potts_lr_t* const* jobs, int n, void* cuda_stream, potts_lr_batch_t** out);

/* nsteps batch steps, asynchronous on the batch stream; steps_per_graph is the
 * chunk captured into one graph (0 = default 10). */
int potts_lr_batch_run(potts_lr_batch_t* b, int nsteps, int steps_per_graph);

/* The parts of a batch step as separate asynchronous launches on the batch
 * stream: n sweeps of every slot of every job (one kernel launch per precision
 * class, FP32 rebuilds as they fall due), and one exchange step of every job
 * (one launch).  batch_run is equivalent to alternating these. */
int potts_lr_batch_sweep(potts_lr_batch_t* b, int n);
int potts_lr_batch_exchange(potts_lr_batch_t* b);

/* Energies and magnetisations of every slot of every job, in job order then
 * slot order (sum of the jobs' R entries each), one kernel launch.
 * potts_lr_batch_measure: host arrays, synchronises.
 * potts_lr_batch_measure_device: device arrays, asynchronous. */
int potts_lr_batch_measure(potts_lr_batch_t* b, double* E, double* M);
int potts_lr_batch_measure_device(potts_lr_batch_t* b, double* E, double* M);

int potts_lr_batch_sync(potts_lr_batch_t* b);
void potts_lr_batch_destroy(potts_lr_batch_t* b);

/* Checkpoint of every job of the batch in one call: the jobs' checkpoints
 * (each exactly what potts_lr_get_state writes for that job) back to back in
 * job order, len = potts_lr_batch_state_size bytes.  All copies are issued on
 * the batch stream with one synchronisation at the end (pinned host memory
 * makes them run at link speed).  potts_lr_batch_set_state checks every job's
 * part (everything potts_lr_set_state checks) before it changes any device
 * memory; a mismatch returns ESTATE and leaves every job as it was.  Errors:
 * EINVAL (NULL), ESTATE (len or a part does not match), ECUDA. */
int potts_lr_batch_state_size(potts_lr_batch_t* b, size_t* len);
int potts_lr_batch_get_state(potts_lr_batch_t* b, void* buf, size_t len);
int potts_lr_batch_set_state(potts_lr_batch_t* b, const void* buf, size_t len);

/* Allocation-free measurement (the paper has no counterpart).  Same energy
 * (Eq. 2 via the distance counts N_r) and magnetisation (Eq. 10) as
 * potts_lr_measure, for callers that cannot allocate device memory and so
 * cannot create a handle: code inside a host framework that owns all device
 * memory, or a latency-critical loop that must not pay the synchronisation a
 * cudaMalloc/cudaFree can bring.  It calls no cudaMalloc, cudaFree or other
 * allocating routine; its scratch (the per-configuration results the kernel
 * writes before they are copied out) is a fixed device array inside this
 * library, 64 KB, held on every GPU that loads the library until exit.
 *   spins:  device array, R configurations of packed spins, [R][ceil(L/8)]
 *           uint32 words, spin i of configuration r in bits 4(i%8)..4(i%8)+3
 *           of word i/8 of row r (values 0..q-1)
 *   jstar:  device array of L doubles, J*(r) for r = 0..L-1 (potts_lr_jstar)
 *   E, M:   device arrays of R doubles (outputs); pair_factor = c (1 or 2)
 *   cuda_stream: cudaStream_t to run on (NULL = the default stream); the call
 *           is asynchronous on it.
 * EINVAL for a NULL pointer, L outside [2, 65536], q outside [2, 16],
 * pair_factor not 1 or 2, or R outside [1, 4096] (the scratch size); ECUDA for
 * a runtime error.  The first call on a device looks up the device address of
 * the scratch array (cudaGetSymbolAddress), so make that first call before any
 * stream capture; the first call after a cudaDeviceReset looks it up again
 * (the address is cached with the device's context).  Every call writes every scratch entry it later reads, so
 * nothing needs clearing between calls; but all calls share the one array, so
 * calls that overlap on the GPU (different streams, or threads) race. */
int potts_lr_measure_static(const uint32_t* spins, int L, int q, int R, const double* jstar, int pair_factor,
                            double* E, double* M, void* cuda_stream);

/* Measurement utility (the paper has no counterpart): throughput of this
 * GPU's FP64 add pipe (what = 0, adds/s), FP32 add pipe (what = 1, adds/s),
 * shared memory (what = 2, bytes/s loaded + stored), L2 (what = 3, bytes/s
 * loaded + stored on a 32 MB buffer resident in L2) or 64-bit integer adds
 * (what = 4, adds/s: the FX64 field update), measured with CUDA
 * events on the current device; the roofline denominators of the sweep
 * kernels.  Synchronous; allocates 16 bytes of device memory for the call
 * (32 MB for what = 3).  On any failure (ECUDA, ENOMEM) *value is left
 * untouched. */
int potts_lr_probe(int what, double* value);

/* Which sweep kernel the handle runs (the paper has no counterpart; it lets a
 * benchmark label and bound what it timed).  info: host array of n int32
 * (n >= 1; entries past 7 are not written): [0] kernel (0 = fields in shared
 * or global memory, 1 = fields in registers, 2 = fields shared by a CTA
 * cluster in shared memory, 3 = the direct sweep without fields, 4 = fields
 * in the registers of a CTA cluster); [1] fields in shared memory (0/1); [2]
 * coupling table in shared memory (0/1); [3] register configuration (1..8,
 * else 0); [4] cluster size (2, 4 or 8, else 0); [5]
 * threads per CTA; [6] dynamic shared memory per CTA in bytes.  EINVAL for a
 * NULL handle or info, or n < 1. */
int potts_lr_sweep_info(potts_lr_t* h, int32_t* info, int n);

#ifdef __cplusplus
}
#endif

#endif /* POTTS_LR_H */
