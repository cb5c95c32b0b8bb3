/*
 * Plain CPU oracle for parallel-tempering Metropolis simulation of the
 * one-dimensional q-state Potts chain with long-range periodic couplings
 * (Boer, "GPU-based simulation of the long-range Potts model via parallel
 * tempering", arXiv:1308.5426).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously-correct reference
 * that the GPU path is checked against.  Only the test suite, the smoke check
 * of the package entry and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the GPU library: the
 * Philox generator below is written here from its published definition, the
 * coupling table J* arrives as an input array (built by oracle/jstar.py), and
 * every energy is a plain double sum.
 *
 * Everything is FP64.  Conventions (the paper is silent or ambiguous on these;
 * each reading is listed in the design notes):
 *   - spins s_i in 0..q-1 (the paper's 1..q shifted by one, Eq. 1);
 *   - H = -(c/2) * sum_{i != j} J*(|i-j|) delta(s_i, s_j)   (Eq. 2 with a pair
 *     factor c: c = 2 is the ordered double sum as Eq. 2 is printed, c = 1
 *     counts each unordered pair once as the energy listing of Sec. 4.2 does);
 *   - J*(0) = 0 (self-interaction excluded, i != j);
 *   - Metropolis (Eq. 8): sites k = 0..L-1 in order, one proposal per site,
 *     proposal uniform over the other q-1 states, accept iff dE <= 0 or
 *     u < exp(-beta dE); or, in random-site order (the other reading of
 *     Sec. 4.2), L attempts m = 0..L-1 per sweep, attempt m at a site drawn
 *     uniformly, k_m = floor(x3 * L / 2^32), then the same proposal and rule;
 *   - replica exchange (Eq. 9, Sec. 4.2): stage 0 pairs (t, t+1) with t even,
 *     stage 1 with t odd, accept iff D >= 0 or u < exp(D),
 *     D = (beta_t - beta_{t+1}) (E_t - E_{t+1}); configurations move between
 *     temperature slots, the slots keep their temperatures;
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with
 *     key (seed_lo, seed_hi) and counter
 *         init:       (i, t, 0, 0)
 *         Metropolis: (k, t, n, 1)   n = absolute sweep index
 *         Metropolis, random-site order: (m, t, n, 3)
 *         exchange:   (t, stage, m, 2)   m = absolute exchange index
 *     init spin = floor(x0 * q / 2^32);
 *     proposal b = (a + 1 + floor(x0 * (q-1) / 2^32)) mod q;
 *     u = ((((x1 << 32) | x2) >> 11) + 1) * 2^-53, in (0, 1].
 *
 * A "near tie" is a decision whose margin |beta dE + ln u| (Metropolis) or
 * |D - ln u| (exchange) is below 1e-9: there rounding differences between two
 * correct FP64 implementations may flip the decision.  They are counted, the
 * first sweep at which one happened is recorded per slot, and each is logged
 * (kind, slot or pair, sweep or exchange index, attempt or stage, the
 * oracle's own decision, the decision taken).
 *
 * Re-synchronisation at near ties (the reading of Eq. 8 and Eq. 9 for two
 * implementations whose exp and log round differently): the caller may hand
 * the oracle a table of decisions taken elsewhere, keyed by (kind, slot or
 * pair, sweep or exchange index, attempt or stage).  At a decision the oracle
 * itself counts as a near tie, and only there, it adopts the tabled decision
 * instead of its own.  Adoptions are counted per slot (and for the exchange),
 * as are those that reversed the oracle's own decision.  Anywhere else the
 * table is never consulted, so it cannot hide a real disagreement.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_INIT 0u
#define ORC_TAG_METRO 1u
#define ORC_TAG_EXCH 2u
#define ORC_TAG_SITE 3u
#define ORC_NEAR_TIE 1e-9
#define ORC_LOG_CAP 4096 /* near-tie events kept per job (all are counted) */

/* ---- Philox4x32-10, from the published definition (SC'11, Sec. 3) ---- */
static void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t bump0 = 0x9E3779B9u, bump1 = 0xBB67AE85u; /* Weyl key bumps */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * c0;
        uint64_t p1 = (uint64_t)mul1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += bump0; k1 += bump1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* exported for the generator pin test */
void oracle_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    orc_philox(ctr, key, out);
}

static double orc_unit(uint32_t x1, uint32_t x2)
{
    uint64_t bits = (((uint64_t)x1 << 32) | (uint64_t)x2) >> 11; /* 53 bits */
    return (double)(bits + 1u) * 0x1p-53;                         /* (0, 1] */
}

typedef struct {
    int L, q, R, c;
    int random_sites; /* 0: sites in order; 1: each attempt at a uniformly drawn site */
    uint32_t key[2];
    double* J;        /* J[r] = J*(r), r = 0..L-1, J[0] = 0 */
    double* beta;     /* beta[t], slot t */
    uint8_t* s;       /* s[t*L + i]: configuration currently held by slot t */
    double* E;        /* running energy of the configuration held by slot t */
    double* h;        /* fields h[(t*q + x)*L + i] = sum_{j != i} J*(|i-j|) delta(x, s_j) */
    uint32_t nsweep;  /* sweeps done since create */
    uint32_t nexch;   /* exchange steps done since create */
    uint64_t* acc_flip;   /* per slot */
    uint64_t* att_swap;   /* per pair (t, t+1) */
    uint64_t* acc_swap;   /* per pair (t, t+1) */
    uint64_t* near_metro; /* per slot */
    int64_t* first_near;  /* per slot: first sweep with a Metropolis near tie, or -1 */
    uint64_t near_exch;
    int64_t first_near_exch; /* first exchange index with a near tie, or -1 */
    /* near-tie log: [ORC_LOG_CAP][6] = {kind (0 Metropolis, 1 exchange), slot t
       (exchange: pair (t, t+1)), sweep n (exchange: index m), attempt m within
       the sweep (exchange: stage), own decision, decision taken} */
    int32_t* log;
    uint64_t nlog;        /* events seen (the first ORC_LOG_CAP are kept) */
    pthread_mutex_t log_mu;
    /* decisions to adopt at near ties: [novr][5] = {kind, t, index, attempt or
       stage, decision} */
    int32_t* ovr;
    int novr;
    uint64_t* adopted_metro; /* per slot: near-tie decisions taken from the table */
    uint64_t* flipped_metro; /* per slot: of those, the ones that reversed the oracle's own */
    uint64_t adopted_exch, flipped_exch;
} oracle_t;

static double orc_J(const oracle_t* o, int i, int j)
{
    int r = i > j ? i - j : j - i; /* |i - j|, Eq. 5 distance */
    return o->J[r];
}

/* E = -(c/2) sum_{i != j} J*(|i-j|) delta(s_i, s_j), the plain double sum (Eq. 2) */
double oracle_energy_direct(const oracle_t* o, int t)
{
    const uint8_t* s = o->s + (size_t)t * o->L;
    double sum = 0.0;
    for (int i = 0; i < o->L; ++i)
        for (int j = 0; j < o->L; ++j)
            if (i != j && s[i] == s[j]) sum += orc_J(o, i, j);
    return -0.5 * (double)o->c * sum;
}

/* M = (q N_max / L - 1) / (q - 1), Eq. 10 */
double oracle_magnetisation(const oracle_t* o, int t)
{
    const uint8_t* s = o->s + (size_t)t * o->L;
    int counts[256] = {0};
    for (int i = 0; i < o->L; ++i) counts[s[i]]++;
    int nmax = 0;
    for (int x = 0; x < o->q; ++x)
        if (counts[x] > nmax) nmax = counts[x];
    return ((double)o->q * (double)nmax / (double)o->L - 1.0) / (double)(o->q - 1);
}

/* fields of slot t from scratch: h[x][i] = sum_{j != i} J*(|i-j|) delta(x, s_j) */
static void orc_fields_direct(oracle_t* o, int t)
{
    const int L = o->L, q = o->q;
    const uint8_t* s = o->s + (size_t)t * L;
    double* h = o->h + (size_t)t * q * L;
    for (int x = 0; x < q; ++x)
        for (int i = 0; i < L; ++i) {
            double sum = 0.0;
            for (int j = 0; j < L; ++j)
                if (j != i && s[j] == x) sum += orc_J(o, i, j);
            h[(size_t)x * L + i] = sum;
        }
}

/* the tabled decision for a near tie at (kind, t, index, attempt), or -1 */
static int orc_override(const oracle_t* o, int kind, int t, uint32_t index, int attempt)
{
    for (int i = 0; i < o->novr; ++i) {
        const int32_t* e = o->ovr + 5 * (size_t)i;
        if (e[0] == kind && e[1] == t && (uint32_t)e[2] == index && e[3] == attempt) return e[4] ? 1 : 0;
    }
    return -1;
}

/* append one near-tie event (slots may be swept on several threads) */
static void orc_log(oracle_t* o, int kind, int t, uint32_t index, int attempt, int own, int taken)
{
    pthread_mutex_lock(&o->log_mu);
    if (o->nlog < ORC_LOG_CAP) {
        int32_t* e = o->log + 6 * (size_t)o->nlog;
        e[0] = kind; e[1] = t; e[2] = (int32_t)index; e[3] = attempt; e[4] = own; e[5] = taken;
    }
    o->nlog++;
    pthread_mutex_unlock(&o->log_mu);
}

void oracle_destroy(oracle_t* o)
{
    if (!o) return;
    free(o->J); free(o->beta); free(o->s); free(o->E); free(o->h);
    free(o->acc_flip); free(o->att_swap); free(o->acc_swap);
    free(o->near_metro); free(o->first_near);
    free(o->log); free(o->ovr); free(o->adopted_metro); free(o->flipped_metro);
    pthread_mutex_destroy(&o->log_mu);
    free(o);
}

oracle_t* oracle_create(int L, int q, int c, const double* J, int R, const double* beta,
                        uint64_t seed, int with_fields)
{
    if (L < 2 || q < 2 || q > 255 || R < 1 || (c != 1 && c != 2)) return NULL;
    oracle_t* o = (oracle_t*)calloc(1, sizeof(oracle_t));
    if (!o) return NULL;
    o->L = L; o->q = q; o->R = R; o->c = c;
    o->key[0] = (uint32_t)(seed & 0xffffffffu);
    o->key[1] = (uint32_t)(seed >> 32);
    o->J = (double*)malloc(sizeof(double) * L);
    o->beta = (double*)malloc(sizeof(double) * R);
    o->s = (uint8_t*)malloc((size_t)R * L);
    o->E = (double*)malloc(sizeof(double) * R);
    o->h = with_fields ? (double*)malloc(sizeof(double) * (size_t)R * q * L) : NULL;
    o->acc_flip = (uint64_t*)calloc(R, sizeof(uint64_t));
    o->att_swap = (uint64_t*)calloc(R, sizeof(uint64_t));
    o->acc_swap = (uint64_t*)calloc(R, sizeof(uint64_t));
    o->near_metro = (uint64_t*)calloc(R, sizeof(uint64_t));
    o->first_near = (int64_t*)malloc(sizeof(int64_t) * R);
    o->log = (int32_t*)malloc(sizeof(int32_t) * 6 * ORC_LOG_CAP);
    o->adopted_metro = (uint64_t*)calloc(R, sizeof(uint64_t));
    o->flipped_metro = (uint64_t*)calloc(R, sizeof(uint64_t));
    pthread_mutex_init(&o->log_mu, NULL);
    if (!o->J || !o->beta || !o->s || !o->E || (with_fields && !o->h) || !o->acc_flip ||
        !o->att_swap || !o->acc_swap || !o->near_metro || !o->first_near || !o->log || !o->adopted_metro ||
        !o->flipped_metro) {
        oracle_destroy(o);
        return NULL;
    }
    memcpy(o->J, J, sizeof(double) * L);
    o->J[0] = 0.0;
    memcpy(o->beta, beta, sizeof(double) * R);
    o->first_near_exch = -1;
    for (int t = 0; t < R; ++t) {
        o->first_near[t] = -1;
        for (int i = 0; i < L; ++i) {
            uint32_t ctr[4] = {(uint32_t)i, (uint32_t)t, 0u, ORC_TAG_INIT}, x[4];
            orc_philox(ctr, o->key, x);
            o->s[(size_t)t * L + i] = (uint8_t)(((uint64_t)x[0] * (uint64_t)q) >> 32);
        }
        o->E[t] = oracle_energy_direct(o, t);
        if (o->h) orc_fields_direct(o, t);
    }
    return o;
}

/* one Metropolis sweep of slot t at absolute sweep index n (Eq. 8).
   mode 0: dE by the direct O(L) sum; mode 1: dE from the slot's fields. */
static void orc_sweep_slot(oracle_t* o, int t, uint32_t n, int mode)
{
    const int L = o->L, q = o->q;
    uint8_t* s = o->s + (size_t)t * L;
    double* h = o->h ? o->h + (size_t)t * q * L : NULL;
    const double beta = o->beta[t];
    for (int m = 0; m < L; ++m) {
        uint32_t ctr[4] = {(uint32_t)m, (uint32_t)t, n, o->random_sites ? ORC_TAG_SITE : ORC_TAG_METRO}, x[4];
        orc_philox(ctr, o->key, x);
        const int k = o->random_sites ? (int)(((uint64_t)x[3] * (uint64_t)L) >> 32) : m;
        const int a = s[k];
        const int b = (a + 1 + (int)(((uint64_t)x[0] * (uint64_t)(q - 1)) >> 32)) % q;
        const double u = orc_unit(x[1], x[2]);
        double dE;
        if (mode == 0) {
            /* dE = c * sum_{j != k} J*(|k-j|) [delta(a, s_j) - delta(b, s_j)] */
            double sum = 0.0;
            for (int j = 0; j < L; ++j) {
                if (j == k) continue;
                if (s[j] == a) sum += orc_J(o, k, j);
                if (s[j] == b) sum -= orc_J(o, k, j);
            }
            dE = (double)o->c * sum;
        } else {
            dE = (double)o->c * (h[(size_t)a * L + k] - h[(size_t)b * L + k]);
        }
        int accept;
        const double xarg = beta * dE;
        if (dE <= 0.0) accept = 1;
        else accept = u < exp(-xarg);
        if (xarg < 40.0 && fabs(xarg + log(u)) < ORC_NEAR_TIE) {
            o->near_metro[t]++;
            if (o->first_near[t] < 0) o->first_near[t] = (int64_t)n;
            const int own = accept;
            const int ov = orc_override(o, 0, t, n, m);
            if (ov >= 0) {
                o->adopted_metro[t]++;
                if (ov != own) o->flipped_metro[t]++;
                accept = ov;
            }
            orc_log(o, 0, t, n, m, own, accept);
        }
        if (!accept) continue;
        s[k] = (uint8_t)b;
        o->E[t] += dE;
        o->acc_flip[t]++;
        if (h) {
            for (int i = 0; i < L; ++i) {
                const double Jik = orc_J(o, i, k); /* J[0] = 0 leaves i = k alone */
                h[(size_t)a * L + i] -= Jik;
                h[(size_t)b * L + i] += Jik;
            }
        }
    }
}

typedef struct {
    oracle_t* o;
    int first, stride, mode;
    uint32_t n;
} orc_job_t;

static void* orc_sweep_worker(void* arg)
{
    orc_job_t* job = (orc_job_t*)arg;
    for (int t = job->first; t < job->o->R; t += job->stride)
        orc_sweep_slot(job->o, t, job->n, job->mode);
    return NULL;
}

/* nsweeps sweeps of every slot; slots are independent within a sweep, so
   they may be spread over nthreads POSIX threads. */
int oracle_sweep(oracle_t* o, int nsweeps, int mode, int nthreads)
{
    if (mode == 1 && !o->h) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > o->R) nthreads = o->R;
    for (int it = 0; it < nsweeps; ++it) {
        const uint32_t n = o->nsweep;
        if (nthreads == 1) {
            for (int t = 0; t < o->R; ++t) orc_sweep_slot(o, t, n, mode);
        } else {
            pthread_t th[256];
            orc_job_t jobs[256];
            if (nthreads > 256) nthreads = 256;
            for (int w = 0; w < nthreads; ++w) {
                jobs[w].o = o; jobs[w].first = w; jobs[w].stride = nthreads;
                jobs[w].mode = mode; jobs[w].n = n;
                if (pthread_create(&th[w], NULL, orc_sweep_worker, &jobs[w]) != 0) return -2;
            }
            for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
        }
        o->nsweep++;
    }
    return 0;
}

static void orc_swap_slots(oracle_t* o, int t)
{
    const int L = o->L;
    uint8_t* s0 = o->s + (size_t)t * L;
    uint8_t* s1 = s0 + L;
    for (int i = 0; i < L; ++i) { uint8_t v = s0[i]; s0[i] = s1[i]; s1[i] = v; }
    double e = o->E[t]; o->E[t] = o->E[t + 1]; o->E[t + 1] = e;
    if (o->h) {
        const size_t n = (size_t)o->q * L;
        double* h0 = o->h + (size_t)t * n;
        double* h1 = h0 + n;
        for (size_t i = 0; i < n; ++i) { double v = h0[i]; h0[i] = h1[i]; h1[i] = v; }
    }
}

/* one exchange step: stage 0 (t even), then stage 1 (t odd), Eq. 9 */
void oracle_exchange(oracle_t* o)
{
    const uint32_t m = o->nexch;
    for (int stage = 0; stage < 2; ++stage) {
        for (int t = stage; t + 1 < o->R; t += 2) {
            uint32_t ctr[4] = {(uint32_t)t, (uint32_t)stage, m, ORC_TAG_EXCH}, x[4];
            orc_philox(ctr, o->key, x);
            const double u = orc_unit(x[1], x[2]);
            const double D = (o->beta[t] - o->beta[t + 1]) * (o->E[t] - o->E[t + 1]);
            int accept;
            if (D >= 0.0) accept = 1;
            else accept = u < exp(D);
            if (D > -40.0 && fabs(D - log(u)) < ORC_NEAR_TIE) {
                o->near_exch++;
                if (o->first_near_exch < 0) o->first_near_exch = (int64_t)m;
                const int own = accept;
                const int ov = orc_override(o, 1, t, m, stage);
                if (ov >= 0) {
                    o->adopted_exch++;
                    if (ov != own) o->flipped_exch++;
                    accept = ov;
                }
                orc_log(o, 1, t, m, stage, own, accept);
            }
            o->att_swap[t]++;
            if (accept) {
                o->acc_swap[t]++;
                orc_swap_slots(o, t);
            }
        }
    }
    o->nexch++;
}

/* ---- accessors ---- */
void oracle_get_spins(const oracle_t* o, uint8_t* out) { memcpy(out, o->s, (size_t)o->R * o->L); }
void oracle_set_spins(oracle_t* o, const uint8_t* in)
{
    memcpy(o->s, in, (size_t)o->R * o->L);
    for (int t = 0; t < o->R; ++t) {
        o->E[t] = oracle_energy_direct(o, t);
        if (o->h) orc_fields_direct(o, t);
    }
}
void oracle_get_running_energy(const oracle_t* o, double* out) { memcpy(out, o->E, sizeof(double) * o->R); }
void oracle_get_fields(const oracle_t* o, double* out)
{
    if (o->h) memcpy(out, o->h, sizeof(double) * (size_t)o->R * o->q * o->L);
}
void oracle_set_counters(oracle_t* o, uint32_t nsweep, uint32_t nexch) { o->nsweep = nsweep; o->nexch = nexch; }
void oracle_set_random_sites(oracle_t* o, int on) { o->random_sites = on ? 1 : 0; }
void oracle_get_counters(const oracle_t* o, uint32_t* nsweep, uint32_t* nexch)
{
    *nsweep = o->nsweep;
    *nexch = o->nexch;
}
/* per-slot accepted flips, per-pair attempted/accepted swaps, near ties */
void oracle_get_stats(const oracle_t* o, uint64_t* acc_flip, uint64_t* att_swap, uint64_t* acc_swap,
                      uint64_t* near_metro, int64_t* first_near, uint64_t* near_exch, int64_t* first_near_exch)
{
    memcpy(acc_flip, o->acc_flip, sizeof(uint64_t) * o->R);
    memcpy(att_swap, o->att_swap, sizeof(uint64_t) * o->R);
    memcpy(acc_swap, o->acc_swap, sizeof(uint64_t) * o->R);
    memcpy(near_metro, o->near_metro, sizeof(uint64_t) * o->R);
    memcpy(first_near, o->first_near, sizeof(int64_t) * o->R);
    *near_exch = o->near_exch;
    *first_near_exch = o->first_near_exch;
}

/* Replace the table of decisions to adopt at near ties: n entries of
   {kind (0 Metropolis, 1 exchange), slot t (exchange: pair (t, t+1)), sweep n
   (exchange: index m), attempt within the sweep (exchange: stage), decision
   (0 reject, 1 accept)}.  Returns 0, or -1 if the copy cannot be allocated. */
int oracle_set_overrides(oracle_t* o, const int32_t* ev, int n)
{
    int32_t* copy = NULL;
    if (n > 0) {
        copy = (int32_t*)malloc(sizeof(int32_t) * 5 * (size_t)n);
        if (!copy) return -1;
        memcpy(copy, ev, sizeof(int32_t) * 5 * (size_t)n);
    }
    free(o->ovr);
    o->ovr = copy;
    o->novr = n > 0 ? n : 0;
    return 0;
}

/* Near-tie events so far (up to cap of them, [cap][6] as in oracle_t.log);
   returns how many were seen in all. */
uint64_t oracle_get_near_log(const oracle_t* o, int32_t* out, int cap)
{
    uint64_t keep = o->nlog < ORC_LOG_CAP ? o->nlog : ORC_LOG_CAP;
    if (cap >= 0 && keep > (uint64_t)cap) keep = (uint64_t)cap;
    if (keep) memcpy(out, o->log, sizeof(int32_t) * 6 * (size_t)keep);
    return o->nlog;
}

/* adoptions of tabled decisions: per slot (Metropolis) and for the exchange,
   all of them and those that reversed the oracle's own decision */
void oracle_get_adopted(const oracle_t* o, uint64_t* adopted_metro, uint64_t* flipped_metro, uint64_t* adopted_exch,
                        uint64_t* flipped_exch)
{
    memcpy(adopted_metro, o->adopted_metro, sizeof(uint64_t) * o->R);
    memcpy(flipped_metro, o->flipped_metro, sizeof(uint64_t) * o->R);
    *adopted_exch = o->adopted_exch;
    *flipped_exch = o->flipped_exch;
}
