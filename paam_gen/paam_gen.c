/*
 * paam_gen.c -- seeded synthetic ROS 2 system generator.
 *
 * This module produces INPUTS only: chain periods, deadlines, priorities,
 * executor placement, callback WCETs and accelerator-segment WCETs.  It holds
 * none of the response-time analysis arithmetic; both the CPU oracle and the
 * CUDA path consume what it writes.
 *
 * The workload shape follows the analytical study of Sec. V-D (callbacks per
 * chain, one accelerator, random periods, chain utilisation split equally
 * over its callbacks) and the system model of Sec. II-C (chains of
 * callbacks, each callback with a CPU WCET and zero or more accelerator
 * segments; chains on single-threaded executors pinned to cores).
 *
 * Randomness: every system i draws from two private xoshiro256** streams
 * (structure and values) seeded through SplitMix64 from (seed, i, stream),
 * so the output is bit-identical however the index range is split over
 * threads.
 */
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int64_t n_sys;
    uint64_t seed;
    int32_t n_min, n_max;     /* chains per system, inclusive                   */
    double n_geom_p;          /* > 0: N = n_min + Geom(p) clipped to n_max       */
    int32_t cb_min, cb_max;   /* callbacks per chain, uniform inclusive          */
    int32_t x_min, x_max;     /* executors per system, uniform inclusive         */
    int32_t exec_per_core;    /* executor k runs on core k / exec_per_core       */
    int32_t util_mode;        /* 0: U ~ Unif[util_lo, util_hi]; 1: sweep         */
    double util_lo, util_hi;  /* sweep: U = util_lo + util_step * (i mod util_n) */
    double util_step;
    int32_t util_n;
    int32_t seg_per_cb;       /* segment slots per callback, each Bernoulli(p)   */
    double p_acc;
    int64_t a_min, a_max;     /* accelerator segment WCET, uniform inclusive, ns */
    double t_min, t_max;      /* chain period, log-uniform, ns                   */
    double d_lo, d_hi;        /* D = floor(T * Unif[d_lo, d_hi]), at least 1     */
    double p_spin;            /* probability that a chain busy-waits             */
    int32_t exec_prio_mode;   /* 0: CAPA (max chain priority on the executor)    */
                              /* 1: random distinct executor priorities          */
    int32_t pad_;
} paam_gen_params;

typedef struct {
    uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_init(rng_t *r, uint64_t seed, uint64_t idx, uint64_t stream)
{
    uint64_t x = seed ^ (idx * 0xD1B54A32D192ED03ULL) ^ ((stream + 1) * 0x8CB92BA72F3D8DD7ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* uniform double in [0, 1) with 53 random bits */
static double unif01(rng_t *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [lo, hi] (multiply-high range reduction) */
static int64_t unif_int(rng_t *r, int64_t lo, int64_t hi)
{
    uint64_t n = (uint64_t)(hi - lo) + 1u;
    if (n == 0) return lo + (int64_t)rng_next(r); /* full 64-bit range */
    return lo + (int64_t)(uint64_t)(((__uint128_t)rng_next(r) * n) >> 64);
}

/* ---- structure of one system: counts drawn from stream 0 --------------- */

#define GEN_MAX_CHAINS 4096
#define GEN_MAX_CB (1 << 18)

typedef struct {
    int32_t n_chain, n_exec;
    int32_t n_cb, n_seg;
} sys_counts;

/* Draws the structure of system i.  When cb_per_chain / seg_per_cb_out are
 * non-NULL the per-chain callback counts and per-callback segment counts are
 * written there (in chain order). */
static sys_counts draw_structure(const paam_gen_params *p, int64_t i, int32_t *cb_per_chain,
                                 int32_t *seg_per_cb_out)
{
    rng_t r;
    rng_init(&r, p->seed, (uint64_t)i, 0);
    sys_counts k;
    int32_t n;
    if (p->n_geom_p > 0.0) {
        n = p->n_min;
        while (n < p->n_max && unif01(&r) >= p->n_geom_p) ++n;
    } else {
        n = (int32_t)unif_int(&r, p->n_min, p->n_max);
    }
    k.n_chain = n;
    k.n_exec = (int32_t)unif_int(&r, p->x_min, p->x_max);
    k.n_cb = 0;
    k.n_seg = 0;
    for (int32_t c = 0; c < n; ++c) {
        int32_t ncb = (int32_t)unif_int(&r, p->cb_min, p->cb_max);
        if (cb_per_chain) cb_per_chain[c] = ncb;
        for (int32_t j = 0; j < ncb; ++j) {
            int32_t ns = 0;
            for (int32_t q = 0; q < p->seg_per_cb; ++q) ns += (unif01(&r) < p->p_acc) ? 1 : 0;
            if (seg_per_cb_out) seg_per_cb_out[k.n_cb] = ns;
            k.n_cb += 1;
            k.n_seg += ns;
        }
    }
    return k;
}

/* Per-system counts for systems [lo, hi). */
void paam_gen_count(const paam_gen_params *p, int64_t lo, int64_t hi, int32_t *n_chain,
                    int32_t *n_cb, int32_t *n_seg, int32_t *n_exec)
{
    for (int64_t i = lo; i < hi; ++i) {
        sys_counts k = draw_structure(p, i, NULL, NULL);
        n_chain[i] = k.n_chain;
        n_cb[i] = k.n_cb;
        n_seg[i] = k.n_seg;
        n_exec[i] = k.n_exec;
    }
}

/*
 * Fills systems [lo, hi).  sys_chain_off / sys_exec_off / sys_cb_start /
 * sys_seg_start are the exclusive prefix sums of the counts (computed by the
 * caller); the closing sentinels of chain_cb_off and cb_seg_off are written
 * by the caller too.
 */
void paam_gen_fill(const paam_gen_params *p, int64_t lo, int64_t hi, const int64_t *sys_chain_off,
                   const int64_t *sys_exec_off, const int64_t *sys_cb_start,
                   const int64_t *sys_seg_start, int64_t *chain_cb_off, int64_t *cb_seg_off,
                   int64_t *T, int64_t *D, int32_t *prio, int32_t *exec, uint8_t *spin, int64_t *E,
                   int64_t *A, int32_t *acc, int32_t *exec_core, int32_t *exec_prio)
{
    static __thread int32_t cb_per_chain[GEN_MAX_CHAINS];
    static __thread int32_t perm[GEN_MAX_CHAINS];
    static __thread double util[GEN_MAX_CHAINS];
    static __thread int32_t seg_cnt[GEN_MAX_CB];
    const double lt0 = log(p->t_min), lt1 = log(p->t_max);
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t c0 = sys_chain_off[i], x0 = sys_exec_off[i];
        const int64_t cb0 = sys_cb_start[i], s0 = sys_seg_start[i];
        sys_counts k = draw_structure(p, i, cb_per_chain, seg_cnt);
        {
            int64_t cb = cb0, seg = s0;
            for (int32_t c = 0; c < k.n_chain; ++c) {
                chain_cb_off[c0 + c] = cb;
                for (int32_t j = 0; j < cb_per_chain[c]; ++j) {
                    cb_seg_off[cb] = seg;
                    seg += seg_cnt[cb - cb0];
                    cb += 1;
                }
            }
        }
        const int32_t n = k.n_chain, nx = k.n_exec;

        rng_t r;
        rng_init(&r, p->seed, (uint64_t)i, 1);
        /* total CPU utilisation of the system */
        double U;
        if (p->util_mode == 1)
            U = p->util_lo + p->util_step * (double)(i % (int64_t)(p->util_n > 0 ? p->util_n : 1));
        else
            U = p->util_lo + (p->util_hi - p->util_lo) * unif01(&r);
        /* UUniFast split of U over the n chains */
        {
            double sum = U;
            for (int32_t c = 0; c < n - 1; ++c) {
                double next = sum * pow(unif01(&r), 1.0 / (double)(n - 1 - c));
                util[c] = sum - next;
                sum = next;
            }
            if (n > 0) util[n - 1] = sum;
        }
        /* periods (log-uniform) and deadlines */
        for (int32_t c = 0; c < n; ++c) {
            double t = exp(lt0 + (lt1 - lt0) * unif01(&r));
            int64_t Tc = (int64_t)llround(t);
            if (Tc < 1) Tc = 1;
            T[c0 + c] = Tc;
            int64_t Dc = Tc;
            if (!(p->d_lo == 1.0 && p->d_hi == 1.0)) {
                double f = p->d_lo + (p->d_hi - p->d_lo) * unif01(&r);
                Dc = (int64_t)floor((double)Tc * f);
                if (Dc < 1) Dc = 1;
                if (Dc > Tc) Dc = Tc;
            }
            D[c0 + c] = Dc;
        }
        /* distinct chain priorities: a random permutation of 0..n-1 */
        for (int32_t c = 0; c < n; ++c) perm[c] = c;
        for (int32_t c = n - 1; c > 0; --c) {
            int32_t j = (int32_t)unif_int(&r, 0, c);
            int32_t t = perm[c];
            perm[c] = perm[j];
            perm[j] = t;
        }
        for (int32_t c = 0; c < n; ++c) prio[c0 + c] = perm[c];
        /* executor placement and spin / suspend behaviour */
        for (int32_t c = 0; c < n; ++c) exec[c0 + c] = (int32_t)unif_int(&r, 0, nx - 1);
        for (int32_t c = 0; c < n; ++c) spin[c0 + c] = (unif01(&r) < p->p_spin) ? 1 : 0;
        /* callback CPU WCETs: chain utilisation split equally over callbacks */
        for (int32_t c = 0; c < n; ++c) {
            int64_t cbs = chain_cb_off[c0 + c];
            int32_t ncb = cb_per_chain[c];
            int64_t e = 0;
            if (ncb > 0) {
                double v = floor(util[c] * (double)T[c0 + c] / (double)ncb);
                e = v < 0.0 ? 0 : (int64_t)v;
            }
            for (int32_t j = 0; j < ncb; ++j) E[cbs + j] = e;
        }
        /* accelerator segment WCETs (single accelerator, index 0) */
        for (int64_t q = s0; q < s0 + k.n_seg; ++q) {
            A[q] = unif_int(&r, p->a_min, p->a_max);
            acc[q] = 0;
        }
        /* executors: cores and priorities */
        for (int32_t x = 0; x < nx; ++x) exec_core[x0 + x] = x / (p->exec_per_core > 0 ? p->exec_per_core : 1);
        if (p->exec_prio_mode == 1) {
            for (int32_t x = 0; x < nx; ++x) perm[x] = x;
            for (int32_t x = nx - 1; x > 0; --x) {
                int32_t j = (int32_t)unif_int(&r, 0, x);
                int32_t t = perm[x];
                perm[x] = perm[j];
                perm[j] = t;
            }
            for (int32_t x = 0; x < nx; ++x) exec_prio[x0 + x] = perm[x];
        } else {
            for (int32_t x = 0; x < nx; ++x) exec_prio[x0 + x] = -(x + 1);
            for (int32_t c = 0; c < n; ++c) {
                int32_t x = exec[c0 + c];
                if (prio[c0 + c] > exec_prio[x0 + x]) exec_prio[x0 + x] = prio[c0 + c];
            }
        }
    }
}

/* Fisher-Yates permutations for the priority-assignment search: candidate
 * slot k of system i is a permutation of 0..n_i-1 drawn from stream 2 + k.
 * out is [hi-lo][K][nmax]; slots < first_slot are left untouched and
 * entries past n_i are set to -1. */
void paam_gen_perms(uint64_t seed, int64_t lo, int64_t hi, int32_t K, int32_t first_slot,
                    const int32_t *n_of_sys, int32_t nmax, int16_t *out)
{
    for (int64_t i = lo; i < hi; ++i) {
        const int32_t n = n_of_sys[i];
        for (int32_t k = first_slot; k < K; ++k) {
            int16_t *o = out + ((i - lo) * (int64_t)K + k) * nmax;
            rng_t r;
            rng_init(&r, seed, (uint64_t)i, 2 + (uint64_t)k);
            for (int32_t c = 0; c < nmax; ++c) o[c] = (int16_t)(c < n ? c : -1);
            for (int32_t c = n - 1; c > 0; --c) {
                int32_t j = (int32_t)unif_int(&r, 0, c);
                int16_t t = o[c];
                o[c] = o[j];
                o[j] = t;
            }
        }
    }
}

/* Assignment of accelerator segments to n_units units of the accelerator,
 * per system, by worst-fit decreasing (the bin-packing heuristic the PAAM
 * server applies at client registration): segments in decreasing order of
 * utilisation A / T of their chain (ties: lower segment index first), each to
 * the unit with the least utilisation so far (ties: the lower unit).  Writes
 * acc[q] for the segments of systems [lo, hi).  n_units <= 64. */
void paam_gen_assign_wfd(int64_t lo, int64_t hi, const int64_t *sys_chain_off, const int64_t *chain_cb_off,
                         const int64_t *cb_seg_off, const int64_t *T, const int64_t *A, int32_t n_units,
                         int32_t *acc)
{
    double load[64];
    for (int64_t s = lo; s < hi; ++s) {
        const int64_t c0 = sys_chain_off[s], c1 = sys_chain_off[s + 1];
        if (c1 == c0) continue;
        const int64_t q0 = cb_seg_off[chain_cb_off[c0]], q1 = cb_seg_off[chain_cb_off[c1]];
        const int64_t nq = q1 - q0;
        if (nq <= 0) continue;
        double *u = (double *)malloc((size_t)nq * sizeof(double));
        int64_t *ord = (int64_t *)malloc((size_t)nq * sizeof(int64_t));
        for (int64_t c = c0; c < c1; ++c)
            for (int64_t q = cb_seg_off[chain_cb_off[c]]; q < cb_seg_off[chain_cb_off[c + 1]]; ++q)
                u[q - q0] = (double)A[q] / (double)T[c];
        for (int64_t i = 0; i < nq; ++i) ord[i] = i;
        for (int64_t i = 1; i < nq; ++i) { /* insertion sort: decreasing u, stable */
            const int64_t x = ord[i];
            int64_t j = i;
            while (j > 0 && u[ord[j - 1]] < u[x]) {
                ord[j] = ord[j - 1];
                --j;
            }
            ord[j] = x;
        }
        for (int32_t k = 0; k < n_units; ++k) load[k] = 0.0;
        for (int64_t i = 0; i < nq; ++i) {
            int32_t best = 0;
            for (int32_t k = 1; k < n_units; ++k)
                if (load[k] < load[best]) best = k;
            load[best] += u[ord[i]];
            acc[q0 + ord[i]] = best;
        }
        free(u);
        free(ord);
    }
}
