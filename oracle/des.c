/*
 * des.c -- discrete-event simulation of a tiny PAAM system.
 *
 * TEST INFRASTRUCTURE ONLY.  It simulates the run-time behaviour the analysis
 * of Sec. IV-F claims to bound, in unit time steps, so that a test can check
 * "bound >= every observed response" on exhaustively enumerated release
 * offsets.  It knows nothing of Eqs. 1-6.
 *
 * Simulated rules
 *   - chains release jobs periodically (offset + k T); a job runs its
 *     callbacks in order; a new job of a chain waits for the previous one;
 *   - executors are single-threaded and non-preemptive: an idle executor
 *     dispatches the ready callback of highest chain priority, which then
 *     holds it until it completes (Sec. II-C, PiCAS);
 *   - executors on one core are scheduled preemptively by executor priority;
 *     an executor wants the core while it runs CPU work, while it spins on
 *     an accelerator request, or while it is idle with a ready callback;
 *   - a callback with eta segments runs its CPU time E split into eta + 1
 *     parts around the segments; each segment is a request to the accelerator
 *     server followed by eps units of client-side CPU overhead (Sec. IV-F);
 *   - each accelerator has its own server (R1); a server maps the chains
 *     using its accelerator into n buckets by descending priority, evenly
 *     (R2); within a bucket requests run non-preemptively in chain-priority
 *     order (R3); a higher bucket preempts a lower one (R4); a request
 *     occupies its accelerator for A + 2 kappa units (preemption cost charged
 *     in full);
 *   - a spinning client occupies its core while its request is handled; a
 *     suspending one releases the core but still holds its executor.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define DES_MAXN 8
#define DES_MAXCB 32
#define DES_MAXSEG 64
#define DES_MAXX 8
#define DES_MAXJOBS 64
#define DES_MAXACC 4

enum { PH_NONE = 0, PH_READY, PH_CPU, PH_ACCEL, PH_EPS };

typedef struct {
    /* static */
    int64_t T, prio, spin, exec, bucket[DES_MAXACC];
    int32_t cb_lo, cb_n;
    /* dynamic */
    int64_t next_rel;
    int64_t queue[DES_MAXJOBS];
    int32_t qh, qt;
    int32_t active;     /* a job is in progress */
    int64_t rel;        /* its release */
    int32_t cb;         /* current callback (local index) */
    int32_t part;       /* CPU part index within the callback */
    int32_t phase;
    int64_t rem;        /* remaining units of the current CPU / eps phase */
    int64_t acc_rem;    /* remaining accelerator units of the current request */
    int32_t acc_started;
    int32_t req_acc;    /* the accelerator of the current request */
} sim_chain;

typedef struct {
    int32_t n, nx, n_buckets;
    int64_t eps, kappa;
    const int64_t *E;   /* per callback (simulated execution time) */
    const int32_t *nseg;
    const int32_t *seg_lo;
    const int64_t *A;   /* per segment (simulated execution time) */
    const int32_t *acc; /* per segment: its accelerator */
    int32_t n_acc;
    const int32_t *exec_core, *exec_prio;
    sim_chain ch[DES_MAXN];
    int32_t busy[DES_MAXX]; /* chain holding the executor, -1 idle */
} sim_t;

/* CPU part j of a callback with CPU time e split into k + 1 parts */
static int64_t cpu_part(int64_t e, int32_t k, int32_t j)
{
    return (e * (j + 1)) / (k + 1) - (e * j) / (k + 1);
}

static int wants_cpu(const sim_t *s, int32_t x)
{
    int32_t c = s->busy[x];
    if (c >= 0) {
        const sim_chain *h = &s->ch[c];
        if (h->phase == PH_CPU || h->phase == PH_EPS) return 1;
        if (h->phase == PH_ACCEL && h->spin) return 1;
        return 0;
    }
    for (int32_t k = 0; k < s->n; ++k)
        if (s->ch[k].exec == x && s->ch[k].active && s->ch[k].phase == PH_READY) return 1;
    return 0;
}

/* running executor of a core: highest executor priority wanting the core */
static int32_t core_runner(const sim_t *s, int32_t core)
{
    int32_t best = -1;
    for (int32_t x = 0; x < s->nx; ++x) {
        if (s->exec_core[x] != core || !wants_cpu(s, x)) continue;
        if (best < 0 || s->exec_prio[x] > s->exec_prio[best]) best = x;
    }
    return best;
}

/* the request accelerator u currently serves, or -1 */
static int32_t accel_pick(sim_t *s, int32_t u)
{
#define WAITS(c) (s->ch[c].active && s->ch[c].phase == PH_ACCEL && s->ch[c].req_acc == u)
    int64_t best_b = INT64_MAX;
    for (int32_t c = 0; c < s->n; ++c)
        if (WAITS(c) && s->ch[c].bucket[u] < best_b) best_b = s->ch[c].bucket[u];
    if (best_b == INT64_MAX) return -1;
    for (int32_t c = 0; c < s->n; ++c) /* an in-progress request keeps its bucket's worker */
        if (WAITS(c) && s->ch[c].bucket[u] == best_b && s->ch[c].acc_started) return c;
    int32_t pick = -1;
    for (int32_t c = 0; c < s->n; ++c)
        if (WAITS(c) && s->ch[c].bucket[u] == best_b && (pick < 0 || s->ch[c].prio > s->ch[pick].prio))
            pick = c;
    s->ch[pick].acc_started = 1;
    return pick;
#undef WAITS
}

/* move chain c past any finished phase; returns 1 if something changed */
static int advance(sim_t *s, int32_t c, int64_t now, int64_t *max_resp)
{
    sim_chain *h = &s->ch[c];
    int changed = 0;
    for (;;) {
        if (!h->active) {
            if (h->qh == h->qt) return changed;
            h->rel = h->queue[h->qh++];
            h->active = 1;
            h->cb = 0;
            h->phase = h->cb_n > 0 ? PH_READY : PH_NONE;
            changed = 1;
            if (h->cb_n == 0) { /* empty chain completes at once */
                int64_t r = now - h->rel;
                if (r > max_resp[c]) max_resp[c] = r;
                h->active = 0;
            }
            continue;
        }
        const int32_t cbg = h->cb_lo + h->cb;
        if (h->phase == PH_CPU && h->rem == 0) {
            if (h->part < s->nseg[cbg]) { /* next: accelerator request of segment `part` */
                h->phase = PH_ACCEL;
                h->acc_rem = s->A[s->seg_lo[cbg] + h->part] + 2 * s->kappa;
                h->req_acc = s->acc ? s->acc[s->seg_lo[cbg] + h->part] : 0;
                h->acc_started = 0;
            } else { /* callback done */
                s->busy[h->exec] = -1;
                h->cb += 1;
                if (h->cb < h->cb_n) {
                    h->phase = PH_READY;
                } else {
                    int64_t r = now - h->rel;
                    if (r > max_resp[c]) max_resp[c] = r;
                    h->active = 0;
                    h->phase = PH_NONE;
                }
            }
            changed = 1;
            continue;
        }
        if (h->phase == PH_ACCEL && h->acc_rem == 0) {
            h->phase = PH_EPS;
            h->rem = s->eps;
            h->acc_started = 0;
            changed = 1;
            continue;
        }
        if (h->phase == PH_EPS && h->rem == 0) {
            h->part += 1;
            h->phase = PH_CPU;
            h->rem = cpu_part(s->E[cbg], s->nseg[cbg], h->part);
            changed = 1;
            continue;
        }
        return changed;
    }
}

static void dispatch(sim_t *s, int32_t x)
{
    int32_t pick = -1;
    for (int32_t k = 0; k < s->n; ++k)
        if (s->ch[k].exec == x && s->ch[k].active && s->ch[k].phase == PH_READY &&
            (pick < 0 || s->ch[k].prio > s->ch[pick].prio))
            pick = k;
    if (pick < 0) return;
    sim_chain *h = &s->ch[pick];
    const int32_t cbg = h->cb_lo + h->cb;
    s->busy[x] = pick;
    h->part = 0;
    h->phase = PH_CPU;
    h->rem = cpu_part(s->E[cbg], s->nseg[cbg], 0);
}

/*
 * One simulation run with fixed offsets.  Jobs are released at
 * offset_c + k T_c < rel_end; the run continues until every released job
 * has completed or t reaches t_limit (then the unfinished jobs report
 * t_limit - release).  max_resp[c] is raised to the largest response seen.
 * Returns 0, or -1 if a chain's job queue overflowed.
 */
static int run_once(sim_t *s, const int64_t *offset, int64_t rel_end, int64_t t_limit,
                    int64_t *max_resp)
{
    int32_t n_cores = 0;
    for (int32_t x = 0; x < s->nx; ++x)
        if (s->exec_core[x] + 1 > n_cores) n_cores = s->exec_core[x] + 1;
    for (int32_t c = 0; c < s->n; ++c) {
        sim_chain *h = &s->ch[c];
        h->next_rel = offset[c];
        h->qh = h->qt = 0;
        h->active = 0;
        h->phase = PH_NONE;
        h->rem = h->acc_rem = 0;
        h->acc_started = 0;
    }
    for (int32_t x = 0; x < s->nx; ++x) s->busy[x] = -1;

    for (int64_t t = 0; t < t_limit; ++t) {
        /* releases */
        int pending = 0;
        for (int32_t c = 0; c < s->n; ++c) {
            sim_chain *h = &s->ch[c];
            if (h->next_rel == t && t < rel_end) {
                if (h->qt >= DES_MAXJOBS) return -1;
                h->queue[h->qt++] = t;
                h->next_rel += h->T;
            }
        }
        /* zero-time transitions until stable */
        for (int guard = 0; guard < 10000; ++guard) {
            int changed = 0;
            for (int32_t c = 0; c < s->n; ++c) changed |= advance(s, c, t, max_resp);
            for (int32_t core = 0; core < n_cores; ++core) {
                int32_t x = core_runner(s, core);
                if (x >= 0 && s->busy[x] < 0) {
                    dispatch(s, x);
                    changed = 1;
                }
            }
            for (int32_t u = 0; u < s->n_acc; ++u) {
                int32_t a = accel_pick(s, u);
                if (a >= 0 && s->ch[a].acc_rem == 0) changed |= advance(s, a, t, max_resp);
            }
            if (!changed) break;
        }
        for (int32_t c = 0; c < s->n; ++c)
            if (s->ch[c].active || s->ch[c].qh != s->ch[c].qt || s->ch[c].next_rel < rel_end) pending = 1;
        if (!pending) return 0;
        /* one unit of execution */
        for (int32_t core = 0; core < n_cores; ++core) {
            int32_t x = core_runner(s, core);
            if (x < 0) continue;
            if (s->busy[x] < 0) continue;
            sim_chain *h = &s->ch[s->busy[x]];
            if ((h->phase == PH_CPU || h->phase == PH_EPS) && h->rem > 0) h->rem -= 1;
            /* a spinning client burns the unit without progress */
        }
        for (int32_t u = 0; u < s->n_acc; ++u) { /* each accelerator serves its own requests */
            int32_t a = accel_pick(s, u);
            if (a >= 0 && s->ch[a].acc_rem > 0) s->ch[a].acc_rem -= 1;
        }
    }
    for (int32_t c = 0; c < s->n; ++c) { /* unfinished work: report at least the elapsed time */
        sim_chain *h = &s->ch[c];
        if (h->active && t_limit - h->rel > max_resp[c]) max_resp[c] = t_limit - h->rel;
        for (int32_t q = h->qh; q < h->qt; ++q)
            if (t_limit - h->queue[q] > max_resp[c]) max_resp[c] = t_limit - h->queue[q];
    }
    return 0;
}

/*
 * Explore one tiny system: every release-offset vector on the integer grid
 * (offset_c in [0, T_c)), for each execution-time variant: all WCETs, then
 * each callback CPU time and each segment time in turn replaced by the
 * variant value floor(x / 2).  Jobs are released during
 * max_offset + 2 * hyperperiod; the run may continue to t_limit_extra
 * beyond that to let them finish.  max_resp[c] receives the largest
 * response observed per chain.  Returns 0, or a negative code.
 *
 * Per-chain inputs: T, prio, exec, spin, cb_n (callbacks).  Per callback (in
 * chain order): E, nseg.  Per segment: A.  Executors: core, priority.
 */
int des_explore(int32_t n, const int64_t *T, const int32_t *prio, const int32_t *exec,
                const uint8_t *spin, const int32_t *cb_n, const int64_t *E, const int32_t *nseg,
                const int64_t *A, const int32_t *acc, int32_t nx, const int32_t *exec_core, const int32_t *exec_prio,
                int32_t n_buckets, int64_t eps, int64_t kappa, int64_t t_limit_extra,
                int32_t all_variants, int64_t *max_resp)
{
    if (n < 1 || n > DES_MAXN || nx < 1 || nx > DES_MAXX) return -2;
    sim_t s;
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.nx = nx;
    s.n_buckets = n_buckets;
    s.eps = eps;
    s.kappa = kappa;
    s.exec_core = exec_core;
    s.exec_prio = exec_prio;
    int32_t seg_lo[DES_MAXCB];
    int32_t ncb = 0, nsg = 0;
    int64_t segs_of[DES_MAXN];
    for (int32_t c = 0; c < n; ++c) {
        s.ch[c].T = T[c];
        s.ch[c].prio = prio[c];
        s.ch[c].spin = spin[c];
        s.ch[c].exec = exec[c];
        s.ch[c].cb_lo = ncb;
        s.ch[c].cb_n = cb_n[c];
        segs_of[c] = 0;
        for (int32_t j = 0; j < cb_n[c]; ++j) {
            if (ncb >= DES_MAXCB) return -2;
            seg_lo[ncb] = nsg;
            nsg += nseg[ncb];
            segs_of[c] += nseg[ncb];
            ncb += 1;
        }
    }
    if (nsg > DES_MAXSEG) return -2;
    s.acc = acc;
    s.n_acc = 1;
    for (int32_t q = 0; acc && q < nsg; ++q) {
        if (acc[q] < 0 || acc[q] >= DES_MAXACC) return -2;
        if (acc[q] + 1 > s.n_acc) s.n_acc = acc[q] + 1;
    }
    /* rule R2 per accelerator: its users ranked by descending chain priority,
     * n evenly sized groups */
    for (int32_t u = 0; u < s.n_acc; ++u) {
        int32_t uses[DES_MAXN], users = 0;
        for (int32_t c = 0; c < n; ++c) {
            uses[c] = 0;
            for (int32_t j = s.ch[c].cb_lo; j < s.ch[c].cb_lo + s.ch[c].cb_n; ++j)
                for (int32_t q = seg_lo[j]; q < seg_lo[j] + nseg[j]; ++q) uses[c] |= (acc ? acc[q] : 0) == u;
            users += uses[c];
        }
        for (int32_t c = 0; c < n; ++c) {
            int32_t r = 0;
            for (int32_t k = 0; k < n; ++k)
                if (uses[k] && prio[k] > prio[c]) r += 1;
            s.ch[c].bucket[u] = uses[c] ? ((int64_t)r * n_buckets) / users : INT64_MAX;
        }
    }
    (void)segs_of;
    int64_t Ev[DES_MAXCB], Av[DES_MAXSEG];
    s.E = Ev;
    s.A = Av;
    s.nseg = nseg;
    s.seg_lo = seg_lo;

    int64_t hyper = 1, tmax = 0;
    for (int32_t c = 0; c < n; ++c) {
        int64_t a = hyper, b = T[c];
        while (b) {
            int64_t r = a % b;
            a = b;
            b = r;
        }
        hyper = hyper / a * T[c];
        if (T[c] > tmax) tmax = T[c];
    }
    const int64_t rel_end = tmax + 2 * hyper;
    const int64_t t_limit = rel_end + t_limit_extra;
    for (int32_t c = 0; c < n; ++c) max_resp[c] = 0;

    const int32_t n_var = all_variants ? 1 + ncb + nsg : 1;
    int64_t off[DES_MAXN];
    for (int32_t v = 0; v < n_var; ++v) {
        for (int32_t j = 0; j < ncb; ++j) Ev[j] = E[j];
        for (int32_t q = 0; q < nsg; ++q) Av[q] = A[q];
        if (v >= 1 && v <= ncb) Ev[v - 1] = E[v - 1] / 2;
        if (v > ncb) Av[v - 1 - ncb] = A[v - 1 - ncb] / 2;
        for (int32_t c = 0; c < n; ++c) off[c] = 0;
        for (;;) {
            if (run_once(&s, off, rel_end, t_limit, max_resp) < 0) return -3;
            int32_t c = 0;
            while (c < n) {
                off[c] += 1;
                if (off[c] < T[c]) break;
                off[c] = 0;
                c += 1;
            }
            if (c == n) break;
        }
    }
    return 0;
}
