/*
 * paam_oracle.c -- plain CPU oracle for PAAM's admission-control analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant with the CUDA path.
 *
 * It evaluates, for every chain of every system, the worst-case response-time
 * bound of Theorem 1 (Eq. 6) in the paper's own order:
 *
 *   1. per-chain aggregates of the system model (Sec. II-C): E_c, the largest
 *      callback WCET, delta_c, and A*_{i,j} = A_{i,j} + 2 kappa (Sec. IV-F);
 *   2. bucket down-sampling of accelerator-using chains (Sec. IV-C, rule R2);
 *   3. same-bucket lower-priority blocking on the accelerator (the max term
 *      shared by Eq. 3 and Eq. 4);
 *   4. CPU blocking B_c from lower-priority chains of the same executor
 *      (Lemma 4, Eq. 5);
 *   5. per-segment handling-time fixed points (Lemma 2, Eq. 3) with the
 *      arrival bound mu(t) = ceil(t / T) + 1 (Lemma 1, Eq. 2);
 *   6. the chain recurrence of Theorem 1 (Eq. 6), in which H_c is the minimum
 *      of the per-segment sum and the per-chain bound (Lemma 3, Eq. 4) and
 *      H*_c = H_c + delta_c * eps (Eq. 1).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - buckets: accelerator-using chains ranked by descending priority, rank r
 *     of |U| goes to group floor(r * n / |U|) (0 = highest bucket);
 *   - a segment fixed point whose iterate exceeds the chain's deadline makes
 *     the per-segment bound infinite (the minimum then takes Eq. 4);
 *   - the chain recurrence starts from B_c + E_c + H*_c with Eq. 4's
 *     interference part empty; the result is the least fixed point either way;
 *   - H*_h of an interfering chain is evaluated at that chain's own R_h;
 *   - a chain whose needed H*_h (same-executor higher-priority chains, and
 *     spinning chains of higher-priority executors on the core) is not
 *     schedulable gets status DEP; DEP wins over OVERRUN;
 *   - executor priorities, when not given, are the highest chain priority on
 *     the executor (criticality-as-priority, Sec. II-C).
 *
 * All times are int64 nanoseconds; there is no other rounding than the
 * ceiling of Eq. 2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ST_SCHED = 0, ST_OVERRUN = 1, ST_DEP = 2, ST_ITERCAP = 3 };

#define O_INF INT64_MAX
#define O_MAXACC 8 /* accelerators per system handled here */

/* diagnostic counters (test infrastructure): fixed-point iterations per system */
static __thread int64_t g_seg_iters, g_chain_iters, g_max_loop;
#define O_ITER_LIMIT 100000000LL /* never reached: every iteration raises some mu */

typedef struct {
    /* inputs, gathered per chain */
    int64_t T, D;
    int64_t prio;  /* chain priority: larger is higher */
    int64_t exec;  /* executor index local to the system */
    int64_t core;  /* core of that executor */
    int64_t eprio; /* priority of that executor */
    int64_t spin;  /* 1: busy-waits during accelerator requests */
    int64_t seg_lo, seg_hi;
    /* step 1 (totals over the chain's segments) */
    int64_t E, Emax, delta, S, M;
    /* steps 2-5 */
    int64_t bucket, blk, B, Hseg;
    /* the same per accelerator (rule R1: one server per accelerator, analysed
     * independently); with one accelerator, index 0 equals the fields above */
    int64_t dA[O_MAXACC], SA[O_MAXACC], MA[O_MAXACC], bucketA[O_MAXACC], blkA[O_MAXACC], HsegA[O_MAXACC];
    /* step 6 */
    int64_t R, Hstar;
    int64_t status, done;
} chain_t;

/* ceiling of t / T for t >= 0, T > 0 */
static int64_t ceil_div(int64_t t, int64_t T) { return t / T + (t % T != 0 ? 1 : 0); }

/* Lemma 1 (Eq. 2): at most ceil(t / T) + 1 arrivals in any interval t */
static int64_t mu(int64_t t, int64_t T) { return ceil_div(t, T) + 1; }

/* Eq. 4 for chain c's requests to accelerator a, evaluated at window t */
static int64_t H_chain(const chain_t *ch, int64_t n, int64_t c, int64_t a, int64_t t, int64_t *work)
{
    int64_t h = ch[c].SA[a] + ch[c].dA[a] * ch[c].blkA[a];
    for (int64_t k = 0; k < n; ++k) {
        if (ch[k].dA[a] > 0 && ch[k].prio > ch[c].prio) { /* k in hps of every segment of c on a */
            h += mu(t, ch[k].T) * ch[k].SA[a];
            if (work) *work += 1;
        }
    }
    return h;
}

/* H_c(t) = sum over the accelerators c uses of min(per-segment sum of Eq. 3,
 * Eq. 4 at t) (one accelerator: the minimum itself);
 * H*_c = H_c + delta_c eps (Eq. 1) */
static int64_t H_star(const chain_t *ch, int64_t n, int64_t c, int64_t t, int64_t eps, int64_t *work)
{
    if (ch[c].delta == 0) return 0;
    int64_t h = 0;
    for (int64_t a = 0; a < O_MAXACC; ++a) {
        if (ch[c].dA[a] == 0) continue;
        const int64_t hc = H_chain(ch, n, c, a, t, work);
        h += ch[c].HsegA[a] < hc ? ch[c].HsegA[a] : hc;
    }
    return h + ch[c].delta * eps;
}

static void analyze_system(int64_t s, const int64_t *sys_chain_off, const int64_t *chain_cb_off,
                           const int64_t *cb_seg_off, const int64_t *T, const int64_t *D,
                           const int32_t *prio, const int32_t *exec, const uint8_t *spin,
                           const int64_t *E, const int64_t *A, const int32_t *acc,
                           const int64_t *sys_exec_off, const int32_t *exec_core, const int32_t *exec_prio,
                           const int16_t *rank, int32_t n_buckets, int64_t eps, int64_t kappa,
                           int32_t blocking_mode, int64_t *R_out, uint8_t *st_out, uint8_t *verdict,
                           int64_t *aux, int64_t *work_out)
{
    const int64_t c0 = sys_chain_off[s], n = sys_chain_off[s + 1] - c0;
    const int64_t x0 = sys_exec_off[s], nx = sys_exec_off[s + 1] - x0;
    chain_t *ch = (chain_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(chain_t));
    int64_t work = 0;

    /* inputs; with a rank override (priority search) rank 0 is the highest */
    for (int64_t c = 0; c < n; ++c) {
        ch[c].T = T[c0 + c];
        ch[c].D = D[c0 + c];
        ch[c].prio = rank ? (int64_t)(n - 1 - rank[c]) : (int64_t)prio[c0 + c];
        ch[c].exec = exec[c0 + c];
        ch[c].core = exec_core[x0 + ch[c].exec];
        ch[c].spin = spin[c0 + c];
    }
    for (int64_t c = 0; c < n; ++c) {
        if (exec_prio && !rank) {
            ch[c].eprio = exec_prio[x0 + ch[c].exec];
        } else { /* criticality-as-priority: highest chain priority on the executor */
            int64_t best = INT64_MIN;
            for (int64_t k = 0; k < n; ++k)
                if (ch[k].exec == ch[c].exec && ch[k].prio > best) best = ch[k].prio;
            ch[c].eprio = best;
        }
    }
    (void)nx;

    /* step 1: system-model aggregates (Sec. II-C) and A* = A + 2 kappa (Sec. IV-F) */
    for (int64_t c = 0; c < n; ++c) {
        const int64_t cb_lo = chain_cb_off[c0 + c], cb_hi = chain_cb_off[c0 + c + 1];
        ch[c].seg_lo = cb_seg_off[cb_lo];
        ch[c].seg_hi = cb_seg_off[cb_hi];
        for (int64_t b = cb_lo; b < cb_hi; ++b) {
            ch[c].E += E[b];
            if (E[b] > ch[c].Emax) ch[c].Emax = E[b];
            for (int64_t q = cb_seg_off[b]; q < cb_seg_off[b + 1]; ++q) {
                const int64_t a_star = A[q] + 2 * kappa;
                const int64_t u = acc ? acc[q] : 0; /* the accelerator of this segment */
                ch[c].delta += 1;
                ch[c].S += a_star;
                if (a_star > ch[c].M) ch[c].M = a_star;
                ch[c].dA[u] += 1;
                ch[c].SA[u] += a_star;
                if (a_star > ch[c].MA[u]) ch[c].MA[u] = a_star;
            }
        }
    }

    /* step 2: buckets -- accelerator users split into n evenly sized groups,
     * highest priorities first (Sec. IV-C; rule R2) */
    for (int64_t a = 0; a < O_MAXACC; ++a) { /* each accelerator's server has its own buckets (R1) */
        int64_t n_users = 0;
        for (int64_t c = 0; c < n; ++c) n_users += ch[c].dA[a] > 0 ? 1 : 0;
        for (int64_t c = 0; c < n; ++c) {
            ch[c].bucketA[a] = -1;
            if (ch[c].dA[a] == 0) continue;
            int64_t r = 0;
            for (int64_t k = 0; k < n; ++k)
                if (ch[k].dA[a] > 0 && ch[k].prio > ch[c].prio) r += 1;
            ch[c].bucketA[a] = r * (int64_t)n_buckets / n_users;
        }
    }

    /* step 3: the longest request of a lower-priority chain in the same bucket
     * (rules R2-R3; the max term of Eq. 3 and Eq. 4) */
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t a = 0; a < O_MAXACC; ++a) {
            ch[c].blkA[a] = 0;
            if (ch[c].dA[a] == 0) continue;
            for (int64_t l = 0; l < n; ++l)
                if (ch[l].dA[a] > 0 && ch[l].prio < ch[c].prio && ch[l].bucketA[a] == ch[c].bucketA[a] &&
                    ch[l].MA[a] > ch[c].blkA[a])
                    ch[c].blkA[a] = ch[l].MA[a];
        }
    }

    /* step 4: non-preemptive blocking by one callback of a lower-priority chain
     * on the same executor (Lemma 4) */
    for (int64_t c = 0; c < n; ++c) {
        ch[c].B = 0;
        for (int64_t l = 0; l < n; ++l)
            if (ch[l].exec == ch[c].exec && ch[l].prio < ch[c].prio && ch[l].Emax > ch[c].B)
                ch[c].B = ch[l].Emax;
    }

    /* step 5: per-segment handling times (Lemma 2, Eq. 3); each segment's
     * bound is kept for the safe blocking term below */
    const int64_t q_sys = n > 0 ? ch[0].seg_lo : 0;
    const int64_t n_q = n > 0 ? ch[n - 1].seg_hi - q_sys : 0;
    int64_t *hq = (int64_t *)calloc((size_t)(n_q > 0 ? n_q : 1), sizeof(int64_t));
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t a = 0; a < O_MAXACC; ++a) ch[c].HsegA[a] = 0;
        for (int64_t q = ch[c].seg_lo; q < ch[c].seg_hi; ++q) {
            const int64_t a_star = A[q] + 2 * kappa;
            const int64_t u = acc ? acc[q] : 0;
            int64_t h = a_star + ch[c].blkA[u]; /* the first two terms */
            int64_t it = 0, evals = 0;
            for (;;) {
                if (h > ch[c].D) {
                    h = O_INF;
                    break;
                }
                int64_t nh = a_star + ch[c].blkA[u];
                for (int64_t k = 0; k < n; ++k) {
                    if (ch[k].dA[u] > 0 && ch[k].prio > ch[c].prio) {
                        nh += mu(h, ch[k].T) * ch[k].SA[u];
                        work += 1;
                    }
                }
                g_seg_iters += 1;
                evals += 1;
                if (nh == h) break;
                h = nh;
                if (++it > O_ITER_LIMIT) {
                    h = O_INF;
                    break;
                }
            }
            if (evals > g_max_loop) g_max_loop = evals;
            hq[q - q_sys] = h;
            if (h == O_INF || ch[c].HsegA[u] == O_INF)
                ch[c].HsegA[u] = O_INF;
            else
                ch[c].HsegA[u] += h;
        }
        /* per-chain summaries (for the diagnostic output): with one accelerator
         * these are that accelerator's values */
        ch[c].Hseg = 0;
        ch[c].blk = 0;
        ch[c].bucket = -1;
        for (int64_t a = 0; a < O_MAXACC; ++a) {
            if (ch[c].dA[a] == 0) continue;
            ch[c].Hseg = (ch[c].Hseg == O_INF || ch[c].HsegA[a] == O_INF) ? O_INF : ch[c].Hseg + ch[c].HsegA[a];
            if (ch[c].blkA[a] > ch[c].blk) ch[c].blk = ch[c].blkA[a];
            if (ch[c].bucket < 0) ch[c].bucket = ch[c].bucketA[a];
        }
    }

    /* safe blocking (blocking_mode 1, a reading beyond the paper): a
     * lower-priority callback keeps the single-threaded executor for its CPU
     * work and for each of its accelerator requests, each bounded by its
     * segment's Lemma 2 handling time plus the overhead eps; B_c is the
     * longest such callback of a lower-priority chain on c's executor, and
     * infinite when one of those segments has no bound */
    if (blocking_mode == 1) {
        int64_t *hold = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
        for (int64_t l = 0; l < n; ++l) {
            const int64_t cb_lo = chain_cb_off[c0 + l], cb_hi = chain_cb_off[c0 + l + 1];
            for (int64_t b = cb_lo; b < cb_hi; ++b) {
                int64_t t = E[b];
                for (int64_t q = cb_seg_off[b]; q < cb_seg_off[b + 1] && t != O_INF; ++q)
                    t = hq[q - q_sys] == O_INF ? O_INF : t + hq[q - q_sys] + eps;
                if (t > hold[l]) hold[l] = t;
            }
        }
        for (int64_t c = 0; c < n; ++c) {
            ch[c].B = 0;
            for (int64_t l = 0; l < n; ++l)
                if (ch[l].exec == ch[c].exec && ch[l].prio < ch[c].prio && hold[l] > ch[c].B) ch[c].B = hold[l];
        }
        free(hold);
    }
    free(hq);

    /* step 6: Theorem 1 (Eq. 6) chain by chain, each after every chain whose
     * H* it needs: higher-priority chains of its executor and spinning chains
     * of higher-priority executors on its core */
    int64_t remaining = n;
    while (remaining > 0) {
        int64_t progressed = 0;
        for (int64_t c = 0; c < n; ++c) {
            if (ch[c].done) continue;
            int ready = 1, dep_failed = 0;
            for (int64_t h = 0; h < n; ++h) {
                int needed = 0;
                if (h == c) continue;
                if (ch[h].exec == ch[c].exec && ch[h].prio > ch[c].prio) needed = 1; /* hp(c) */
                if (ch[h].exec != ch[c].exec && ch[h].core == ch[c].core &&
                    ch[h].eprio > ch[c].eprio && ch[h].spin)
                    needed = 1; /* spinning member of hpp(c) */
                if (!needed) continue;
                if (!ch[h].done) ready = 0;
                else if (ch[h].status != ST_SCHED) dep_failed = 1;
            }
            if (!ready) continue;
            ch[c].done = 1;
            remaining -= 1;
            progressed = 1;
            if (dep_failed) {
                ch[c].status = ST_DEP;
                ch[c].R = -1;
                continue;
            }
            if (ch[c].B == O_INF) { /* unbounded blocking (safe mode only) */
                ch[c].status = ST_OVERRUN;
                ch[c].R = -1;
                continue;
            }
            /* start: B_c + E_c + H*_c with the interference part of Eq. 4 empty */
            int64_t h0 = 0;
            if (ch[c].delta > 0) {
                for (int64_t a = 0; a < O_MAXACC; ++a) {
                    if (ch[c].dA[a] == 0) continue;
                    const int64_t own = ch[c].SA[a] + ch[c].dA[a] * ch[c].blkA[a];
                    h0 += ch[c].HsegA[a] < own ? ch[c].HsegA[a] : own;
                }
                h0 += ch[c].delta * eps;
            }
            int64_t R = ch[c].B + ch[c].E + h0;
            int64_t it = 0, evals = 0;
            ch[c].status = ST_OVERRUN;
            for (;;) {
                if (R > ch[c].D) break;
                int64_t hs = H_star(ch, n, c, R, eps, &work);
                int64_t Rn = ch[c].B + ch[c].E + hs;
                for (int64_t h = 0; h < n; ++h) {
                    if (h == c) continue;
                    if (ch[h].exec == ch[c].exec && ch[h].prio > ch[c].prio) {
                        /* hp(c): E_h + H*_h */
                        Rn += mu(R, ch[h].T) * (ch[h].E + ch[h].Hstar);
                        work += 1;
                    } else if (ch[h].exec != ch[c].exec && ch[h].core == ch[c].core &&
                               ch[h].eprio > ch[c].eprio) {
                        /* hpp(c): E_h + spin(h) */
                        const int64_t sp = ch[h].spin ? ch[h].Hstar : ch[h].delta * eps;
                        Rn += mu(R, ch[h].T) * (ch[h].E + sp);
                        work += 1;
                    }
                }
                g_chain_iters += 1;
                evals += 1;
                if (Rn == R) {
                    ch[c].status = ST_SCHED;
                    ch[c].Hstar = hs;
                    break;
                }
                R = Rn;
                if (++it > O_ITER_LIMIT) {
                    ch[c].status = ST_ITERCAP;
                    break;
                }
            }
            if (evals > g_max_loop) g_max_loop = evals;
            ch[c].R = ch[c].status == ST_SCHED ? R : -1;
        }
        if (!progressed) break; /* unreachable: the dependency relation is acyclic */
    }

    uint8_t ok = 1;
    for (int64_t c = 0; c < n; ++c) {
        R_out[c0 + c] = ch[c].R;
        st_out[c0 + c] = (uint8_t)ch[c].status;
        if (ch[c].status != ST_SCHED) ok = 0;
        if (aux) {
            int64_t *a = aux + (c0 + c) * 12;
            a[0] = ch[c].E;
            a[1] = ch[c].Emax;
            a[2] = ch[c].delta;
            a[3] = ch[c].S;
            a[4] = ch[c].M;
            a[5] = ch[c].bucket;
            a[6] = ch[c].blk;
            a[7] = ch[c].B;
            a[8] = ch[c].Hseg == O_INF ? -1 : ch[c].Hseg;
            a[9] = ch[c].status == ST_SCHED ? ch[c].Hstar : -1;
            a[10] = ch[c].eprio;
            a[11] = ch[c].prio;
        }
    }
    if (verdict) verdict[s] = ok;
    if (work_out) work_out[s] = work;
    free(ch);
}

/* per system: evaluations of the segment recurrences (Eq. 3), of the chain
 * recurrences (Eq. 6), and the most evaluations any one of them took
 * (max_loop may be NULL) */
void oracle_analyze_iters(int64_t lo, int64_t hi, const int64_t *sys_chain_off,
                          const int64_t *chain_cb_off, const int64_t *cb_seg_off, const int64_t *T,
                          const int64_t *D, const int32_t *prio, const int32_t *exec,
                          const uint8_t *spin, const int64_t *E, const int64_t *A, const int32_t *acc,
                          const int64_t *sys_exec_off, const int32_t *exec_core,
                          const int32_t *exec_prio, int32_t n_buckets, int64_t eps, int64_t kappa,
                          int32_t blocking_mode, int64_t *R, uint8_t *status, int64_t *seg_iters,
                          int64_t *chain_iters, int64_t *max_loop)
{
    for (int64_t s = lo; s < hi; ++s) {
        g_seg_iters = 0;
        g_chain_iters = 0;
        g_max_loop = 0;
        analyze_system(s, sys_chain_off, chain_cb_off, cb_seg_off, T, D, prio, exec, spin, E, A, acc,
                       sys_exec_off, exec_core, exec_prio, NULL, n_buckets, eps, kappa, blocking_mode, R,
                       status, NULL, NULL, NULL);
        seg_iters[s] = g_seg_iters;
        chain_iters[s] = g_chain_iters;
        if (max_loop) max_loop[s] = g_max_loop;
    }
}

/*
 * Analyse systems [lo, hi).  exec_prio may be NULL (derived).  blocking_mode
 * 0 is Lemma 4 as printed, 1 the safe reading (see step 5).  aux, when
 * non-NULL, receives 12 int64 per chain: E, Emax, delta, S*, M*, bucket, blk,
 * B, Hseg (-1 = infinite), H* at R (-1 unless SCHED), executor priority,
 * chain priority.  work, when non-NULL, receives per system the number of
 * interference terms mu(t) * C evaluated.
 */
void oracle_analyze(int64_t lo, int64_t hi, const int64_t *sys_chain_off,
                    const int64_t *chain_cb_off, const int64_t *cb_seg_off, const int64_t *T,
                    const int64_t *D, const int32_t *prio, const int32_t *exec,
                    const uint8_t *spin, const int64_t *E, const int64_t *A, const int32_t *acc,
                    const int64_t *sys_exec_off, const int32_t *exec_core,
                    const int32_t *exec_prio, int32_t n_buckets, int64_t eps, int64_t kappa,
                    int32_t blocking_mode, int64_t *R, uint8_t *status, uint8_t *verdict, int64_t *aux,
                    int64_t *work)
{
    for (int64_t s = lo; s < hi; ++s)
        analyze_system(s, sys_chain_off, chain_cb_off, cb_seg_off, T, D, prio, exec, spin, E, A, acc,
                       sys_exec_off, exec_core, exec_prio, NULL, n_buckets, eps, kappa, blocking_mode, R,
                       status, verdict, aux, work);
}

/*
 * Priority-assignment search: for systems [lo, hi) and K candidate rank
 * orders per system (ranks[s][k][c], 0 = highest, row length nmax), analyse
 * every candidate with derived executor priorities.  cand_ok[s*K + k] = 1 when
 * every chain is schedulable; first_ok[s] = smallest such k, or -1.
 */
void oracle_search(int64_t lo, int64_t hi, const int64_t *sys_chain_off,
                   const int64_t *chain_cb_off, const int64_t *cb_seg_off, const int64_t *T,
                   const int64_t *D, const int32_t *prio, const int32_t *exec, const uint8_t *spin,
                   const int64_t *E, const int64_t *A, const int32_t *acc, const int64_t *sys_exec_off,
                   const int32_t *exec_core, int32_t n_buckets, int64_t eps, int64_t kappa,
                   int32_t blocking_mode, const int16_t *ranks, int32_t K, int32_t nmax, int32_t stop_at_first,
                   uint8_t *cand_ok, int32_t *first_ok, int64_t *R_scratch, uint8_t *st_scratch)
{
    for (int64_t s = lo; s < hi; ++s) {
        first_ok[s] = -1;
        for (int32_t k = 0; k < K; ++k) {
            uint8_t v = 0;
            analyze_system(s, sys_chain_off, chain_cb_off, cb_seg_off, T, D, prio, exec, spin, E,
                           A, acc, sys_exec_off, exec_core, NULL, ranks + (s * (int64_t)K + k) * nmax,
                           n_buckets, eps, kappa, blocking_mode, R_scratch, st_scratch, NULL, NULL, NULL);
            v = 1;
            for (int64_t c = sys_chain_off[s]; c < sys_chain_off[s + 1]; ++c)
                if (st_scratch[c] != ST_SCHED) v = 0;
            if (cand_ok) cand_ok[s * (int64_t)K + k] = v;
            if (v && first_ok[s] < 0) {
                first_ok[s] = k;
                if (stop_at_first) break;
            }
        }
    }
}

/*
 * Audsley-style priority seed (a reading: the paper assigns priorities by
 * hand, and its admission test of Sec. IV-A is not OPA-compatible because
 * bucket ranks, blocking and the DEP rule depend on the whole order).
 *
 * For each system of n chains, ranks are given from the lowest priority up:
 * at level l = n-1, n-2, ..., 0 each unassigned chain c is tried in index
 * order.  The trial order keeps the ranks already given (all below l), puts c
 * at rank l and the other unassigned chains at ranks 0..l-1 in
 * deadline-monotonic order (D ascending, ties by index).  The first c that is
 * schedulable (status SCHED) in the exact analysis of the trial order, with
 * derived executor priorities, takes rank l.  If none is, the unassigned chain
 * with the largest D (ties: highest index) takes it, so that a system where
 * no chain ever passes gets the deadline-monotonic order.  ranks_out[s*nmax + c] is
 * the rank of chain c (0 = highest), -1 beyond the system's chains.
 */
void oracle_audsley(int64_t lo, int64_t hi, const int64_t *sys_chain_off,
                    const int64_t *chain_cb_off, const int64_t *cb_seg_off, const int64_t *T,
                    const int64_t *D, const int32_t *prio, const int32_t *exec, const uint8_t *spin,
                    const int64_t *E, const int64_t *A, const int32_t *acc, const int64_t *sys_exec_off,
                    const int32_t *exec_core, int32_t n_buckets, int64_t eps, int64_t kappa,
                    int32_t blocking_mode, int32_t nmax, int16_t *ranks_out, int64_t *R_scratch,
                    uint8_t *st_scratch)
{
    for (int64_t s = lo; s < hi; ++s) {
        const int64_t c0 = sys_chain_off[s], n = sys_chain_off[s + 1] - c0;
        int16_t *rank = ranks_out + s * (int64_t)nmax;
        int16_t *trial = (int16_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int16_t));
        for (int64_t c = 0; c < nmax; ++c) rank[c] = -1;
        for (int64_t level = n - 1; level >= 0; --level) {
            int64_t chosen = -1;
            for (int64_t c = 0; c < n && chosen < 0; ++c) {
                if (rank[c] >= 0) continue;
                for (int64_t k = 0; k < n; ++k) {
                    if (rank[k] >= 0) {
                        trial[k] = rank[k];
                    } else if (k == c) {
                        trial[k] = (int16_t)level;
                    } else { /* position among the other unassigned chains, deadline-monotonic */
                        int64_t pos = 0;
                        for (int64_t u = 0; u < n; ++u)
                            if (u != c && u != k && rank[u] < 0 &&
                                (D[c0 + u] < D[c0 + k] || (D[c0 + u] == D[c0 + k] && u < k)))
                                pos += 1;
                        trial[k] = (int16_t)pos;
                    }
                }
                analyze_system(s, sys_chain_off, chain_cb_off, cb_seg_off, T, D, prio, exec, spin, E, A, acc,
                               sys_exec_off, exec_core, NULL, trial, n_buckets, eps, kappa, blocking_mode,
                               R_scratch, st_scratch, NULL, NULL, NULL);
                if (st_scratch[c0 + c] == ST_SCHED) chosen = c;
            }
            if (chosen < 0) { /* no chain passes: the largest deadline goes lowest */
                for (int64_t c = 0; c < n; ++c)
                    if (rank[c] < 0 && (chosen < 0 || D[c0 + c] >= D[c0 + chosen])) chosen = c;
            }
            rank[chosen] = (int16_t)level;
        }
        free(trial);
    }
}
