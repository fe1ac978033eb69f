/*
 * paam_rta.h -- C ABI of the GB300 batched PAAM response-time analysis.
 *
 * PAAM (Sec. IV) serves the accelerator segments of ROS 2 callback chains
 * through a priority-driven server executor and admits a new client only if
 * every chain's worst-case response time (WCRT) stays within its deadline
 * (admission control, Sec. IV-A and Sec. IV-F).  This library evaluates that
 * WCRT bound -- Theorem 1 (Eq. 6) with Eqs. 1-4 and Lemma 4 (Eq. 5) -- for
 * very many independent systems at once on one GB300 GPU, exactly, in int64
 * nanoseconds.  Every step of the analysis runs in the library's own CUDA
 * kernels (sm_103a); there is no CPU fallback.
 *
 * Conventions
 *   - Every call returns PAAM_OK (0) or a negative PAAM_E_* code; nothing
 *     throws across the ABI.  paam_strerror() names a code.
 *   - The caller owns every buffer it passes; the library owns contexts,
 *     batches and models and frees them in the matching *_free / destroy.
 *   - "device" pointers are CUDA device (or managed) memory of the context's
 *     GPU; "host" pointers are ordinary or pinned host memory.
 *   - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls that produce device outputs only enqueue work
 *     on it, unless stated otherwise.
 *   - All times are int64 nanoseconds.
 */
#ifndef PAAM_RTA_H
#define PAAM_RTA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define PAAM_OK 0
#define PAAM_E_INVAL (-1)       /* malformed input: offsets, D > T, T <= 0, negative time,
                                   duplicate priority, executor index out of range, ... */
#define PAAM_E_RANGE (-2)       /* a bound could overflow int64 (see paam_rta_load_systems) */
#define PAAM_E_NOMEM (-3)       /* device or host allocation failed */
#define PAAM_E_CUDA (-4)        /* a CUDA runtime call failed */
#define PAAM_E_TIMEOUT (-5)     /* a bounded device wait gave up */
#define PAAM_E_UNSUPPORTED (-6) /* input outside what the library implements */
#define PAAM_E_STATE (-7)       /* object used with the wrong context / after free */

/* ---- per-chain status --------------------------------------------------- */
#define PAAM_ST_SCHED 0   /* R <= D: the chain meets its deadline                    */
#define PAAM_ST_OVERRUN 1 /* the recurrence exceeded D (Theorem 1 gives no bound <= D) */
#define PAAM_ST_DEP 2     /* a chain whose H* this chain needs is not schedulable     */
#define PAAM_ST_ITERCAP 3 /* a fixed-point recurrence reached PAAM_MAX_ITER evaluations;
                             unreachable for a loaded batch (paam_rta_load_systems
                             refuses systems whose bound exceeds it), kept as a guard */

#define PAAM_MAX_CHAINS 64        /* chains per system                           */
#define PAAM_MAX_TIME (1LL << 40) /* largest T, D, E, A accepted (about 18 min)  */
#define PAAM_MAX_ACC 4            /* accelerators per batch (indices 0..3)        */
#define PAAM_MAX_OVERHEAD (1LL << 32) /* largest eps, kappa accepted             */
#define PAAM_MAX_ITER (1 << 20)   /* evaluations any one fixed-point recurrence of a
                                     system may need (paam_rta_load_systems)      */

typedef struct paam_ctx paam_ctx;
typedef struct paam_batch paam_batch;
typedef struct paam_model paam_model;

/*
 * A batch of systems in structure-of-arrays, CSR form (system model of
 * Sec. II-C).  System s owns chains [sys_chain_off[s], sys_chain_off[s+1])
 * and executors [sys_exec_off[s], sys_exec_off[s+1]); chain c owns callbacks
 * [chain_cb_off[c], chain_cb_off[c+1]) executed in order; callback b owns
 * accelerator segments [cb_seg_off[b], cb_seg_off[b+1]).  Callbacks are not
 * shared between chains.
 *
 *   T[c], D[c]     period and constrained deadline, 0 < D <= T
 *   prio[c]        chain priority, larger = higher, distinct within a system
 *   exec[c]        executor of the chain, local index in [0, executors of s)
 *   spin[c]        1 if the chain busy-waits on accelerator requests, else 0
 *   E[b]           CPU WCET of callback b (all its CPU segments), >= 0
 *   A[q]           WCET of accelerator segment q, >= 0
 *   acc[q]         accelerator of segment q, 0 .. PAAM_MAX_ACC - 1 (NULL: all
 *                  0).  Each accelerator has its own server (rule R1) and is
 *                  analysed on its own: buckets, same-bucket blocking and hps
 *                  are per accelerator, and H_c sums the per-accelerator
 *                  handling times.  A batch that uses a second accelerator
 *                  is analysed by the exact int64 kernel (slower)
 *   exec_core[x]   CPU core of executor x, >= 0
 *   exec_prio[x]   executor (process) priority, larger = higher, distinct among
 *                  executors of one core; NULL = derived as the highest chain
 *                  priority on the executor (criticality-as-priority, Sec. II-C)
 *
 * Offsets are non-decreasing, start at 0 and end at the matching count.  All
 * pointers are host memory (is_device = 0) or device memory of the
 * context's GPU (is_device = 1).
 */
typedef struct {
    int64_t n_sys, n_chain, n_cb, n_seg, n_exec;
    const int64_t *sys_chain_off; /* [n_sys + 1]   */
    const int64_t *chain_cb_off;  /* [n_chain + 1] */
    const int64_t *cb_seg_off;    /* [n_cb + 1]    */
    const int64_t *T;             /* [n_chain]     */
    const int64_t *D;             /* [n_chain]     */
    const int32_t *prio;          /* [n_chain]     */
    const int32_t *exec;          /* [n_chain]     */
    const uint8_t *spin;          /* [n_chain]     */
    const int64_t *E;             /* [n_cb]        */
    const int64_t *A;             /* [n_seg]       */
    const int32_t *acc;           /* [n_seg] or NULL */
    const int64_t *sys_exec_off;  /* [n_sys + 1]   */
    const int32_t *exec_core;     /* [n_exec]      */
    const int32_t *exec_prio;     /* [n_exec] or NULL */
    int32_t is_device;
    int32_t reserved_;
} paam_systems_view;

/*
 * Analysis parameters (Sec. IV-F).
 *   n_buckets      n >= 1 worker buckets of the server (rule R2); accelerator
 *                  users are ranked by descending chain priority and rank r of
 *                  |U| users goes to bucket floor(r * n / |U|)
 *   blocking_mode  0: B_c as in Lemma 4 (largest CPU WCET of one callback of
 *                  a lower-priority chain on the executor);
 *                  1: a safe reading of the same blocking: that callback also
 *                  holds the single-threaded executor during each of its
 *                  accelerator requests, so B_c is the largest E_i + sum over
 *                  callback i's segments of (Lemma 2 bound + eps) of a
 *                  lower-priority chain on the executor, and a segment
 *                  without a bound (above its chain's deadline) makes the
 *                  chain PAAM_ST_OVERRUN.  Mode 1 runs the exact int64 kernel
 *                  for every system (slower).  Other values: PAAM_E_INVAL
 *   eps_ns         per-request server overhead epsilon (Eq. 1), 0..2^32
 *   kappa_ns       device preemption cost kappa, A* = A + 2 kappa, 0..2^32
 */
typedef struct {
    int32_t n_buckets;
    int32_t blocking_mode;
    int64_t eps_ns;
    int64_t kappa_ns;
} paam_analysis_opts;

/* Create a context bound to CUDA device `device_ordinal`. */
int paam_create(paam_ctx **out, int device_ordinal);

/* Release a context (its batches and models must be freed first). */
void paam_destroy(paam_ctx *ctx);

/* Short English name of a return code. */
const char *paam_strerror(int code);

/*
 * Copy a batch of systems into library-owned device memory and validate it on
 * the GPU.  Blocks until validation finishes (it synchronises `stream`).
 *
 * Errors: PAAM_E_INVAL for malformed input (see paam_systems_view), a system
 * with more than PAAM_MAX_CHAINS chains, or a time above PAAM_MAX_TIME;
 * PAAM_E_RANGE when N * (ceil(Dmax / Tmin) + 1) * Cmax + Base could exceed
 * 2^62 for some system (the largest value any fixed-point iterate of Eqs. 3-6
 * can take with eps, kappa <= PAAM_MAX_OVERHEAD), so that no int64 sum
 * overflows; PAAM_E_RANGE also when a system's iteration bound
 * L = sum over its chains h of ceil(Dmax / T_h), plus 2, exceeds
 * PAAM_MAX_ITER (Dmax: the system's largest deadline).  Each recurrence of
 * Eqs. 3 and 6 rises strictly until it converges or passes its deadline, and
 * after its first step it can rise again only when some arrival count
 * ceil(t / T_h) + 1 of Lemma 1 has grown, which happens at most
 * ceil(Dmax / T_h) times per chain h below the deadline; so no recurrence of
 * an accepted system takes more than L evaluations, and the analysis kernels
 * stop any that would at PAAM_MAX_ITER (PAAM_ST_ITERCAP).  PAAM_E_INVAL for
 * an accelerator index outside 0..PAAM_MAX_ACC-1; PAAM_E_NOMEM / PAAM_E_CUDA.
 * On error *out is NULL and nothing is leaked.
 */
int paam_rta_load_systems(paam_ctx *ctx, const paam_systems_view *view, void *stream,
                          paam_batch **out);

/* Number of systems / chains of a loaded batch (0 for NULL). */
int64_t paam_batch_n_sys(const paam_batch *b);
int64_t paam_batch_n_chain(const paam_batch *b);

/* Free a batch (after the work that uses it has completed). */
void paam_batch_free(paam_batch *b);

/*
 * WCRT analysis of every chain of every system (Theorem 1, Eq. 6, with
 * Eqs. 1-4 and Lemma 4).  Enqueued on `stream`; outputs are device buffers:
 *   R[n_chain]       int64: the least fixed point of Eq. 6 when the chain is
 *                    schedulable, else -1
 *   status[n_chain]  PAAM_ST_* per chain
 *   verdict[n_sys]   1 if every chain of the system is PAAM_ST_SCHED (the
 *                    admission test of Sec. IV-A), else 0
 * verdict may be NULL.  Results are bit-identical to the definition for any
 * launch configuration.  The first call for a given (outputs, options,
 * launch configuration) captures the analysis into a CUDA graph owned by the
 * batch; later calls with the same key replay it on `stream`.  A batch may be
 * analysed by one host thread at a time.  Errors: PAAM_E_INVAL (NULL outputs, n_buckets < 1),
 * PAAM_E_RANGE (eps or kappa above PAAM_MAX_OVERHEAD), PAAM_E_INVAL
 * (blocking_mode not 0 or 1), PAAM_E_CUDA (launch failure).
 */
int paam_rta_analyze_batch(paam_ctx *ctx, const paam_batch *batch, const paam_analysis_opts *opts,
                           int64_t *R, uint8_t *status, uint8_t *verdict, void *stream);

/*
 * Exact priority-assignment search.  The paper fixes chain priorities by
 * criticality (CAPA, Sec. II-C); this call evaluates K candidate chain
 * priority orders per system with the same exact analysis and reports which
 * ones pass the admission test (every chain schedulable, Sec. IV-A).
 *
 *   ranks[n_sys][K][nmax]  device int16: ranks[s][k][c] is the rank of chain c
 *                          (local index) of system s in candidate k, 0 =
 *                          highest priority; each row's first n_s entries
 *                          must be a permutation of 0..n_s-1 (entries past
 *                          n_s are ignored); nmax >= the batch's largest chain
 *                          count.  Executor priorities follow the candidate
 *                          (highest chain priority on the executor).
 *   stop_at_first          0: analyse every candidate; 1: candidates above the
 *                          best schedulable one found for a system may be
 *                          skipped (their cand_ok entry then reads 0).
 *   cand_ok[n_sys * K]     device, optional: 1 where candidate k of system s
 *                          (index s * K + k) is schedulable.
 *   first_ok[n_sys]        device: smallest schedulable k, or -1.
 *
 * The result does not depend on the launch configuration or on the order in
 * which candidates are processed.  The call synchronises `stream`.  Errors:
 * PAAM_E_INVAL (a rank row that is not a permutation, bad sizes),
 * PAAM_E_RANGE (n_sys * K above 2^31 - 1, eps/kappa above the cap),
 * PAAM_E_UNSUPPORTED, PAAM_E_NOMEM, PAAM_E_CUDA.
 */
int paam_rta_search_priorities(paam_ctx *ctx, const paam_batch *batch, const paam_analysis_opts *opts,
                               const int16_t *ranks, int32_t K, int32_t nmax, int32_t stop_at_first,
                               uint8_t *cand_ok, int32_t *first_ok, void *stream);

/*
 * The same search over an ordered subset of each system's candidates:
 * ranks holds Kc candidates per system ([n_sys][Kc][nmax]); slot j of system
 * s visits candidate order[s * K + j] (device int32 in [0, Kc)), so K slots
 * are analysed per system in that order.  first_ok[s] is the candidate index
 * (not the slot) of the first admitted slot, or -1; cand_ok is indexed
 * s * Kc + candidate and reads 0 for candidates not visited.  A surrogate
 * ranking plus this call is the guided search: only candidates it visits
 * can be admitted, and every admission is exact.
 */
int paam_rta_search_ordered(paam_ctx *ctx, const paam_batch *batch, const paam_analysis_opts *opts,
                            const int16_t *ranks, int32_t Kc, int32_t nmax, const int32_t *order, int32_t K,
                            int32_t stop_at_first, uint8_t *cand_ok, int32_t *first_ok, void *stream);

/*
 * The analysis of a batch held in host memory (paam_rta_load_systems +
 * paam_rta_analyze_batch + copies of the results, in one call), pipelined:
 * the batch is split into chunks of whole systems, and the host-to-device
 * copy of chunk c + 1 runs while chunk c is validated and analysed and the
 * results of earlier chunks are copied back.  The results are those of
 * paam_rta_analyze_batch on the same systems (Theorem 1, Eq. 6).
 *
 *   v               host view (is_device = 0); page-locked memory lets the
 *                   copies run asynchronously, other host memory works but
 *                   serialises them.  Validated as by paam_rta_load_systems,
 *                   chunk by chunk.
 *   launch_config   index of a launch configuration
 *                   (paam_rta_num_launch_configs), or -1 for the default.
 *   chunk_systems   systems per chunk, or <= 0 for automatic chunks of
 *                   halving size (half the batch, a quarter, ... down to
 *                   about 64 MB of input, the rest in the last chunk).
 *   R, status       host [n_chain]; verdict host [n_sys], optional.
 *
 * Device memory for the whole batch is taken from the device's memory pool
 * for the duration of the call.  Returns when every result is on the host.
 * Errors: those of paam_rta_load_systems (PAAM_E_INVAL with the first bad
 * chunk; no result of it or a later chunk is written), PAAM_E_RANGE,
 * PAAM_E_NOMEM, PAAM_E_CUDA.
 */
int paam_rta_analyze_host(paam_ctx *ctx, const paam_systems_view *v, const paam_analysis_opts *opts,
                          int32_t launch_config, int64_t chunk_systems, int64_t *R, uint8_t *status,
                          uint8_t *verdict);

/*
 * Audsley-style priority seed: a candidate order for the search, built from
 * the lowest priority level up with the exact analysis (Theorem 1) as the
 * test.  The paper assigns priorities by hand; this greedy is a reading of
 * Audsley's lowest-level-first assignment for a test that is not
 * OPA-compatible (bucket ranks, blocking and the DEP rule depend on the whole
 * order), so it is a seed for the search, not an optimum.
 *
 * For a system of n chains, at level l = n-1 down to 0 each unassigned chain
 * c is tried in index order: the chains already placed keep their ranks (all
 * below l), c takes rank l and the other unassigned chains ranks 0..l-1 in
 * deadline-monotonic order (D ascending, ties by index).  The first c that is
 * schedulable in the exact analysis of that order (executor priorities
 * derived from it) takes level l; if none is, the unassigned chain with the
 * largest D (ties: highest index) does.
 *
 *   opts                   as for the analysis (n_buckets, eps, kappa,
 *                          blocking_mode); the batch's own priorities are
 *                          not used.
 *   nmax                   row length of ranks_out, >= the batch's largest
 *                          chain count.
 *   ranks_out[n_sys][nmax] device int16: rank of chain c of system s (0 =
 *                          highest priority), -1 beyond the system's chains;
 *                          a row is a candidate row of
 *                          paam_rta_search_priorities.
 *
 * Every trial of every system at one level is analysed in one launch of the
 * exact int64 kernel, which stops each trial once chain c is done.  Scratch
 * is taken from the stream's pool (at most about 512 MB; larger batches run
 * in system chunks).  The call synchronises `stream`.  Errors: PAAM_E_INVAL
 * (bad sizes or options), PAAM_E_RANGE (eps/kappa above the cap),
 * PAAM_E_STATE (a batch of another context), PAAM_E_NOMEM, PAAM_E_CUDA.
 */
int paam_rta_audsley_order(paam_ctx *ctx, const paam_batch *batch, const paam_analysis_opts *opts, int32_t nmax,
                           int16_t *ranks_out, void *stream);

/*
 * Surrogate ranking model (not in the paper: it serves the priority search).
 * A multilayer perceptron 1024 -> 256 -> 256 -> 256 -> 64 (GELU hidden
 * layers, bf16 weights for bf16 tensor-core GEMMs with fp32 accumulation,
 * fp32 master weights and AdamW moments) maps 16 features of each of up to
 * 64 chains of a system under one priority order to each chain's predicted
 * exact R / D (clipped to [0, 2]; 2 for an unschedulable chain).  The model
 * only orders candidates: admission always comes from the exact analysis.
 *
 * paam_surrogate_train: trains on every system of `batch` with their own
 * priorities; R / status are that batch's exact analysis outputs (device).
 * *model NULL creates a model (initialised from opts->seed); otherwise the
 * given model keeps training.  Synchronous.  opts->epoch_loss (host,
 * optional) receives the mean minibatch loss of each epoch.
 *
 * paam_surrogate_infer: scores candidate k of system s (same ranks layout as
 * paam_rta_search_priorities) by its largest predicted R / D and writes the
 * top_k candidate indices per system in increasing score to ranked
 * ([n_sys][top_k] device int32); scores ([n_sys][K] device float) optional.
 * The first n_pinned candidate slots of every system (0 <= n_pinned <= K,
 * e.g. heuristic seeds) are ranked first, in slot order, ahead of every
 * scored candidate; their scores are still written.  Synchronises `stream`.
 *
 * paam_surrogate_predict: per-chain predictions ([n_sys][64] device float) of
 * the batch's own priority orders.
 *
 * paam_surrogate_grad: loss and gradients (host, paam_model_num_params()
 * floats, parameter order as paam_model_get_params) of one minibatch X
 * ([rows][1024] device bf16), L ([rows][64] device float, < 0 = no chain),
 * rows a multiple of 128; the model is not updated.  For testing.
 *
 * Parameter order (get / set): per layer the weights [out][in] row-major,
 * then the biases.  paam_model_save / load write and read a checkpoint
 * (weights, biases, AdamW moments and step count).
 */
typedef struct {
    int32_t epochs;        /* passes over the batch                              */
    int32_t batch_rows;    /* minibatch size, a multiple of 128                   */
    float lr, weight_decay, beta1, beta2, adam_eps;
    uint64_t seed;         /* initialisation of a new model and minibatch order  */
    int32_t n_buckets;     /* analysis parameters of the labels (features use    */
    int32_t reserved_;     /*   the bucket count and kappa)                      */
    int64_t kappa_ns;
    float *epoch_loss;     /* host, optional, [epochs]                           */
} paam_train_opts;

int paam_model_create(paam_ctx *ctx, uint64_t seed, paam_model **out);
void paam_model_free(paam_model *model);
int64_t paam_model_num_params(void);
int paam_model_get_params(const paam_model *model, float *host);
int paam_model_set_params(paam_model *model, const float *host);
int paam_model_save(const paam_model *model, const char *path);
int paam_model_load(paam_ctx *ctx, const char *path, paam_model **out);
int paam_surrogate_train(paam_ctx *ctx, const paam_batch *batch, const int64_t *R, const uint8_t *status,
                         const paam_train_opts *opts, paam_model **model);
int paam_surrogate_infer(paam_ctx *ctx, const paam_model *model, const paam_batch *batch, const int16_t *ranks,
                         int32_t K, int32_t nmax, int32_t n_buckets, int64_t kappa_ns, int32_t n_pinned,
                         int32_t top_k, int32_t *ranked, float *scores, void *stream);
int paam_surrogate_predict(paam_ctx *ctx, const paam_model *model, const paam_batch *batch, int32_t n_buckets,
                           int64_t kappa_ns, float *pred, void *stream);

/*
 * paam_surrogate_search: the priority-assignment search with exact verdicts,
 * guided by the network (the admission test of Sec. IV-A on each visited
 * candidate, the analysis of Sec. IV-F).  Per system, candidates 0 ..
 * n_pinned-1 (the pinned seeds) are analysed first, in slot order; for the
 * systems none of them admits, the network scores the other K - n_pinned
 * candidates, and its 32 best (in increasing score) and then the rest (in
 * index order) are analysed, each system stopping at its first admitted
 * candidate.  Every candidate of a system is visited
 * unless an earlier one is admitted, so first_ok[s] >= 0 exactly when
 * paam_rta_search_priorities finds an admitted candidate of s; first_ok[s] is
 * then the one found first in this order (a candidate index), else -1.
 * ranks and nmax as for paam_rta_search_priorities (K candidates per system,
 * at most 64 chains); o as for the analysis (its n_buckets and kappa_ns also
 * feed the features); first_ok device int32 [n_sys].  Blocks until done.
 * PAAM_E_INVAL for bad arguments (n_pinned outside 0..K, a rank row that is
 * not a permutation), PAAM_E_STATE for a model or batch of another context,
 * PAAM_E_RANGE for n_sys * K above 2^31 - 1.
 */
int paam_surrogate_search(paam_ctx *ctx, const paam_model *model, const paam_batch *batch,
                          const paam_analysis_opts *opts, const int16_t *ranks, int32_t K, int32_t nmax,
                          int32_t n_pinned, int32_t *first_ok, void *stream);
int paam_surrogate_grad(paam_ctx *ctx, paam_model *model, const void *X, const float *L, int32_t rows,
                        float *grads_host, float *loss_host);

/*
 * The network's inputs: for item = system * K + candidate, 64 chain slots x
 * 16 features (bf16, device, [n_sys * K][1024]); slots past the system's
 * chains are zero.  Per chain: E / T, S* / T, D / T, log2(T / Tmin) / 4,
 * rank / n, min(delta, 16) / 16, Emax / D, M* / D, sum over hp of (E + S*) / T,
 * sum over hpp of E / T, sum over hps of S* / T, B / D, blk / D, (E + S*) / D,
 * sum over hp and hpp of (E + S*) / D, 1 -- each clipped to [0, 8] (E, S*,
 * M*, B, blk, hp, hpp, hps as
 * in the analysis, under the candidate's priorities).  ranks NULL and K = 1
 * take the batch's own priorities.  Enqueued on `stream`.
 */
int paam_surrogate_features(paam_ctx *ctx, const paam_batch *batch, const int16_t *ranks, int32_t K,
                            int32_t nmax, int32_t n_buckets, int64_t kappa_ns, void *X, void *stream);

/*
 * End-to-end bounds of chains that span several executors (Sec. IV-F, the
 * end-to-end latency of a chain made of sub-chains that run on different
 * executors): each sub-chain is analysed as a chain of its own executor by
 * paam_rta_analyze_batch, and the end-to-end bound is the sum of their
 * response times plus a communication cost per hand-over,
 *   R* = sum over the m sub-chains of R_c + (m - 1) eps_prime_ns.
 * (The paper adds one communication cost eps' < eps; it is read here as one
 * per hand-over between consecutive sub-chains.)
 *   e2e_off[n_e2e + 1]   device, CSR offsets into e2e_chain (non-decreasing,
 *                        e2e_off[0] = 0)
 *   e2e_chain[...]       device, the batch-wide chain indices of each end-to-end
 *                        chain's sub-chains (0 <= index < n_chain)
 *   D_e2e[n_e2e]         device, end-to-end deadlines (ns, > 0)
 *   R, status            device, the outputs of paam_rta_analyze_batch
 *   R_e2e, status_e2e    device outputs: R* and PAAM_ST_SCHED when every
 *                        sub-chain is PAAM_ST_SCHED and R* <= D*; else R* = -1
 *                        and PAAM_ST_DEP if a sub-chain is DEP, otherwise
 *                        PAAM_ST_OVERRUN (an empty chain is SCHED with R* = 0)
 * eps_prime_ns is 0..PAAM_MAX_OVERHEAD.  The call synchronises `stream`.
 * Errors: PAAM_E_INVAL (NULL arrays, n_e2e < 0, a sub-chain index out of
 * range or decreasing offsets, found on the device), PAAM_E_RANGE (eps'),
 * PAAM_E_NOMEM, PAAM_E_CUDA.  Out-of-range entries are not read.
 */
int paam_rta_end_to_end(paam_ctx *ctx, const paam_batch *batch, int64_t n_e2e, const int64_t *e2e_off,
                        const int64_t *e2e_chain, const int64_t *D_e2e, int64_t eps_prime_ns,
                        const int64_t *R, const uint8_t *status, int64_t *R_e2e, uint8_t *status_e2e,
                        void *stream);

/*
 * Device preemption cost kappa (Sec. IV-F; measured by the method of the
 * paper's GPU preemption-delay benchmark, Sec. V): on `device`, two streams
 * at the lowest and the highest stream priority each get their own buffers
 * for kernel `kind` (0 MatMul, 1 Reduction, 2 VectorAdd, 3 Histogram; kernels
 * of this library).  Each of `iters` iterations launches the kernel on the
 * low-priority stream and at once on the high-priority stream, times the
 * high-priority one with stream events, then times it again alone;
 *   delay_us[i] = (with the low-priority kernel running) - (alone), in us,
 *   base_us[i]  = the time alone (optional, may be NULL).
 * delay_us is host memory of `iters` floats.  Synchronises the device;
 * allocates and frees device memory.  Errors: PAAM_E_INVAL (kind outside
 * 0..3, iters < 1, NULL delay_us), PAAM_E_NOMEM, PAAM_E_CUDA.
 */
int paam_measure_preemption(int device, int kind, int iters, float *delay_us, float *base_us);

/*
 * Launch configurations.  The analysis has several built-in launch
 * configurations (lanes per system, chain-table size of the first pass, lanes
 * per system for systems with more chains, CTA size, static shares or a
 * device work queue, index or size order of the systems); every one produces
 * bit-identical results.  A batch starts with configuration 12 (16 lanes per
 * system, work queue).
 *
 * paam_rta_autotune times every configuration on the batch itself (the
 * analysis is run 6 times per configuration, the first run discarded, and
 * the median of the other 5 kept), keeps the fastest for later
 * paam_rta_analyze_batch calls on this batch, and returns its index (>= 0)
 * or a negative error.  times_ms, if not NULL, receives up to max_out
 * per-configuration median times in milliseconds.  It
 * synchronises `stream` and allocates temporary device outputs.
 */
int paam_rta_num_launch_configs(void);
int paam_rta_autotune(paam_ctx *ctx, paam_batch *batch, const paam_analysis_opts *opts, void *stream,
                      float *times_ms, int max_out);

/*
 * paam_rta_autotune_search: the same for the priority search.  Every
 * configuration runs paam_rta_search_priorities on `ranks` (layout as
 * there; 6 runs, the first discarded, the median of 5 kept, timed on the host
 * around each call), and the fastest is kept on the batch for later analyses
 * and searches.  Returns its index or a negative error; times_ms as above.
 * Synchronises `stream`.
 */
int paam_rta_autotune_search(paam_ctx *ctx, paam_batch *batch, const paam_analysis_opts *opts, const int16_t *ranks,
                             int32_t K, int32_t nmax, int32_t stop_at_first, void *stream, float *times_ms,
                             int max_out);
int paam_rta_set_launch_config(paam_batch *batch, int index); /* PAAM_E_INVAL if out of range */
int paam_rta_get_launch_config(const paam_batch *batch);

/*
 * Allocation-free analysis.  (The paper has no counterpart: this entry point
 * exists for callers of this library that cannot allocate memory at the time
 * they need an admission test -- a real-time executor whose control loop
 * forbids allocation after start-up, a host that has handed its whole device
 * memory to another allocator, or an integration that must account for all
 * of its memory before it runs.)
 *
 * Same results as paam_rta_load_systems + paam_rta_analyze_batch, but the
 * call needs no context and allocates nothing: `view` must hold DEVICE
 * pointers (is_device = 1) to the caller's tables, R / status / verdict are
 * the caller's device outputs, and the bookkeeping the analysis needs lives in
 * one fixed device array of the library (PAAM_NOALLOC_MAX_SYS * 8 + 128 bytes,
 * about 512 KiB), present on every GPU that loads the library until the
 * process exits.
 *
 *   - n_sys above PAAM_NOALLOC_MAX_SYS is rejected with PAAM_E_RANGE (split
 *     larger batches into several calls);
 *   - the input is validated exactly as paam_rta_load_systems does, so the
 *     call synchronises `stream` once (after validation) and returns the
 *     same error codes; the analysis itself is then enqueued on `stream`;
 *   - every call looks up the array's device address on the current device
 *     (a lookup, no allocation), so the address stays right across a
 *     cudaDeviceReset; the first call on a device also reads two device
 *     attributes once; make that first call before any stream capture;
 *   - every call shares the array and it keeps the last call's contents
 *     (each call resets the parts that must start at zero): calls whose work
 *     overlaps on the GPU -- other streams, other host threads -- race and
 *     must be serialised by the caller.
 */
#define PAAM_NOALLOC_MAX_SYS 65536
int paam_rta_analyze_noalloc(const paam_systems_view *view, const paam_analysis_opts *opts, int64_t *R,
                             uint8_t *status, uint8_t *verdict, void *stream);

/*
 * Tensor-core GEMM used by the surrogate network, exposed for testing:
 * C[M, N] (fp32, row-major) = A[M, K] * B[N, K]^T with A and B bf16 row-major
 * device matrices (leading dimension K), fp32 accumulation.  K must be a
 * multiple of 64 and N of 64.  Enqueued on `stream`; *err (device int32,
 * zeroed by the caller) receives PAAM_E_TIMEOUT if a bounded device wait
 * expired.  Not part of the paper.
 */
int paam_tc_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int32_t *err, void *stream);

/*
 * The network's activation as its GEMM epilogues compute it, exposed for
 * testing: for i < n, gelu[i] = z Phi(z) and grad[i] = Phi(z) + z Phi'(z) at
 * z = z[i] (fp32 device arrays; either output may be NULL), with GELU in its
 * tanh form: Phi(z) is taken as (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2
 * (Hendrycks and Gimpel 2016) and phi as its derivative.
 * Enqueued on `stream`.  PAAM_E_INVAL for n < 0 or a NULL z with n > 0.
 * Not part of the paper.
 */
int paam_diag_gelu(const float *z, float *gelu, float *grad, int64_t n, void *stream);

/*
 * The multiply-shift divisor the analysis kernels build for every period T
 * (Lemma 1, Eq. 2: ceil(t / T) is taken as a multiply-high and a shift),
 * exposed for testing: for i < n, l[i] = ceil(log2 T[i]) and m[i] =
 * ceil(2^(31 + l[i]) / T[i]), with which floor(x / T) = floor(x m / 2^(31 + l))
 * for every x < 2^31 (Granlund and Montgomery 1994, Theorem 4.2).  T, m and l
 * are uint32 device arrays of n elements; each T[i] must lie in [1, 2^30)
 * (outside it the outputs are unspecified, nothing is read or written beyond
 * the arrays).  Enqueued on `stream`.  PAAM_E_INVAL for n < 0 or a NULL
 * array with n > 0.  Not part of the paper.
 */
int paam_diag_divisor(const uint32_t *T, uint32_t *m, uint32_t *l, int64_t n, void *stream);

/*
 * Diagnostics: number of CUDA kernels this library has launched in this
 * process (all contexts).  Not part of the paper; used to report how many
 * of the library's own kernels ran inside a timed region.
 */
uint64_t paam_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* PAAM_RTA_H */
