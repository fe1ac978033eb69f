// internal.cuh -- definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/paam_rta.h"

#define PAAM_CUDA_TRY(expr)                                    \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) {                               \
            paam_note_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return PAAM_E_CUDA;                                \
        }                                                      \
    } while (0)

void paam_note_cuda_error(cudaError_t e, const char *expr, const char *file, int line);

// Counts kernel launches made by this library (paam_launch_count()).
void paam_count_launch(unsigned n = 1);
// launches counted while a stream was being captured (they run when the graph is launched)
void paam_uncount_launch(unsigned n);

struct AnalysisParams {
    int32_t n_buckets;
    int32_t blocking_mode; // 0: Lemma 4 as printed; 1: the safe reading (analyze_wide.cu only)
    int32_t K; // 0: analyse every system once; K > 0: candidate mode (below)
    int64_t eps;
    int64_t kappa;
    // Candidate mode (priority-assignment search): work item i is system
    // i % n_sys under candidate i / n_sys (candidates in order, so that early
    // exit prunes well; sys_major below changes that); its chain priorities come from the rank row
    // ranks[(system * K + candidate) * nmax ..] (0 = highest), executor priorities derived
    // (criticality-as-priority).  A candidate stops at its first chain that is
    // not schedulable; results go to cand_ok[i] (optional) and to a running
    // minimum first_ok[system] of the schedulable candidate indices, cand_ok
    // indexed system * K + candidate.  early:
    // skip candidates above the current minimum.  err receives PAAM_E_INVAL
    // when a rank row is not a permutation of 0..n-1.
    const int16_t *ranks;
    int64_t n_sys;
    int32_t nmax;
    int32_t Kc;           // candidates per system in ranks / cand_ok (K = slots visited)
    const int32_t *order; // optional [n_sys][K]: candidate visited in slot j (else slot j = candidate j)
    int32_t early;
    // sys_major (the exhaustive search, no early exit): item i is instead candidate
    // i % K of system i / K, so that a system's candidates run one after another and
    // share its chain records in L1
    int32_t sys_major;
    uint8_t *cand_ok;
    int32_t *first_ok;
    int32_t *err;
    // Work queue: with queue_batch > 0 a group takes queue_batch consecutive
    // items at a time from the device counter *queue (zero at launch) instead
    // of a fixed grid-stride share, so groups that drew small systems take
    // more; items are still handed out in increasing order.
    unsigned long long *queue;
    int32_t queue_batch;
    // Size binning: with sys_order set, the k-th system handed out is
    // sys_order[k] (systems sorted by chain count), so the groups that share a
    // warp analyse systems of one size and stay converged longer.
    const int32_t *sys_order;
    // Target mode (the Audsley-style seed; the int64 and lazy kernels): with
    // target set, candidate (system, c) is decided by one chain,
    // target[system * Kc + c] (-1: skip the item): cand_ok receives whether
    // that chain is schedulable, the analysis stops once it is done, and
    // first_ok is not touched.
    const int16_t *target;
    // Register-table kernels (analyze_reg.cu): skip systems with fewer chains (the
    // 64-chain pass after the 32-lane lazy pass over the same deferral list)
    int32_t min_chains;
    // Candidate mode, optional (the 16- and 32-lane lazy kernels): each chain's
    // aggregates computed once for all candidates (paam_launch_chain_records),
    // four uint4 per chain
    const uint4 *chain_recs;
};

// Item i of a launch: system index and candidate index (0 outside candidate mode).
__device__ __forceinline__ void item_of(const AnalysisParams &p, int64_t i, int64_t &sys, int32_t &cand)
{
    if (p.K > 0) {
        if (p.sys_major) { // a 32-bit division where the index fits
            const int64_t q = (uint64_t)i <= 0xffffffffu ? (int64_t)((uint32_t)i / (uint32_t)p.K) : i / p.K;
            sys = q;
            cand = (int32_t)(i - q * p.K);
        } else {
            cand = (int32_t)(i / p.n_sys);
            sys = i - (int64_t)cand * p.n_sys;
        }
    } else {
        sys = i;
        cand = 0;
    }
    if (p.sys_order) sys = p.sys_order[sys];
}

// Items [0, n) of a launch for one group: the static grid-stride share, or
// batches from the work queue (see AnalysisParams), fetched by the group's
// first lane and broadcast.  One call site of f, so the system body is
// inlined once.
template <int G, typename F>
__device__ __forceinline__ void for_each_item(const AnalysisParams &p, int64_t n, int grp, int groups, int lane,
                                              unsigned gmask, F &&f)
{
    const bool q = p.queue_batch > 0;
    int64_t i = q ? 0 : (int64_t)blockIdx.x * groups + grp;
    int64_t end = q ? 0 : n; // the queue starts with an empty batch
    const int64_t step = q ? 1 : (int64_t)gridDim.x * groups;
    for (;;) {
        if (i >= end) {
            if (!q) break;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)p.queue_batch);
            base = __shfl_sync(gmask, base, 0, G);
            if ((int64_t)base >= n) break;
            i = (int64_t)base;
            end = i + p.queue_batch < n ? i + p.queue_batch : n;
        }
        f(i);
        i += step;
    }
}

// Candidate index visited in slot `slot` of system `sys`.
__device__ __forceinline__ int32_t cand_of(const AnalysisParams &p, int64_t sys, int32_t slot)
{
    return p.order ? p.order[sys * p.K + slot] : slot;
}

// Early exit of the search: is slot `cand` of `sys` above the best one found so far?
__device__ __forceinline__ bool cand_pruned(const AnalysisParams &p, int64_t sys, int32_t cand)
{
    if (p.K == 0 || !p.early) return false;
    return cand > *(volatile const int32_t *)(p.first_ok + sys);
}

// Batch-wide maxima recorded by validation; they decide which kernels an
// analysis needs (the 32-bit fast path covers every system when they fit).
enum { ST_TMAX = 0, ST_DMAX, ST_ECMAX, ST_SCMAX, ST_DELTAMAX, ST_ACCMAX, ST_COUNT };

// Streams, events and page-locked words of the pipelined host analysis
// (host_pipeline.cu), created on first use and kept for the context's life.
struct HostPipe {
    cudaStream_t in = nullptr, val = nullptr, an = nullptr, out = nullptr;
    cudaEvent_t *ev = nullptr;
    int n_ev = 0;
    void *words = nullptr; // page-locked
    size_t words_bytes = 0;
};

struct paam_ctx {
    int device;
    int n_sm;
    int max_smem_optin;
    cudaStream_t capture_stream; // private stream used to capture analysis graphs
    int32_t *d_err;        // validation: [0] code, [1] first bad system, [2] max chains, [3] max executors
    unsigned long long *d_stats; // validation: ST_* maxima
    HostPipe *pipe;
};

void paam_host_pipe_release(paam_ctx *ctx); // host_pipeline.cu

// Device copy of a validated batch: the same SoA/CSR arrays as
// paam_systems_view, all inside one allocation.
struct paam_batch {
    paam_ctx *ctx;
    int64_t n_sys, n_chain, n_cb, n_seg, n_exec;
    int64_t *sys_chain_off, *chain_cb_off, *cb_seg_off, *T, *D, *E, *A, *sys_exec_off;
    int32_t *prio, *exec, *exec_core, *exec_prio; // exec_prio NULL => derived
    uint8_t *spin;
    int32_t *acc; // accelerator of each segment; NULL when every segment uses accelerator 0
    int32_t max_chains; // largest chain count of any system
    int32_t max_exec;
    unsigned long long stats[ST_COUNT];
    // scratch for one analysis: [0] systems deferred to the wide configuration,
    // [1] systems deferred to the exact int64 kernel, both n_sys long; counts
    int32_t *list_big, *list_wide;
    int32_t *counts; // [0] big, [1] wide
    unsigned long long *queue; // [3] work-queue counters of the three passes (NULL: none)
    int32_t *sys_order;        // [n_sys] systems by increasing chain count within windows of consecutive systems (NULL: not built)
    void *block;
    size_t block_bytes;
    int cfg_index; // launch configuration (index into kLaunchCfgs)
    // the analysis captured as a CUDA graph, replayed while its key matches
    cudaGraphExec_t graph;
    int graph_kernels;
    struct {
        int64_t *R;
        uint8_t *status, *verdict;
        AnalysisParams p;
        int cfg_index;
    } graph_key;
};

// Read-only view handed to the kernels.
struct BatchDev {
    int64_t n_sys;
    const int64_t *__restrict__ sys_chain_off;
    const int64_t *__restrict__ chain_cb_off;
    const int64_t *__restrict__ cb_seg_off;
    const int64_t *__restrict__ T;
    const int64_t *__restrict__ D;
    const int64_t *__restrict__ E;
    const int64_t *__restrict__ A;
    const int64_t *__restrict__ sys_exec_off;
    const int32_t *__restrict__ prio;
    const int32_t *__restrict__ exec;
    const int32_t *__restrict__ exec_core;
    const int32_t *__restrict__ exec_prio;
    const uint8_t *__restrict__ spin;
    const int32_t *__restrict__ acc; // NULL: one accelerator
};

inline BatchDev batch_dev(const paam_batch *b)
{
    BatchDev d;
    d.n_sys = b->n_sys;
    d.sys_chain_off = b->sys_chain_off;
    d.chain_cb_off = b->chain_cb_off;
    d.cb_seg_off = b->cb_seg_off;
    d.T = b->T;
    d.D = b->D;
    d.E = b->E;
    d.A = b->A;
    d.sys_exec_off = b->sys_exec_off;
    d.prio = b->prio;
    d.exec = b->exec;
    d.exec_core = b->exec_core;
    d.exec_prio = b->exec_prio;
    d.spin = b->spin;
    d.acc = b->acc;
    return d;
}

// A launch configuration of the analysis: kernel family (0 = shared-memory
// tables, analyze_fast.cu; 1 = register tables, analyze_reg.cu), group width
// and chain-table size of the first pass, family and group width of the pass
// over systems with more chains (table size 64), CTA size.
struct LaunchCfg {
    int impl_small, g_small, maxn_small, impl_big, g_big, threads;
    int queue;  // 0: static grid-stride shares; > 0: work queue, items per fetch
    int binned; // 1: hand systems out by chain count within windows (batch->sys_order)
};

// Systems per window of the size binning (b->sys_order is sorted within each
// window of this many consecutive systems).
constexpr int kBinWindow = 8192;

// paam_rta_search_ordered continued from a given state (search.cu): first_ok
// holds K (nothing admitted yet) or -1 (skip the system) per system; the
// systems' slots are visited in `order` (the library's own, not checked) with
// stop at the first admitted candidate, and first_ok then holds its candidate
// index or -1.
int paam_search_ordered_from(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o, const int16_t *ranks,
                             int32_t Kc, int32_t nmax, const int32_t *order, int32_t K, int32_t *first_ok,
                             cudaStream_t stream);

// Builds b->sys_order (api.cu): a counting sort of the systems by chain count
// within each window of consecutive systems.
int paam_launch_bin_by_size(const paam_batch *b, int32_t *order, cudaStream_t stream);

// Register-table kernel with lazy per-chain work (analyze_lazy.cu): 16 lanes
// per system, first pass only (list == count == nullptr).  Systems over 16
// chains, or with a deadline at or above kLazyNarrowD inside the 32-bit
// bound, go to b->list_big; systems outside the 32-bit bound to b->list_wide.
// BLOCKS: resident blocks of 256 threads per SM the register budget is set for (4, 5, 6).
template <int BLOCKS>
int launch_lazy(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream);
constexpr unsigned long long kLazyNarrowD = (1ull << 27) - 16;
// The same kernel with 32 lanes per system over b->list_big (count b->counts[0]):
// systems of up to 32 chains inside the narrow bound; larger ones stay on the
// list for the 64-chain kernel (AnalysisParams::min_chains = 33), systems that
// are not narrow go to b->list_wide.
template <int BLOCKS>
int launch_lazy32(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream);
// The same analysis with one warp per system and two chains per lane
// (analyze_lazy64.cu) over b->list_big after the 32-lane pass: systems of
// AnalysisParams::min_chains (33) to 64 chains inside the narrow bound; those
// that are not narrow (a deadline at or above kLazyDeferWideD) go to b->list_wide.
int launch_lazy64(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream);
// The per-chain records of AnalysisParams::chain_recs for every chain of b
// (analyze_lazy.cu): the aggregates the lazy kernels compute before the
// relations, which do not depend on the priorities.
int paam_launch_chain_records(const paam_batch *b, const AnalysisParams &p, uint4 *recs, cudaStream_t stream);
// impl_big value of a launch configuration whose deferral list goes to the 32-lane
// lazy kernel and then, for systems over 32 chains, to the 64-chain lazy kernel
constexpr int kImplBigLazy32 = 9;
// the lowest deadline that the deferral passes of such a configuration send to the
// int64 kernel (the 64-chain pass's narrow bound)
constexpr unsigned long long kLazyDeferWideD = (1ull << 27) - 64;

// Register-table kernels (analyze_reg.cu): G lanes per system, CPL chains per lane.
template <int G, int CPL>
int launch_reg(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
               const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream);
extern const LaunchCfg kLaunchCfgs[];
extern const int kNumLaunchCfgs;
// Configuration of a batch before any autotuning: the lazy register-table
// kernel with five resident blocks per SM, work queue, systems by size, and
// the 32-lane lazy pass over the deferral list (the fastest on the 1M- and
// 4M-system workloads)
constexpr int kDefaultLaunchCfg = 28;

// Evaluations any one fixed-point recurrence may take before the analysis
// kernels stop it with PAAM_ST_ITERCAP.  Validation refuses systems whose
// bound (sum over chains of ceil(Dmax / T) plus 2) exceeds it, so for a loaded
// batch the cap is never reached; it bounds the kernels' running time all the
// same.
constexpr uint32_t kIterCap = (uint32_t)PAAM_MAX_ITER;

// Enqueue the whole analysis of a batch (analyze_fast.cu); *n_kernels receives
// the number of kernels it launched.
int paam_enqueue_analysis(const paam_batch *b, const AnalysisParams &p, const LaunchCfg &cfg, int64_t *R,
                          uint8_t *status, uint8_t *verdict, cudaStream_t stream, int *n_kernels);

// Validation kernel (api.cu): err = {code, first bad system, max chains, max
// executors} (initialise to {0, INT32_MAX, 0, 0}), stats = ST_* maxima (zeroed).
int paam_launch_validate(const paam_batch *b, const int32_t *acc, int32_t *err, unsigned long long *stats,
                         cudaStream_t stream);

// Half-open index ranges the systems of a validation must stay inside.
struct ValidateRange {
    int64_t chain_lo, chain_hi, cb_lo, cb_hi, seg_lo, seg_hi, exec_lo, exec_hi;
};

// The same over the systems of b (which may be a window of a larger batch:
// offsets stay absolute), each system's indices checked against r; sentinels
// adds the whole batch's first- and last-offset checks.
int paam_launch_validate_range(const paam_batch *b, const int32_t *acc, const ValidateRange &r, int sentinels,
                               int32_t *err, unsigned long long *stats, cudaStream_t stream);

// The lazy register-table analysis for batches with several accelerators
// (analyze_lazy_acc.cu): 16 lanes per system, one chain per lane, instantiated
// for the batch's accelerator count (2-4); systems over 16 chains, outside the
// 32-bit bound or not narrow go to b->list_wide (count b->counts[1]) for the
// int64 kernel.
int paam_launch_lazy_acc(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                         int64_t max_items, cudaStream_t stream);


// Chains up to which a search (or the Audsley-style seed) keeps each chain's
// aggregates for all its candidates (paam_launch_chain_records, 64 bytes per chain).
constexpr int64_t kRecChains = (int64_t)1 << 22;

// The safe reading of Lemma 4 (blocking_mode 1) in the lazy kernel (analyze_lazy.cu):
// systems of up to 16 chains and 128 segments inside the narrow 32-bit bound, one
// accelerator; the others are appended to b->list_wide (count b->counts[1]).
int paam_launch_lazy_safe(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                          int64_t max_items, cudaStream_t stream);

// Target mode of the lazy kernel (analyze_lazy.cu), reading p.chain_recs when set:
// candidates of systems with up to 16 chains inside the narrow 32-bit bound, one
// accelerator, Lemma 4 as printed; the others are appended to list (count *count)
// for the int64 kernel.
int paam_launch_lazy_target(const paam_batch *bt, const AnalysisParams &p, int32_t *list, int32_t *count,
                            int64_t max_items, cudaStream_t stream);

// Exact int64 kernel (analyze_wide.cu) over list[0 .. *count) or, with
// list == nullptr, over every system.
int paam_launch_wide(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st,
                     uint8_t *verdict, const int32_t *list, const int32_t *count, int64_t max_items,
                     cudaStream_t stream);
