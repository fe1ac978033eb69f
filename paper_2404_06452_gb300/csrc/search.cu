// search.cu -- exact priority-assignment search over candidate orders.
//
// Every (system, candidate) pair is one exact analysis (Sec. IV-F) with the
// candidate's chain priorities and criticality-as-priority executor
// priorities (Sec. II-C); a candidate is schedulable when every chain is
// (the admission test of Sec. IV-A).  The analysis kernels run in candidate
// mode (see AnalysisParams): candidates are visited in order and each stops
// at its first unschedulable chain; with stop_at_first a candidate above the
// best one already found for its system is skipped.
#include <algorithm>
#include <chrono>

#include "internal.cuh"

namespace {


__global__ void search_init(int32_t *first_ok, int64_t n_sys, int32_t K, uint8_t *cand_ok, int64_t n_cand)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sys; i += stride) first_ok[i] = K;
    if (cand_ok)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_cand; i += stride) cand_ok[i] = 0;
}

// slot of the first admitted candidate -> its candidate index (or -1; a system
// that started at -1, with nothing to visit, keeps it)
__global__ void search_final(int32_t *first_ok, int64_t n_sys, int32_t K, const int32_t *order)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sys; i += stride) {
        const int32_t v = first_ok[i];
        first_ok[i] = (v < 0 || v >= K) ? -1 : (order ? order[i * K + v] : v);
    }
}

__global__ void check_order(const int32_t *order, int64_t n, int32_t Kc, int32_t *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (order[i] < 0 || order[i] >= Kc) atomicExch(err, PAAM_E_INVAL);
}

} // namespace

extern "C" int paam_rta_search_priorities(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o,
                                          const int16_t *ranks, int32_t K, int32_t nmax, int32_t stop_at_first,
                                          uint8_t *cand_ok, int32_t *first_ok, void *stream_)
{
    return paam_rta_search_ordered(ctx, b, o, ranks, K, nmax, nullptr, K, stop_at_first, cand_ok, first_ok,
                                   stream_);
}

namespace {

// resume: first_ok holds, per system, K (nothing admitted yet) or -1 (skip the
// system); its slots are visited with stop_at_first, the order is trusted (the
// library's own) and nothing else is initialised.
int search_ordered_impl(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o, const int16_t *ranks,
                        int32_t Kc, int32_t nmax, const int32_t *order, int32_t K, int32_t stop_at_first,
                        uint8_t *cand_ok, int32_t *first_ok, void *stream_, bool resume)
{
    if (!ctx || !b || !o || !first_ok) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    if (o->n_buckets < 1 || o->eps_ns < 0 || o->kappa_ns < 0) return PAAM_E_INVAL;
    if (o->eps_ns > PAAM_MAX_OVERHEAD || o->kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (o->blocking_mode != 0 && o->blocking_mode != 1) return PAAM_E_INVAL;
    if (Kc < 1 || K < 1 || (!order && K != Kc) || nmax < b->max_chains || nmax < 1 || (b->n_sys > 0 && !ranks))
        return PAAM_E_INVAL;
    if (b->n_sys * (int64_t)Kc > (int64_t)INT32_MAX) return PAAM_E_RANGE;
    if (b->n_sys * (int64_t)K > (int64_t)INT32_MAX) return PAAM_E_RANGE;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    const int64_t items = b->n_sys * (int64_t)K;

    // per-call scratch: the two deferral lists over items, their counts, an error word,
    // and (batches of up to kRecChains chains) each chain's aggregates, shared by
    // all its candidates
    void *tmp = nullptr;
    const size_t list_bytes = 4 * (size_t)items;
    const size_t rec_bytes = b->n_chain <= kRecChains ? 64 * (size_t)b->n_chain : 0;
    const size_t rec_off = (2 * list_bytes + 64 + 255) & ~(size_t)255; // 16-byte aligned records
    if (cudaMallocAsync(&tmp, rec_off + rec_bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    paam_batch bs = *b; // same tables, item-sized lists
    bs.list_big = (int32_t *)tmp;
    bs.list_wide = (int32_t *)((char *)tmp + list_bytes);
    bs.counts = (int32_t *)((char *)tmp + 2 * list_bytes);
    int32_t *err = bs.counts + 4;
    bs.queue = (unsigned long long *)(bs.counts + 8); // bytes 32..55 of the 64-byte tail
    bs.graph = nullptr;

    int rc = PAAM_OK;
    const int threads = 256;
    int blocks = (int)((items + threads - 1) / threads);
    if (blocks > 8 * ctx->n_sm) blocks = 8 * ctx->n_sm;
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (!resume) {
        search_init<<<blocks, threads, 0, stream>>>(first_ok, b->n_sys, K, cand_ok, b->n_sys * (int64_t)Kc);
        if (order) check_order<<<blocks, threads, 0, stream>>>(order, items, Kc, err);
    }
    if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
    if (order && !resume && rc == PAAM_OK) { // an out-of-range slot must not reach the analysis kernels
        int32_t herr = 0;
        if (cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            rc = PAAM_E_CUDA;
        else if (herr != 0)
            rc = herr;
    }

    AnalysisParams p = {};
    p.n_buckets = o->n_buckets;
    p.eps = o->eps_ns;
    p.kappa = o->kappa_ns;
    p.blocking_mode = o->blocking_mode;
    p.K = K;
    p.Kc = Kc;
    p.order = order;
    p.ranks = ranks;
    p.n_sys = b->n_sys;
    p.nmax = nmax;
    p.early = stop_at_first ? 1 : 0;
    p.sys_major = (!stop_at_first && !order) ? 1 : 0;
    p.cand_ok = cand_ok;
    p.first_ok = first_ok;
    p.err = err;
    int nk = 0;
    if (rec_bytes && rc == PAAM_OK) {
        p.chain_recs = (const uint4 *)((char *)tmp + rec_off);
        rc = paam_launch_chain_records(b, p, (uint4 *)p.chain_recs, stream);
        ++nk;
    }
    if (rc == PAAM_OK) rc = paam_enqueue_analysis(&bs, p, kLaunchCfgs[b->cfg_index], nullptr, nullptr, nullptr,
                                                  stream, &nk);
    if (rc == PAAM_OK) {
        search_final<<<blocks, threads, 0, stream>>>(first_ok, b->n_sys, K, order);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch((unsigned)nk + (resume ? 1 : (order ? 3 : 2)));
    }
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream) != cudaSuccess) rc = PAAM_E_CUDA;
    cudaFreeAsync(tmp, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    return rc;
}

} // namespace

extern "C" int paam_rta_search_ordered(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o,
                                       const int16_t *ranks, int32_t Kc, int32_t nmax, const int32_t *order,
                                       int32_t K, int32_t stop_at_first, uint8_t *cand_ok, int32_t *first_ok,
                                       void *stream_)
{
    return search_ordered_impl(ctx, b, o, ranks, Kc, nmax, order, K, stop_at_first, cand_ok, first_ok, stream_,
                               false);
}

int paam_search_ordered_from(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o, const int16_t *ranks,
                             int32_t Kc, int32_t nmax, const int32_t *order, int32_t K, int32_t *first_ok,
                             cudaStream_t stream)
{
    return search_ordered_impl(ctx, b, o, ranks, Kc, nmax, order, K, 1, nullptr, first_ok, stream, true);
}

// The search's own autotuner: every launch configuration timed on the search
// itself (host clock around the whole call, one warm-up and the median of five),
// the fastest kept on the batch.  The analysis autotuner times plain
// analyses, whose best shape can differ from the candidate mode's.
extern "C" int paam_rta_autotune_search(paam_ctx *ctx, paam_batch *b, const paam_analysis_opts *o,
                                        const int16_t *ranks, int32_t K, int32_t nmax, int32_t stop_at_first,
                                        void *stream_, float *times_ms, int max_out)
{
    if (!ctx || !b || !o) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    if (b->n_sys == 0) return b->cfg_index;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    int32_t *first = nullptr;
    if (cudaMallocAsync((void **)&first, 4 * (size_t)b->n_sys, stream) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    const int keep = b->cfg_index;
    int best = keep, rc = PAAM_OK;
    double best_ms = 1e300;
    constexpr int kReps = 5;
    for (int i = 0; i < kNumLaunchCfgs && rc == PAAM_OK; ++i) {
        b->cfg_index = i;
        double t[kReps + 1] = {};
        for (int rep = 0; rep <= kReps && rc == PAAM_OK; ++rep) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = paam_rta_search_priorities(ctx, b, o, ranks, K, nmax, stop_at_first, nullptr, first, stream_);
            t[rep] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        std::sort(t + 1, t + kReps + 1);
        const double med = t[1 + kReps / 2];
        if (times_ms && i < max_out) times_ms[i] = (float)med;
        if (med < best_ms) {
            best_ms = med;
            best = i;
        }
    }
    cudaFreeAsync(first, stream);
    cudaStreamSynchronize(stream);
    b->cfg_index = rc == PAAM_OK ? best : keep;
    return rc == PAAM_OK ? best : rc;
}
