// audsley.cu -- Audsley-style priority seed on the GPU: a greedy assignment
// of chain priorities from the lowest level up, each step decided by the
// exact analysis (Sec. IV-F, Theorem 1) of trial orders.
//
// At step j of a system with n chains (level l = n - 1 - j, rank 0 highest)
// every unassigned chain c is a trial: the chains already placed keep their
// ranks (all below l), c takes rank l and the other unassigned chains take
// ranks 0 .. l-1 in deadline-monotonic order (D ascending, ties by index).
// All trials of all systems are analysed at once in target mode, where a
// trial's verdict is whether c itself is schedulable and the analysis stops
// once c is done: the lazy kernel for systems of up to 16 chains inside its
// narrow 32-bit bound (one accelerator, Lemma 4 as printed; each chain's
// aggregates computed once per call for all its trials), the exact int64
// kernel for the rest.  The first passing c in index order takes level l; if
// none passes, the unassigned chain with the largest D (ties: highest index)
// does.  The admission test is not
// OPA-compatible (bucket ranks, blocking and the DEP rule depend on the whole
// order), so the result is a seed for the exact search, not an optimum.
#include "internal.cuh"

namespace {

// trial t of system s at step j: ranks row and target chain
__global__ void audsley_trials(BatchDev b, int32_t j, int32_t Kc, int32_t nmax, const int16_t *__restrict__ rank,
                               int16_t *__restrict__ trial, int16_t *__restrict__ target)
{
    const int64_t items = b.n_sys * (int64_t)Kc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items; i += stride) {
        const int64_t s = i / Kc;
        const int t = (int)(i - s * Kc);
        const int64_t c0 = b.sys_chain_off[s];
        const int n = (int)(b.sys_chain_off[s + 1] - c0);
        const int16_t *rs = rank + s * nmax;
        if (j >= n || t >= n - j) {
            target[i] = -1;
            continue;
        }
        int c = -1; // the t-th unassigned chain by index
        for (int k = 0, seen = 0; k < n; ++k)
            if (rs[k] < 0 && seen++ == t) {
                c = k;
                break;
            }
        const int level = n - 1 - j;
        int16_t *row = trial + i * nmax;
        for (int k = 0; k < n; ++k) {
            int16_t r;
            if (rs[k] >= 0) {
                r = rs[k];
            } else if (k == c) {
                r = (int16_t)level;
            } else { // position among the other unassigned chains, deadline-monotonic
                const int64_t Dk = b.D[c0 + k];
                int pos = 0;
                for (int u = 0; u < n; ++u) {
                    if (u == c || u == k || rs[u] >= 0) continue;
                    const int64_t Du = b.D[c0 + u];
                    pos += (Du < Dk || (Du == Dk && u < k));
                }
                r = (int16_t)pos;
            }
            row[k] = r;
        }
        target[i] = (int16_t)c;
    }
}

// step j: the first passing trial, else the largest deadline, takes level n-1-j
__global__ void audsley_pick(BatchDev b, int32_t j, int32_t Kc, int32_t nmax, int16_t *__restrict__ rank,
                             const int16_t *__restrict__ target, const uint8_t *__restrict__ ok)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < b.n_sys; s += stride) {
        const int64_t c0 = b.sys_chain_off[s];
        const int n = (int)(b.sys_chain_off[s + 1] - c0);
        if (j >= n) continue;
        int16_t *rs = rank + s * nmax;
        int chosen = -1;
        for (int t = 0; t < n - j && chosen < 0; ++t)
            if (ok[s * Kc + t]) chosen = target[s * Kc + t];
        if (chosen < 0)
            for (int k = 0; k < n; ++k)
                if (rs[k] < 0 && (chosen < 0 || b.D[c0 + k] >= b.D[c0 + chosen])) chosen = k;
        rs[chosen] = (int16_t)(n - 1 - j);
    }
}

__global__ void fill_i16(int16_t *p, int64_t n, int16_t v)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

constexpr size_t kTrialBytes = (size_t)512 << 20; // trial rank rows held at once

} // namespace

extern "C" int paam_rta_audsley_order(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o,
                                      int32_t nmax, int16_t *ranks_out, void *stream_)
{
    if (!ctx || !b || !o) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    if (o->n_buckets < 1 || o->eps_ns < 0 || o->kappa_ns < 0) return PAAM_E_INVAL;
    if (o->eps_ns > PAAM_MAX_OVERHEAD || o->kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (o->blocking_mode != 0 && o->blocking_mode != 1) return PAAM_E_INVAL;
    if (nmax < 1 || nmax < b->max_chains || (b->n_sys > 0 && !ranks_out)) return PAAM_E_INVAL;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    const int32_t Kc = b->max_chains > 0 ? b->max_chains : 1; // trials per system at step 0
    const size_t per_sys = (size_t)Kc * ((size_t)nmax * sizeof(int16_t) + sizeof(int16_t) + 1 + sizeof(int32_t));
    int64_t chunk = (int64_t)(kTrialBytes / per_sys);
    if (chunk < 1) chunk = 1;
    if (chunk > b->n_sys) chunk = b->n_sys;
    if (chunk * (int64_t)Kc > (int64_t)INT32_MAX) chunk = INT32_MAX / Kc;

    void *tmp = nullptr;
    const size_t trial_bytes = (size_t)chunk * Kc * nmax * sizeof(int16_t);
    const size_t target_bytes = (size_t)chunk * Kc * sizeof(int16_t);
    const size_t ok_bytes = (size_t)chunk * Kc;
    const size_t list_bytes = 4 * (size_t)chunk * Kc; // trials deferred to the int64 kernel
    // the lazy kernel serves one accelerator and Lemma 4 as printed; with up to
    // kRecChains chains, each chain's aggregates are computed once for all trials
    const bool lazy = !b->acc && o->blocking_mode == 0;
    const size_t rec_bytes = lazy && b->n_chain <= kRecChains ? 64 * (size_t)b->n_chain : 0;
    const size_t rec_off = (trial_bytes + target_bytes + ok_bytes + list_bytes + 512 + 255) & ~(size_t)255;
    if (cudaMallocAsync(&tmp, rec_off + rec_bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    int16_t *trial = (int16_t *)tmp;
    int16_t *target = (int16_t *)((char *)tmp + trial_bytes);
    uint8_t *ok = (uint8_t *)((char *)tmp + trial_bytes + target_bytes);
    int32_t *list = (int32_t *)(((uintptr_t)ok + ok_bytes + 15) & ~(uintptr_t)15);
    int32_t *err = (int32_t *)(((uintptr_t)(list + (size_t)chunk * Kc) + 15) & ~(uintptr_t)15);
    int32_t *count = err + 4;
    uint4 *recs = rec_bytes ? (uint4 *)((char *)tmp + rec_off) : nullptr;

    int rc = PAAM_OK;
    unsigned launches = 0;
    const int threads = 256;
    const int cap = 8 * ctx->n_sm;
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (recs && rc == PAAM_OK) {
        AnalysisParams pr = {};
        pr.eps = o->eps_ns;
        pr.kappa = o->kappa_ns;
        rc = paam_launch_chain_records(b, pr, recs, stream);
    }
    {
        const int64_t n = b->n_sys * (int64_t)nmax;
        int blocks = (int)((n + threads - 1) / threads);
        fill_i16<<<blocks < cap ? blocks : cap, threads, 0, stream>>>(ranks_out, n, (int16_t)-1);
        launches += 1;
    }
    for (int64_t s0 = 0; s0 < b->n_sys && rc == PAAM_OK; s0 += chunk) {
        paam_batch sub = *b; // systems [s0, s0 + m): chain offsets stay absolute
        const int64_t m = b->n_sys - s0 < chunk ? b->n_sys - s0 : chunk;
        sub.n_sys = m;
        sub.sys_chain_off = b->sys_chain_off + s0;
        sub.sys_exec_off = b->sys_exec_off + s0;
        sub.sys_order = nullptr; // the whole batch's order does not index a chunk
        const BatchDev bd = batch_dev(&sub);
        int16_t *rank = ranks_out + s0 * nmax;
        AnalysisParams p = {};
        p.n_buckets = o->n_buckets;
        p.eps = o->eps_ns;
        p.kappa = o->kappa_ns;
        p.blocking_mode = o->blocking_mode;
        p.K = Kc;
        p.Kc = Kc;
        p.ranks = trial;
        p.n_sys = m;
        p.nmax = nmax;
        p.cand_ok = ok;
        p.err = err;
        p.target = target;
        p.chain_recs = recs; // indexed by chain: the chunk's offsets are absolute
        const int64_t items = m * (int64_t)Kc;
        int tb = (int)((items + threads - 1) / threads);
        if (tb > cap) tb = cap;
        int sb = (int)((m + threads - 1) / threads);
        if (sb > cap) sb = cap;
        for (int32_t j = 0; j < b->max_chains && rc == PAAM_OK; ++j) {
            audsley_trials<<<tb, threads, 0, stream>>>(bd, j, Kc, nmax, rank, trial, target);
            if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
            if (rc == PAAM_OK && lazy) {
                if (cudaMemsetAsync(count, 0, sizeof(int32_t), stream) != cudaSuccess) rc = PAAM_E_CUDA;
                if (rc == PAAM_OK) rc = paam_launch_lazy_target(&sub, p, list, count, items, stream);
                if (rc == PAAM_OK)
                    rc = paam_launch_wide(&sub, p, nullptr, nullptr, nullptr, list, count, items, stream);
                launches += 1;
            } else if (rc == PAAM_OK) {
                rc = paam_launch_wide(&sub, p, nullptr, nullptr, nullptr, nullptr, nullptr, items, stream);
            }
            if (rc == PAAM_OK) {
                audsley_pick<<<sb, threads, 0, stream>>>(bd, j, Kc, nmax, rank, target, ok);
                if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
            }
            launches += 3;
        }
    }
    paam_count_launch(launches);
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream) != cudaSuccess) rc = PAAM_E_CUDA;
    cudaFreeAsync(tmp, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    return rc;
}
