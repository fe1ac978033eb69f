// api.cu -- context, batch loading with on-GPU validation, analysis entry.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.cuh"

static std::atomic<uint64_t> g_launches{0};

void paam_count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void paam_uncount_launch(unsigned n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

extern "C" uint64_t paam_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void paam_note_cuda_error(cudaError_t e, const char *expr, const char *file, int line)
{
    if (getenv("PAAM_VERBOSE"))
        fprintf(stderr, "paam: CUDA error %s (%s) at %s:%d: %s\n", cudaGetErrorName(e),
                cudaGetErrorString(e), file, line, expr);
}

extern "C" const char *paam_strerror(int code)
{
    switch (code) {
    case PAAM_OK: return "ok";
    case PAAM_E_INVAL: return "invalid input";
    case PAAM_E_RANGE: return "values out of the exact int64 range";
    case PAAM_E_NOMEM: return "out of memory";
    case PAAM_E_CUDA: return "CUDA runtime error";
    case PAAM_E_TIMEOUT: return "bounded device wait timed out";
    case PAAM_E_UNSUPPORTED: return "unsupported input or option";
    case PAAM_E_STATE: return "object used in the wrong state";
    default: return "unknown error";
    }
}

extern "C" int paam_create(paam_ctx **out, int device_ordinal)
{
    if (!out) return PAAM_E_INVAL;
    *out = nullptr;
    int n_dev = 0;
    PAAM_CUDA_TRY(cudaGetDeviceCount(&n_dev));
    if (device_ordinal < 0 || device_ordinal >= n_dev) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(device_ordinal));
    paam_ctx *c = (paam_ctx *)calloc(1, sizeof(paam_ctx));
    if (!c) return PAAM_E_NOMEM;
    c->device = device_ordinal;
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device_ordinal) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               device_ordinal) != cudaSuccess) {
        free(c);
        return PAAM_E_CUDA;
    }
    if (cudaMalloc(&c->d_err, 4 * sizeof(int32_t)) != cudaSuccess) {
        free(c);
        return PAAM_E_NOMEM;
    }
    if (cudaMalloc(&c->d_stats, ST_COUNT * sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(c->d_err);
        free(c);
        return PAAM_E_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(c->d_err);
        cudaFree(c->d_stats);
        free(c);
        return PAAM_E_CUDA;
    }
    // keep freed batch memory in the device pool so repeated load/free cycles are cheap
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device_ordinal) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return PAAM_OK;
}

extern "C" void paam_destroy(paam_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    paam_host_pipe_release(c);
    cudaFree(c->d_err);
    cudaFree(c->d_stats);
    cudaStreamDestroy(c->capture_stream);
    free(c);
}

// ---------------------------------------------------------------------------
// validation: one thread per system; the first failing code wins
// ---------------------------------------------------------------------------

struct ValidateArgs {
    BatchDev b;
    int64_t n_chain, n_cb, n_seg, n_exec;
    // index ranges a system's chains, callbacks, segments and executors must
    // lie in (the whole batch, or the part of it copied so far); sentinels:
    // also check the first and last offsets of the whole batch
    ValidateRange r;
    int sentinels;
    const int32_t *acc;
    int32_t *err; // [0] code, [1] first bad system (min), [2] max chains, [3] max executors
    unsigned long long *stats; // ST_* maxima
};

__device__ __forceinline__ void fail(int32_t *err, int32_t code, int64_t sys)
{
    atomicCAS(&err[0], 0, code);
    atomicMin(&err[1], (int32_t)(sys < 0x7fffffff ? sys : 0x7fffffff));
}

__global__ void validate_kernel(ValidateArgs a)
{
    const BatchDev &b = a.b;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long lmax[ST_COUNT] = {};
    int32_t nmax = 0, xmax = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < b.n_sys; s += stride) {
        if (s == 0 && a.sentinels) { // global sentinels
            if (b.sys_chain_off[0] != 0 || b.sys_exec_off[0] != 0 || b.chain_cb_off[0] != 0 ||
                b.cb_seg_off[0] != 0 || b.sys_chain_off[b.n_sys] != a.n_chain ||
                b.sys_exec_off[b.n_sys] != a.n_exec || b.chain_cb_off[a.n_chain] != a.n_cb ||
                b.cb_seg_off[a.n_cb] != a.n_seg) {
                fail(a.err, PAAM_E_INVAL, s);
                continue;
            }
        }
        const int64_t c0 = b.sys_chain_off[s], c1 = b.sys_chain_off[s + 1];
        const int64_t x0 = b.sys_exec_off[s], x1 = b.sys_exec_off[s + 1];
        if (c0 < a.r.chain_lo || c1 < c0 || c1 > a.r.chain_hi || x0 < a.r.exec_lo || x1 < x0 ||
            x1 > a.r.exec_hi) {
            fail(a.err, PAAM_E_INVAL, s);
            continue;
        }
        const int64_t n = c1 - c0, nx = x1 - x0;
        if (n > PAAM_MAX_CHAINS || (n > 0 && nx == 0)) {
            fail(a.err, PAAM_E_INVAL, s);
            continue;
        }
        nmax = (int32_t)n > nmax ? (int32_t)n : nmax;
        const int32_t nx32 = (int32_t)(nx < 0x7fffffff ? nx : 0x7fffffff);
        xmax = nx32 > xmax ? nx32 : xmax;
        // executors
        bool bad = false;
        for (int64_t x = x0; x < x1 && !bad; ++x) {
            if (b.exec_core[x] < 0) bad = true;
            if (b.exec_prio)
                for (int64_t y = x0; y < x && !bad; ++y)
                    if (b.exec_core[y] == b.exec_core[x] && b.exec_prio[y] == b.exec_prio[x]) bad = true;
        }
        if (bad) {
            fail(a.err, PAAM_E_INVAL, s);
            continue;
        }
        // chains, callbacks, segments; magnitudes for the range check
        double Dmax = 0.0, Tmin = 1e300, Cmax = 0.0, Base = 0.0, Emax_sys = 0.0, Mmax_sys = 0.0;
        const double OV = (double)PAAM_MAX_OVERHEAD;
        for (int64_t c = c0; c < c1 && !bad; ++c) {
            const int64_t T = b.T[c], D = b.D[c];
            if (T <= 0 || T > PAAM_MAX_TIME || D <= 0 || D > T || b.spin[c] > 1 || b.exec[c] < 0 ||
                b.exec[c] >= nx) {
                bad = true;
                break;
            }
            for (int64_t k = c0; k < c; ++k)
                if (b.prio[k] == b.prio[c]) bad = true;
            const int64_t b0 = b.chain_cb_off[c], b1 = b.chain_cb_off[c + 1];
            if (b0 < a.r.cb_lo || b1 < b0 || b1 > a.r.cb_hi) {
                bad = true;
                break;
            }
            double Ec = 0.0, Sc = 0.0, dc = 0.0;
            unsigned long long Ei = 0, Si = 0, di = 0;
            for (int64_t cb = b0; cb < b1 && !bad; ++cb) {
                const int64_t e = b.E[cb];
                const int64_t q0 = b.cb_seg_off[cb], q1 = b.cb_seg_off[cb + 1];
                if (e < 0 || e > PAAM_MAX_TIME || q0 < a.r.seg_lo || q1 < q0 || q1 > a.r.seg_hi) {
                    bad = true;
                    break;
                }
                Ec += (double)e;
                Ei += (unsigned long long)e;
                if ((double)e > Emax_sys) Emax_sys = (double)e;
                for (int64_t q = q0; q < q1; ++q) {
                    const int64_t av = b.A[q];
                    if (av < 0 || av > PAAM_MAX_TIME) {
                        bad = true;
                        break;
                    }
                    if (a.acc) { // one server per accelerator (R1), up to PAAM_MAX_ACC of them
                        const int32_t u = a.acc[q];
                        if (u < 0 || u >= PAAM_MAX_ACC) {
                            bad = true;
                            break;
                        }
                        lmax[ST_ACCMAX] = max(lmax[ST_ACCMAX], (unsigned long long)u);
                    }
                    const double as = (double)av + 2.0 * OV;
                    Sc += as;
                    dc += 1.0;
                    Si += (unsigned long long)av;
                    di += 1;
                    if (as > Mmax_sys) Mmax_sys = as;
                }
            }
            if ((double)D > Dmax) Dmax = (double)D;
            if ((double)T < Tmin) Tmin = (double)T;
            lmax[ST_TMAX] = max(lmax[ST_TMAX], (unsigned long long)T);
            lmax[ST_DMAX] = max(lmax[ST_DMAX], (unsigned long long)D);
            lmax[ST_ECMAX] = max(lmax[ST_ECMAX], Ei);
            lmax[ST_SCMAX] = max(lmax[ST_SCMAX], Si);
            lmax[ST_DELTAMAX] = max(lmax[ST_DELTAMAX], di);
            const double spin_or_d = (double)D > dc * OV ? (double)D : dc * OV;
            const double C = Ec + spin_or_d + Sc;
            if (C > Cmax) Cmax = C;
            const double base = Ec + Sc + dc * OV;
            if (base > Base) Base = base;
        }
        if (bad) {
            fail(a.err, PAAM_E_INVAL, s);
            continue;
        }
        if (n > 0) {
            // the largest value an iterate can take: interference over n chains with at most
            // ceil(Dmax/Tmin)+1 arrivals each, plus blocking and the chain's own demand
            double dseg_max = 0.0;
            for (int64_t c = c0; c < c1; ++c)
                dseg_max = fmax(dseg_max, (double)(b.cb_seg_off[b.chain_cb_off[c + 1]] -
                                                   b.cb_seg_off[b.chain_cb_off[c]]));
            const double m = ceil(Dmax / Tmin) + 1.0;
            const double bound = (double)n * m * Cmax + Base + Emax_sys + dseg_max * Mmax_sys + Dmax;
            if (!(bound < 2.305843009213694e18)) /* 2^61: margin under 2^62 */
                fail(a.err, PAAM_E_RANGE, s);
            // iteration bound: after its first step a recurrence rises only when an
            // arrival count ceil(t / T_h) + 1 (Lemma 1) has grown, at most
            // ceil(Dmax / T_h) times per chain h while t <= Dmax
            const uint64_t Dm = (uint64_t)Dmax; // exact: below 2^40
            uint64_t iters = 2;
            for (int64_t c = c0; c < c1 && iters <= (uint64_t)PAAM_MAX_ITER; ++c) {
                const uint64_t T = (uint64_t)b.T[c];
                iters += (Dm + T - 1) / T;
            }
            if (iters > (uint64_t)PAAM_MAX_ITER) fail(a.err, PAAM_E_RANGE, s);
        }
    }
    // one atomic per warp and statistic
    for (int off = 16; off > 0; off >>= 1) {
        nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, off));
        xmax = max(xmax, __shfl_xor_sync(0xffffffffu, xmax, off));
        for (int i = 0; i < ST_COUNT; ++i) lmax[i] = max(lmax[i], __shfl_xor_sync(0xffffffffu, lmax[i], off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (nmax) atomicMax(&a.err[2], nmax);
        if (xmax) atomicMax(&a.err[3], xmax);
        for (int i = 0; i < ST_COUNT; ++i)
            if (lmax[i]) atomicMax(&a.stats[i], lmax[i]);
    }

}

int paam_launch_validate(const paam_batch *b, const int32_t *acc, int32_t *err, unsigned long long *stats,
                         cudaStream_t stream)
{
    const ValidateRange whole = {0, b->n_chain, 0, b->n_cb, 0, b->n_seg, 0, b->n_exec};
    return paam_launch_validate_range(b, acc, whole, 1, err, stats, stream);
}

int paam_launch_validate_range(const paam_batch *b, const int32_t *acc, const ValidateRange &r, int sentinels,
                               int32_t *err, unsigned long long *stats, cudaStream_t stream)
{
    ValidateArgs a;
    a.b = batch_dev(b);
    a.n_chain = b->n_chain;
    a.n_cb = b->n_cb;
    a.n_seg = b->n_seg;
    a.n_exec = b->n_exec;
    a.r = r;
    a.sentinels = sentinels;
    a.acc = acc;
    a.err = err;
    a.stats = stats;
    const int threads = 256;
    int64_t blocks = (b->n_sys + threads - 1) / threads;
    if (blocks > 16 * (int64_t)b->ctx->n_sm) blocks = 16 * (int64_t)b->ctx->n_sm;
    if (blocks < 1) blocks = 1;
    validate_kernel<<<(unsigned)blocks, threads, 0, stream>>>(a);
    paam_count_launch();
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// size binning: within each window of kBinWindow consecutive systems, the
// systems by increasing chain count (a counting sort over the 65 possible
// counts; counts are clamped, so a batch that fails validation cannot index
// outside the table).  Neighbouring queue items then have about the same
// chain count, while the systems in flight at any time stay within a few
// windows, whose tables L2 holds: a sort over the whole batch scatters the
// reads and fetches each boundary sector twice.
// ---------------------------------------------------------------------------
namespace {

constexpr int kBins = PAAM_MAX_CHAINS + 1;

__device__ __forceinline__ int size_bin(const int64_t *off, int64_t s)
{
    const int64_t c = off[s + 1] - off[s];
    return c < 0 ? 0 : (c > PAAM_MAX_CHAINS ? PAAM_MAX_CHAINS : (int)c);
}

// one CTA per window: histogram, exclusive scan, scatter to order[w0 + position]
__global__ void bin_window(const int64_t *off, int64_t n_sys, int32_t *order)
{
    __shared__ int32_t h[kBins];
    const int64_t w0 = (int64_t)blockIdx.x * kBinWindow;
    const int64_t w1 = w0 + kBinWindow < n_sys ? w0 + kBinWindow : n_sys;
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t s = w0 + threadIdx.x; s < w1; s += blockDim.x) atomicAdd(&h[size_bin(off, s)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int i = 0; i < kBins; ++i) {
            const int32_t c = h[i];
            h[i] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t s = w0 + threadIdx.x; s < w1; s += blockDim.x)
        order[w0 + atomicAdd(&h[size_bin(off, s)], 1)] = (int32_t)s;
}

} // namespace

int paam_launch_bin_by_size(const paam_batch *b, int32_t *order, cudaStream_t stream)
{
    if (b->n_sys <= 0) return PAAM_OK;
    const int64_t blocks = (b->n_sys + kBinWindow - 1) / kBinWindow;
    bin_window<<<(unsigned)blocks, 256, 0, stream>>>(b->sys_chain_off, b->n_sys, order);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch(1);
    return PAAM_OK;
}

extern "C" int64_t paam_batch_n_sys(const paam_batch *b) { return b ? b->n_sys : 0; }
extern "C" int64_t paam_batch_n_chain(const paam_batch *b) { return b ? b->n_chain : 0; }

extern "C" void paam_batch_free(paam_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->ctx->device);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->block) cudaFree(b->block);
    free(b);
}

extern "C" int paam_rta_load_systems(paam_ctx *ctx, const paam_systems_view *v, void *stream_,
                                     paam_batch **out)
{
    if (!out) return PAAM_E_INVAL;
    *out = nullptr;
    if (!ctx || !v) return PAAM_E_INVAL;
    if (v->n_sys < 0 || v->n_chain < 0 || v->n_cb < 0 || v->n_seg < 0 || v->n_exec < 0)
        return PAAM_E_INVAL;
    if (!v->sys_chain_off || !v->chain_cb_off || !v->cb_seg_off || !v->sys_exec_off)
        return PAAM_E_INVAL;
    if ((v->n_chain > 0 && (!v->T || !v->D || !v->prio || !v->exec || !v->spin)) ||
        (v->n_cb > 0 && !v->E) || (v->n_seg > 0 && !v->A) || (v->n_exec > 0 && !v->exec_core))
        return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;

    paam_batch *b = (paam_batch *)calloc(1, sizeof(paam_batch));
    if (!b) return PAAM_E_NOMEM;
    b->ctx = ctx;
    b->cfg_index = kDefaultLaunchCfg;
    b->n_sys = v->n_sys;
    b->n_chain = v->n_chain;
    b->n_cb = v->n_cb;
    b->n_seg = v->n_seg;
    b->n_exec = v->n_exec;

    struct Item {
        void **dst;
        const void *src;
        size_t bytes;
    } items[] = {
        {(void **)&b->sys_chain_off, v->sys_chain_off, 8 * (size_t)(v->n_sys + 1)},
        {(void **)&b->chain_cb_off, v->chain_cb_off, 8 * (size_t)(v->n_chain + 1)},
        {(void **)&b->cb_seg_off, v->cb_seg_off, 8 * (size_t)(v->n_cb + 1)},
        {(void **)&b->T, v->T, 8 * (size_t)v->n_chain},
        {(void **)&b->D, v->D, 8 * (size_t)v->n_chain},
        {(void **)&b->E, v->E, 8 * (size_t)v->n_cb},
        {(void **)&b->A, v->A, 8 * (size_t)v->n_seg},
        {(void **)&b->sys_exec_off, v->sys_exec_off, 8 * (size_t)(v->n_sys + 1)},
        {(void **)&b->prio, v->prio, 4 * (size_t)v->n_chain},
        {(void **)&b->exec, v->exec, 4 * (size_t)v->n_chain},
        {(void **)&b->exec_core, v->exec_core, 4 * (size_t)v->n_exec},
        {(void **)&b->exec_prio, v->exec_prio, v->exec_prio ? 4 * (size_t)v->n_exec : 0},
        {(void **)&b->spin, v->spin, (size_t)v->n_chain},
    };
    const int n_items = (int)(sizeof(items) / sizeof(items[0]));
    // acc is validated from a temporary copy, not kept (one accelerator per system)
    const size_t acc_bytes = v->acc ? 4 * (size_t)v->n_seg : 0;
    size_t total = 0;
    for (int i = 0; i < n_items; ++i) total += align_up(items[i].bytes);
    total += align_up(acc_bytes) + 256;
    const size_t list_bytes = 4 * (size_t)(v->n_sys > 0 ? v->n_sys : 1);
    total += 2 * align_up(list_bytes) + 256;
    total += align_up(list_bytes); // size-binned order
    if (cudaMallocAsync(&b->block, total, stream) != cudaSuccess) {
        cudaGetLastError();
        free(b);
        return PAAM_E_NOMEM;
    }
    b->block_bytes = total;
    char *p = (char *)b->block;
    const cudaMemcpyKind kind = v->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int rc = PAAM_OK;
    for (int i = 0; i < n_items; ++i) {
        if (items[i].src == nullptr && items[i].bytes == 0) {
            *items[i].dst = nullptr;
            continue;
        }
        *items[i].dst = p;
        if (items[i].bytes &&
            cudaMemcpyAsync(p, items[i].src, items[i].bytes, kind, stream) != cudaSuccess)
            rc = PAAM_E_CUDA;
        p += align_up(items[i].bytes);
    }
    int32_t *acc_dev = nullptr;
    if (acc_bytes) {
        acc_dev = (int32_t *)p;
        if (cudaMemcpyAsync(acc_dev, v->acc, acc_bytes, kind, stream) != cudaSuccess) rc = PAAM_E_CUDA;
    }
    p += align_up(acc_bytes);
    b->list_big = (int32_t *)p;
    p += align_up(list_bytes);
    b->list_wide = (int32_t *)p;
    p += align_up(list_bytes);
    b->counts = (int32_t *)p;
    b->queue = (unsigned long long *)(b->counts + 8); // inside the 256-byte counts area
    p += 256;
    b->sys_order = (int32_t *)p;
    int32_t h_err[4] = {0, 0x7fffffff, 0, 0};
    if (rc == PAAM_OK && b->n_sys > 0) {
        if (cudaMemcpyAsync(ctx->d_err, h_err, sizeof(h_err), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemsetAsync(ctx->d_stats, 0, ST_COUNT * sizeof(unsigned long long), stream) != cudaSuccess)
            rc = PAAM_E_CUDA;
        if (paam_launch_validate(b, acc_dev, ctx->d_err, ctx->d_stats, stream) != PAAM_OK) rc = PAAM_E_CUDA;
        if (rc == PAAM_OK && paam_launch_bin_by_size(b, b->sys_order, stream) != PAAM_OK)
            rc = PAAM_E_CUDA;
        if (rc == PAAM_OK &&
            (cudaMemcpyAsync(h_err, ctx->d_err, sizeof(h_err), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
             cudaMemcpyAsync(b->stats, ctx->d_stats, sizeof(b->stats), cudaMemcpyDeviceToHost, stream) !=
                 cudaSuccess))
            rc = PAAM_E_CUDA;
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && h_err[0] != 0) rc = h_err[0];
    if (rc != PAAM_OK) {
        cudaFree(b->block);
        free(b);
        return rc;
    }
    b->max_chains = h_err[2];
    b->max_exec = h_err[3];
    b->acc = b->stats[ST_ACCMAX] > 0 ? acc_dev : nullptr; // kept only when a second accelerator is used
    *out = b;
    return PAAM_OK;
}

static int check_opts(const paam_analysis_opts *o)
{
    if (o->n_buckets < 1) return PAAM_E_INVAL;
    if (o->eps_ns < 0 || o->kappa_ns < 0) return PAAM_E_INVAL;
    if (o->eps_ns > PAAM_MAX_OVERHEAD || o->kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (o->blocking_mode != 0 && o->blocking_mode != 1) return PAAM_E_INVAL;
    return PAAM_OK;
}

static AnalysisParams params_of(const paam_analysis_opts *o)
{
    AnalysisParams p = {};
    p.n_buckets = o->n_buckets;
    p.eps = o->eps_ns;
    p.kappa = o->kappa_ns;
    p.blocking_mode = o->blocking_mode;
    return p;
}

extern "C" int paam_rta_analyze_batch(paam_ctx *ctx, const paam_batch *b, const paam_analysis_opts *o,
                                      int64_t *R, uint8_t *status, uint8_t *verdict, void *stream_)
{
    if (!ctx || !b || !o) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    int rc = check_opts(o);
    if (rc != PAAM_OK) return rc;
    if (b->n_chain > 0 && (!R || !status)) return PAAM_E_INVAL;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    const AnalysisParams p = params_of(o);
    paam_batch *bm = const_cast<paam_batch *>(b); // the captured graph is a cache inside the handle
    const bool same = bm->graph && bm->graph_key.R == R && bm->graph_key.status == status &&
                      bm->graph_key.verdict == verdict && bm->graph_key.cfg_index == bm->cfg_index &&
                      bm->graph_key.p.n_buckets == p.n_buckets && bm->graph_key.p.eps == p.eps &&
                      bm->graph_key.p.kappa == p.kappa && bm->graph_key.p.blocking_mode == p.blocking_mode;
    if (!same) {
        if (bm->graph) {
            cudaGraphExecDestroy(bm->graph);
            bm->graph = nullptr;
        }
        cudaStream_t cs = ctx->capture_stream;
        PAAM_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int nk = 0;
        rc = paam_enqueue_analysis(b, p, kLaunchCfgs[bm->cfg_index], R, status, verdict, cs, &nk);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (rc != PAAM_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != PAAM_OK ? rc : PAAM_E_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&bm->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            bm->graph = nullptr;
            return PAAM_E_CUDA;
        }
        bm->graph_kernels = nk;
        bm->graph_key.R = R;
        bm->graph_key.status = status;
        bm->graph_key.verdict = verdict;
        bm->graph_key.p = p;
        bm->graph_key.cfg_index = bm->cfg_index;
    }
    PAAM_CUDA_TRY(cudaGraphLaunch(bm->graph, stream));
    paam_count_launch((unsigned)bm->graph_kernels);
    return PAAM_OK;
}

extern "C" int paam_rta_num_launch_configs(void) { return kNumLaunchCfgs; }

extern "C" int paam_rta_set_launch_config(paam_batch *b, int index)
{
    if (!b || index < 0 || index >= kNumLaunchCfgs) return PAAM_E_INVAL;
    b->cfg_index = index;
    return PAAM_OK;
}

extern "C" int paam_rta_get_launch_config(const paam_batch *b) { return b ? b->cfg_index : -1; }

extern "C" int paam_rta_autotune(paam_ctx *ctx, paam_batch *b, const paam_analysis_opts *o, void *stream_,
                                 float *times_ms, int max_out)
{
    if (!ctx || !b || !o) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    int rc = check_opts(o);
    if (rc != PAAM_OK) return rc;
    if (b->n_sys == 0) return 0;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    const AnalysisParams p = params_of(o);
    void *tmp = nullptr;
    const size_t rb = 8 * (size_t)b->n_chain, sb = (size_t)b->n_chain, vb = (size_t)b->n_sys;
    if (cudaMallocAsync(&tmp, rb + sb + vb + 64, stream) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    int64_t *R = (int64_t *)tmp;
    uint8_t *st = (uint8_t *)tmp + rb;
    uint8_t *v = st + sb;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    constexpr int kReps = 5; // timed runs per configuration, after one warm-up run
    for (int i = 0; i < kNumLaunchCfgs && rc == PAAM_OK; ++i) {
        float t[kReps + 1] = {};
        for (int rep = 0; rep <= kReps && rc == PAAM_OK; ++rep) {
            cudaEventRecord(e0, stream);
            rc = paam_enqueue_analysis(b, p, kLaunchCfgs[i], R, st, v, stream, nullptr);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = PAAM_E_CUDA;
            cudaEventElapsedTime(&t[rep], e0, e1);
        }
        // median of the timed runs (the first warms caches and loads the code): a
        // configuration that is fast only now and then does not win on one lucky run
        float *r = t + 1;
        for (int a = 1; a < kReps; ++a)
            for (int c = a; c > 0 && r[c] < r[c - 1]; --c) {
                const float x = r[c];
                r[c] = r[c - 1];
                r[c - 1] = x;
            }
        const float med = r[kReps / 2];
        if (times_ms && i < max_out) times_ms[i] = med;
        if (med < best_ms) {
            best_ms = med;
            best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(tmp, stream);
    cudaStreamSynchronize(stream);
    if (rc != PAAM_OK) return rc;
    b->cfg_index = best;
    return best;
}
