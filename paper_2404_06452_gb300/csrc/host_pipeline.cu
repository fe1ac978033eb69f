// host_pipeline.cu -- the analysis of a batch held in host memory, with the
// host-to-device copies overlapped with validation, analysis and the copies
// of the results back.
//
// The batch is split into chunks of whole systems, and four streams of the
// context carry the work:
//   in   every chunk's slices of the input arrays, enqueued at once, each
//        chunk followed by an event (the device arrays keep the host layout,
//        so offsets stay absolute and nothing is re-based);
//   val  per chunk, after its copy: the checks of paam_rta_load_systems with
//        each system's indices held inside the chunk's copied ranges, and the
//        chunk's validation words back to page-locked host memory;
//   an   per chunk, once the host has read its words: the analysis (Theorem
//        1, the kernels of paam_rta_analyze_batch chosen from the chunk's own
//        maxima);
//   out  per chunk, after its analysis: R, status and verdict to the host.
// The host only waits for validation words, which trail the copy engine by
// one small kernel, so chunk c is analysed while chunk c + 1 is copied and the
// results of earlier chunks travel back.  One call at a time per context.
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

constexpr size_t kMinChunkBytes = (size_t)64 << 20; // input bytes of the smallest automatic chunk
constexpr int kMaxChunks = 4096;
constexpr size_t kWords = 4 * sizeof(int32_t) + ST_COUNT * sizeof(unsigned long long); // per chunk

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// validation words of every chunk: {0, INT32_MAX, 0, 0} then zeroed maxima
__global__ void init_words(char *w, int64_t n_chunks)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_chunks; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t *e = (int32_t *)(w + kWords * (size_t)k);
        e[0] = 0;
        e[1] = INT32_MAX;
        e[2] = 0;
        e[3] = 0;
        unsigned long long *st = (unsigned long long *)(e + 4);
        for (int i = 0; i < ST_COUNT; ++i) st[i] = 0;
    }
}

// the context's streams, at least n_ev events and page-locked words of at least `bytes`
int pipe_get(paam_ctx *ctx, int n_ev, size_t bytes, HostPipe **out)
{
    if (!ctx->pipe) {
        HostPipe *p = new HostPipe();
        ctx->pipe = p;
        if (cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->val, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->an, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking) != cudaSuccess)
            return PAAM_E_CUDA;
    }
    HostPipe *p = ctx->pipe;
    if (!p->in || !p->val || !p->an || !p->out) return PAAM_E_CUDA;
    if (p->n_ev < n_ev) {
        cudaEvent_t *ev = (cudaEvent_t *)calloc((size_t)n_ev, sizeof(cudaEvent_t));
        if (!ev) return PAAM_E_NOMEM;
        for (int i = 0; i < p->n_ev; ++i) ev[i] = p->ev[i];
        free(p->ev);
        p->ev = ev;
        for (int i = p->n_ev; i < n_ev; ++i) {
            if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) return PAAM_E_CUDA;
            p->n_ev = i + 1;
        }
    }
    if (p->words_bytes < bytes) {
        if (p->words) cudaFreeHost(p->words);
        p->words = nullptr;
        p->words_bytes = 0;
        if (cudaMallocHost(&p->words, bytes) != cudaSuccess) return PAAM_E_NOMEM;
        p->words_bytes = bytes;
    }
    *out = p;
    return PAAM_OK;
}

} // namespace

void paam_host_pipe_release(paam_ctx *ctx)
{
    HostPipe *p = ctx->pipe;
    if (!p) return;
    for (int i = 0; i < p->n_ev; ++i)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    free(p->ev);
    if (p->words) cudaFreeHost(p->words);
    if (p->in) cudaStreamDestroy(p->in);
    if (p->val) cudaStreamDestroy(p->val);
    if (p->an) cudaStreamDestroy(p->an);
    if (p->out) cudaStreamDestroy(p->out);
    delete p;
    ctx->pipe = nullptr;
}

extern "C" int paam_rta_analyze_host(paam_ctx *ctx, const paam_systems_view *v, const paam_analysis_opts *o,
                                     int32_t launch_config, int64_t chunk_systems, int64_t *R, uint8_t *status,
                                     uint8_t *verdict)
{
    if (!ctx || !v || !o || v->is_device) return PAAM_E_INVAL;
    if (v->n_sys < 0 || v->n_chain < 0 || v->n_cb < 0 || v->n_seg < 0 || v->n_exec < 0) return PAAM_E_INVAL;
    if (!v->sys_chain_off || !v->chain_cb_off || !v->cb_seg_off || !v->sys_exec_off) return PAAM_E_INVAL;
    if ((v->n_chain > 0 && (!v->T || !v->D || !v->prio || !v->exec || !v->spin || !R || !status)) ||
        (v->n_cb > 0 && !v->E) || (v->n_seg > 0 && !v->A) || (v->n_exec > 0 && !v->exec_core))
        return PAAM_E_INVAL;
    if (launch_config < -1 || launch_config >= kNumLaunchCfgs) return PAAM_E_INVAL;
    if (o->n_buckets < 1 || o->eps_ns < 0 || o->kappa_ns < 0) return PAAM_E_INVAL;
    if (o->eps_ns > PAAM_MAX_OVERHEAD || o->kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (o->blocking_mode != 0 && o->blocking_mode != 1) return PAAM_E_INVAL;
    if (v->n_sys == 0) return PAAM_OK;
    // the whole batch's first and last offsets, read on the host
    if (v->sys_chain_off[0] != 0 || v->sys_exec_off[0] != 0 || v->chain_cb_off[0] != 0 || v->cb_seg_off[0] != 0 ||
        v->sys_chain_off[v->n_sys] != v->n_chain || v->sys_exec_off[v->n_sys] != v->n_exec ||
        v->chain_cb_off[v->n_chain] != v->n_cb || v->cb_seg_off[v->n_cb] != v->n_seg)
        return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));

    // ---- chunks of whole systems ------------------------------------------------
    const size_t in_bytes = 8 * (size_t)(2 * v->n_sys + 2) + (8 + 8 + 8 + 4 + 4 + 1) * (size_t)v->n_chain +
                            (8 + 8) * (size_t)v->n_cb + (8 + (v->acc ? 4 : 0)) * (size_t)v->n_seg +
                            (4 + (v->exec_prio ? 4 : 0)) * (size_t)v->n_exec;
    // chunk k covers systems [starts[k], starts[k + 1])
    std::vector<int64_t> starts{0};
    if (chunk_systems > 0) {
        int64_t per = chunk_systems < v->n_sys ? chunk_systems : v->n_sys;
        if ((v->n_sys + per - 1) / per > kMaxChunks) per = (v->n_sys + kMaxChunks - 1) / kMaxChunks;
        for (int64_t s = per; s < v->n_sys; s += per) starts.push_back(s);
    } else {
        // halving sizes: half the batch, a quarter, ... down to about
        // kMinChunkBytes of input, the rest in the last chunk.  Each copy has a
        // fixed cost on the link, so few chunks; the last one, whose analysis
        // and copies back follow the last byte in, is small; and each chunk's
        // analysis is shorter than the next chunk's copy.
        const double bytes_per_sys = (double)in_bytes / (double)v->n_sys;
        int64_t min_sys = (int64_t)((double)kMinChunkBytes / (bytes_per_sys > 1.0 ? bytes_per_sys : 1.0));
        if (min_sys < 1024) min_sys = 1024;
        int64_t s = 0;
        for (int64_t left = v->n_sys; left / 2 >= min_sys && left - left / 2 >= min_sys; left -= left / 2) {
            s += left / 2;
            starts.push_back(s);
        }
    }
    starts.push_back(v->n_sys);
    const int64_t n_chunks = (int64_t)starts.size() - 1;
    int64_t per = 0; // the largest chunk, which sizes the deferral lists
    for (int64_t k = 0; k < n_chunks; ++k)
        per = starts[(size_t)k + 1] - starts[(size_t)k] > per ? starts[(size_t)k + 1] - starts[(size_t)k] : per;
    struct Chunk {
        int64_t s0, s1, c0, c1, b0, b1, q0, q1, x0, x1;
    };
    std::vector<Chunk> ch((size_t)n_chunks);
    for (int64_t k = 0; k < n_chunks; ++k) {
        Chunk &c = ch[(size_t)k];
        c.s0 = starts[(size_t)k];
        c.s1 = starts[(size_t)k + 1];
        c.c0 = v->sys_chain_off[c.s0];
        c.c1 = v->sys_chain_off[c.s1];
        c.x0 = v->sys_exec_off[c.s0];
        c.x1 = v->sys_exec_off[c.s1];
        if (c.c0 < 0 || c.c1 < c.c0 || c.c1 > v->n_chain || c.x0 < 0 || c.x1 < c.x0 || c.x1 > v->n_exec)
            return PAAM_E_INVAL;
        c.b0 = v->chain_cb_off[c.c0];
        c.b1 = v->chain_cb_off[c.c1];
        if (c.b0 < 0 || c.b1 < c.b0 || c.b1 > v->n_cb) return PAAM_E_INVAL;
        c.q0 = v->cb_seg_off[c.b0];
        c.q1 = v->cb_seg_off[c.b1];
        if (c.q0 < 0 || c.q1 < c.q0 || c.q1 > v->n_seg) return PAAM_E_INVAL;
    }

    // ---- device block: inputs in the host layout, outputs, scratch, validation words
    HostPipe *pl = nullptr;
    int rc = pipe_get(ctx, (int)(3 * n_chunks + 1), kWords * (size_t)n_chunks, &pl);
    if (rc != PAAM_OK) return rc;
    cudaEvent_t *ev_val = pl->ev, *ev_in = pl->ev + n_chunks, *ev_an = pl->ev + 2 * n_chunks;
    cudaEvent_t *ev_alloc = pl->ev + 3 * n_chunks;

    paam_batch t = {}; // the whole batch's device view (offsets absolute)
    t.ctx = ctx;
    t.n_sys = v->n_sys;
    t.n_chain = v->n_chain;
    t.n_cb = v->n_cb;
    t.n_seg = v->n_seg;
    t.n_exec = v->n_exec;
    struct Arr {
        void **dst;
        const void *src;
        size_t elem;
        int64_t n;
    } arr[] = {
        {(void **)&t.sys_chain_off, v->sys_chain_off, 8, v->n_sys + 1},
        {(void **)&t.sys_exec_off, v->sys_exec_off, 8, v->n_sys + 1},
        {(void **)&t.chain_cb_off, v->chain_cb_off, 8, v->n_chain + 1},
        {(void **)&t.T, v->T, 8, v->n_chain},
        {(void **)&t.D, v->D, 8, v->n_chain},
        {(void **)&t.prio, v->prio, 4, v->n_chain},
        {(void **)&t.exec, v->exec, 4, v->n_chain},
        {(void **)&t.spin, v->spin, 1, v->n_chain},
        {(void **)&t.cb_seg_off, v->cb_seg_off, 8, v->n_cb + 1},
        {(void **)&t.E, v->E, 8, v->n_cb},
        {(void **)&t.A, v->A, 8, v->n_seg},
        {(void **)&t.acc, v->acc, 4, v->acc ? v->n_seg : 0},
        {(void **)&t.exec_core, v->exec_core, 4, v->n_exec},
        {(void **)&t.exec_prio, v->exec_prio, 4, v->exec_prio ? v->n_exec : 0},
    };
    const int n_arr = (int)(sizeof(arr) / sizeof(arr[0]));
    const size_t list_bytes = 4 * (size_t)per;
    size_t total = 0;
    for (int i = 0; i < n_arr; ++i) total += align256(arr[i].elem * (size_t)arr[i].n);
    total += align256(8 * (size_t)v->n_chain) + align256((size_t)v->n_chain) + align256((size_t)v->n_sys);
    total += 2 * align256(list_bytes) + 256 + align256(kWords * (size_t)n_chunks);
    void *dev = nullptr;
    if (cudaMallocAsync(&dev, total, pl->an) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    char *p = (char *)dev;
    for (int i = 0; i < n_arr; ++i) {
        *arr[i].dst = arr[i].n > 0 ? p : nullptr;
        p += align256(arr[i].elem * (size_t)arr[i].n);
    }
    int64_t *R_dev = (int64_t *)p;
    p += align256(8 * (size_t)v->n_chain);
    uint8_t *st_dev = (uint8_t *)p;
    p += align256((size_t)v->n_chain);
    uint8_t *vd_dev = (uint8_t *)p;
    p += align256((size_t)v->n_sys);
    t.list_big = (int32_t *)p;
    p += align256(list_bytes);
    t.list_wide = (int32_t *)p;
    p += align256(list_bytes);
    t.counts = (int32_t *)p;
    t.queue = (unsigned long long *)(t.counts + 8);
    p += 256;
    char *wdev = p;
    char *whost = (char *)pl->words;

    // the other streams start after the allocation (ordered on the analysis stream)
    if (cudaEventRecord(*ev_alloc, pl->an) != cudaSuccess || cudaStreamWaitEvent(pl->in, *ev_alloc, 0) != cudaSuccess ||
        cudaStreamWaitEvent(pl->val, *ev_alloc, 0) != cudaSuccess ||
        cudaStreamWaitEvent(pl->out, *ev_alloc, 0) != cudaSuccess)
        rc = PAAM_E_CUDA;
    if (rc == PAAM_OK) {
        init_words<<<1, 256, 0, pl->val>>>(wdev, n_chunks);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
    }
    unsigned launches = 1;

    // ---- copies of every chunk (copy stream), validation of every chunk as it lands
    // (validation stream), each chunk's words back to the page-locked buffer
    for (int64_t k = 0; k < n_chunks && rc == PAAM_OK; ++k) {
        const Chunk &c = ch[(size_t)k];
        // element ranges per array: systems (with the closing offset), chains, callbacks, segments, executors
        const int64_t lo[] = {c.s0, c.s0, c.c0, c.c0, c.c0, c.c0, c.c0, c.c0, c.b0, c.b0, c.q0, c.q0, c.x0, c.x0};
        const int64_t hi[] = {c.s1 + 1, c.s1 + 1, c.c1 + 1, c.c1, c.c1, c.c1, c.c1, c.c1,
                              c.b1 + 1, c.b1, c.q1, c.q1, c.x1, c.x1};
        for (int i = 0; i < n_arr && rc == PAAM_OK; ++i) {
            if (arr[i].n == 0 || hi[i] <= lo[i]) continue;
            const size_t off = arr[i].elem * (size_t)lo[i], bytes = arr[i].elem * (size_t)(hi[i] - lo[i]);
            if (cudaMemcpyAsync((char *)*arr[i].dst + off, (const char *)arr[i].src + off, bytes,
                                cudaMemcpyHostToDevice, pl->in) != cudaSuccess)
                rc = PAAM_E_CUDA;
        }
        if (rc != PAAM_OK || cudaEventRecord(ev_in[k], pl->in) != cudaSuccess) {
            rc = PAAM_E_CUDA;
            break;
        }
        paam_batch sub = t; // systems [s0, s1) of the batch
        sub.n_sys = c.s1 - c.s0;
        sub.sys_chain_off = t.sys_chain_off + c.s0;
        sub.sys_exec_off = t.sys_exec_off + c.s0;
        int32_t *err_d = (int32_t *)(wdev + kWords * (size_t)k);
        const ValidateRange r = {c.c0, c.c1, c.b0, c.b1, c.q0, c.q1, c.x0, c.x1};
        if (cudaStreamWaitEvent(pl->val, ev_in[k], 0) != cudaSuccess ||
            paam_launch_validate_range(&sub, t.acc, r, 0, err_d, (unsigned long long *)(err_d + 4), pl->val) !=
                PAAM_OK ||
            cudaMemcpyAsync(whost + kWords * (size_t)k, err_d, kWords, cudaMemcpyDeviceToHost, pl->val) !=
                cudaSuccess ||
            cudaEventRecord(ev_val[k], pl->val) != cudaSuccess)
            rc = PAAM_E_CUDA;
        launches += 1;
    }

    // ---- per chunk, once its words are on the host: the analysis and the copies back
    AnalysisParams ap = {};
    ap.n_buckets = o->n_buckets;
    ap.eps = o->eps_ns;
    ap.kappa = o->kappa_ns;
    ap.blocking_mode = o->blocking_mode;
    const LaunchCfg &cfg = kLaunchCfgs[launch_config < 0 ? kDefaultLaunchCfg : launch_config];
    for (int64_t k = 0; k < n_chunks && rc == PAAM_OK; ++k) {
        const Chunk &c = ch[(size_t)k];
        if (cudaEventSynchronize(ev_val[k]) != cudaSuccess) {
            rc = PAAM_E_CUDA;
            break;
        }
        const int32_t *err_h = (const int32_t *)(whost + kWords * (size_t)k);
        if (err_h[0] != 0) {
            rc = err_h[0];
            break;
        }
        paam_batch sub = t;
        sub.n_sys = c.s1 - c.s0;
        sub.sys_chain_off = t.sys_chain_off + c.s0;
        sub.sys_exec_off = t.sys_exec_off + c.s0;
        sub.max_chains = err_h[2];
        sub.max_exec = err_h[3];
        memcpy(sub.stats, err_h + 4, sizeof(sub.stats));
        sub.acc = sub.stats[ST_ACCMAX] > 0 ? t.acc : nullptr;
        int nk = 0;
        // the analysis stream already follows the allocation; the chunk's inputs are
        // complete because its validation (which followed the copy) is
        if (cudaStreamWaitEvent(pl->an, ev_val[k], 0) != cudaSuccess) {
            rc = PAAM_E_CUDA;
            break;
        }
        rc = paam_enqueue_analysis(&sub, ap, cfg, R_dev, st_dev, vd_dev + c.s0, pl->an, &nk);
        launches += (unsigned)nk;
        if (rc != PAAM_OK) break;
        if (cudaEventRecord(ev_an[k], pl->an) != cudaSuccess || cudaStreamWaitEvent(pl->out, ev_an[k], 0) != cudaSuccess ||
            (c.c1 > c.c0 &&
             (cudaMemcpyAsync(R + c.c0, R_dev + c.c0, 8 * (size_t)(c.c1 - c.c0), cudaMemcpyDeviceToHost, pl->out) !=
                  cudaSuccess ||
              cudaMemcpyAsync(status + c.c0, st_dev + c.c0, (size_t)(c.c1 - c.c0), cudaMemcpyDeviceToHost,
                              pl->out) != cudaSuccess)) ||
            (verdict && cudaMemcpyAsync(verdict + c.s0, vd_dev + c.s0, (size_t)(c.s1 - c.s0),
                                        cudaMemcpyDeviceToHost, pl->out) != cudaSuccess)) {
            rc = PAAM_E_CUDA;
            break;
        }
    }
    paam_count_launch(launches);
    // drain every stream, then hand the block back to the pool
    const bool drained = cudaStreamSynchronize(pl->in) == cudaSuccess && cudaStreamSynchronize(pl->val) == cudaSuccess &&
                         cudaStreamSynchronize(pl->out) == cudaSuccess && cudaStreamSynchronize(pl->an) == cudaSuccess;
    cudaFreeAsync(dev, pl->an);
    if (cudaStreamSynchronize(pl->an) != cudaSuccess || !drained) {
        if (rc == PAAM_OK) rc = PAAM_E_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess && rc == PAAM_OK) rc = PAAM_E_CUDA;
    return rc;
}
