// noalloc.cu -- the analysis entry point that allocates no memory.
//
// Some callers cannot allocate device memory when they need an admission
// test: a real-time executor whose control loop forbids allocation after
// start-up, a host that has handed its whole device-memory budget to another
// allocator, or an integration that must prove its memory use before it runs.
// paam_rta_analyze_noalloc serves them: it reads the caller's own device
// tables and writes the caller's own outputs, and keeps the small bookkeeping
// the analysis needs (validation words, batch maxima, the lists of systems
// deferred to wider kernels) in the fixed array below.  That array is part of
// the library's device image: every GPU that loads the library holds it until
// the process exits, whether or not this entry point is ever called.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
// layout in 32-bit words: [0, M) wide-configuration list, [M, 2M) int64 list,
// [2M, 2M + 2) their counts, [2M + 4, 2M + 8) validation words,
// [2M + 8, 2M + 8 + 2 * ST_COUNT) batch maxima (64-bit, 8-byte aligned)
constexpr int kM = PAAM_NOALLOC_MAX_SYS;
constexpr int kWords = 2 * kM + 8 + 2 * ST_COUNT + 6 + 6; // ... + three 64-bit work-queue counters

static __device__ __align__(256) int32_t g_noalloc_scratch[kWords];
static_assert(sizeof(g_noalloc_scratch) == (size_t)PAAM_NOALLOC_MAX_SYS * 8 + 128,
              "the header documents the array as PAAM_NOALLOC_MAX_SYS * 8 + 128 bytes");

struct DeviceSetup {
    bool ready;
    int n_sm, max_smem_optin;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// With the device current: its attributes (read on the first call only) and
// the scratch array's device address, looked up on every call so that it is
// right even after the device was reset.  Host code must never pass the
// array's own name to a kernel: on the host it is only a stand-in for the
// device symbol.
int setup_device(int dev, DeviceSetup *out, int32_t **scratch)
{
    if (dev < 0 || dev >= kMaxDevices) return PAAM_E_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        DeviceSetup &d = g_setup[dev];
        if (!d.ready) {
            PAAM_CUDA_TRY(cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev));
            PAAM_CUDA_TRY(cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            d.ready = true;
        }
        *out = d;
    }
    void *ptr = nullptr;
    PAAM_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    *scratch = (int32_t *)ptr;
    return PAAM_OK;
}

} // namespace

extern "C" int paam_rta_analyze_noalloc(const paam_systems_view *v, const paam_analysis_opts *o, int64_t *R,
                                        uint8_t *status, uint8_t *verdict, void *stream_)
{
    if (!v || !o) return PAAM_E_INVAL;
    if (!v->is_device) return PAAM_E_INVAL;
    if (v->n_sys < 0 || v->n_chain < 0 || v->n_cb < 0 || v->n_seg < 0 || v->n_exec < 0) return PAAM_E_INVAL;
    if (v->n_sys > PAAM_NOALLOC_MAX_SYS) return PAAM_E_RANGE;
    if (o->n_buckets < 1 || o->eps_ns < 0 || o->kappa_ns < 0) return PAAM_E_INVAL;
    if (o->eps_ns > PAAM_MAX_OVERHEAD || o->kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (o->blocking_mode != 0 && o->blocking_mode != 1) return PAAM_E_INVAL;
    if (!v->sys_chain_off || !v->chain_cb_off || !v->cb_seg_off || !v->sys_exec_off) return PAAM_E_INVAL;
    if ((v->n_chain > 0 && (!v->T || !v->D || !v->prio || !v->exec || !v->spin || !R || !status)) ||
        (v->n_cb > 0 && !v->E) || (v->n_seg > 0 && !v->A) || (v->n_exec > 0 && !v->exec_core))
        return PAAM_E_INVAL;
    if (v->n_sys == 0) return PAAM_OK;
    int dev = 0;
    PAAM_CUDA_TRY(cudaGetDevice(&dev));
    DeviceSetup dset = {};
    int32_t *scratch = nullptr;
    int rc = setup_device(dev, &dset, &scratch);
    if (rc != PAAM_OK) return rc;
    const DeviceSetup *d = &dset;
    cudaStream_t stream = (cudaStream_t)stream_;

    // a context and a batch that live on this stack frame and point at the
    // caller's tables and at the fixed scratch array
    paam_ctx ctx = {};
    ctx.device = dev;
    ctx.n_sm = d->n_sm;
    ctx.max_smem_optin = d->max_smem_optin;
    paam_batch b = {};
    b.ctx = &ctx;
    b.n_sys = v->n_sys;
    b.n_chain = v->n_chain;
    b.n_cb = v->n_cb;
    b.n_seg = v->n_seg;
    b.n_exec = v->n_exec;
    b.sys_chain_off = (int64_t *)v->sys_chain_off;
    b.chain_cb_off = (int64_t *)v->chain_cb_off;
    b.cb_seg_off = (int64_t *)v->cb_seg_off;
    b.T = (int64_t *)v->T;
    b.D = (int64_t *)v->D;
    b.E = (int64_t *)v->E;
    b.A = (int64_t *)v->A;
    b.sys_exec_off = (int64_t *)v->sys_exec_off;
    b.prio = (int32_t *)v->prio;
    b.exec = (int32_t *)v->exec;
    b.exec_core = (int32_t *)v->exec_core;
    b.exec_prio = (int32_t *)v->exec_prio;
    b.spin = (uint8_t *)v->spin;
    b.list_big = scratch;
    b.list_wide = scratch + kM;
    b.counts = scratch + 2 * kM;
    b.queue = (unsigned long long *)(scratch + 2 * kM + 8 + 2 * ST_COUNT + 6);
    int32_t *err = scratch + 2 * kM + 4;
    unsigned long long *stats = (unsigned long long *)(scratch + 2 * kM + 8);

    // the array keeps the previous call's contents: reset what must start at zero
    const int32_t err0[4] = {0, 0x7fffffff, 0, 0};
    PAAM_CUDA_TRY(cudaMemcpyAsync(err, err0, sizeof(err0), cudaMemcpyHostToDevice, stream));
    PAAM_CUDA_TRY(cudaMemsetAsync(stats, 0, ST_COUNT * sizeof(unsigned long long), stream));
    rc = paam_launch_validate(&b, v->acc, err, stats, stream);
    if (rc != PAAM_OK) return rc;
    int32_t herr[4];
    unsigned long long hstats[ST_COUNT];
    PAAM_CUDA_TRY(cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream));
    PAAM_CUDA_TRY(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, stream));
    PAAM_CUDA_TRY(cudaStreamSynchronize(stream));
    if (herr[0] != 0) return herr[0];
    b.max_chains = herr[2];
    b.max_exec = herr[3];
    for (int i = 0; i < ST_COUNT; ++i) b.stats[i] = hstats[i];
    b.acc = hstats[ST_ACCMAX] > 0 ? (int32_t *)v->acc : nullptr;

    AnalysisParams p = {};
    p.n_buckets = o->n_buckets;
    p.eps = o->eps_ns;
    p.kappa = o->kappa_ns;
    p.blocking_mode = o->blocking_mode;
    int nk = 0;
    rc = paam_enqueue_analysis(&b, p, kLaunchCfgs[kDefaultLaunchCfg], R, status, verdict, stream, &nk);
    if (rc == PAAM_OK) paam_count_launch((unsigned)nk);
    return rc;
}
