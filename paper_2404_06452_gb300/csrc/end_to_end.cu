// end_to_end.cu -- end-to-end bounds of chains spanning several executors
// (Sec. IV-F): R* = sum of the sub-chains' response times + (m - 1) eps'.
//
// One thread per end-to-end chain walks its sub-chain list; the lists are
// short and contiguous, so the kernel only streams the CSR arrays and the
// analysis outputs it indexes.
#include "internal.cuh"

namespace {

__global__ void end_to_end_kernel(int64_t n_e2e, const int64_t *__restrict__ off,
                                  const int64_t *__restrict__ chain, const int64_t *__restrict__ D,
                                  int64_t eps_prime, int64_t n_chain, const int64_t *__restrict__ R,
                                  const uint8_t *__restrict__ st, int64_t *__restrict__ R_out,
                                  uint8_t *__restrict__ st_out, int32_t *err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e2e; e += stride) {
        const int64_t lo = off[e], hi = off[e + 1];
        if (lo < 0 || hi < lo) {
            atomicExch(err, PAAM_E_INVAL);
            R_out[e] = -1;
            st_out[e] = PAAM_ST_OVERRUN;
            continue;
        }
        // one hand-over between consecutive sub-chains; sums saturate at INT64_MAX (then above any D*)
        const int64_t hand = hi > lo ? hi - lo - 1 : 0;
        int64_t sum = (eps_prime > 0 && hand > INT64_MAX / eps_prime) ? INT64_MAX : hand * eps_prime;
        bool dep = false, over = false, bad = false;
        for (int64_t k = lo; k < hi; ++k) {
            const int64_t c = chain[k];
            if (c < 0 || c >= n_chain) {
                bad = true;
                break;
            }
            const uint8_t s = st[c];
            if (s == PAAM_ST_DEP) dep = true;
            else if (s != PAAM_ST_SCHED) over = true;
            else sum = R[c] > INT64_MAX - sum ? INT64_MAX : sum + R[c];
        }
        if (bad) {
            atomicExch(err, PAAM_E_INVAL);
            R_out[e] = -1;
            st_out[e] = PAAM_ST_OVERRUN;
            continue;
        }
        const bool ok = !dep && !over && sum <= D[e];
        R_out[e] = ok ? sum : -1;
        st_out[e] = ok ? PAAM_ST_SCHED : (dep ? PAAM_ST_DEP : PAAM_ST_OVERRUN);
    }
}

} // namespace

extern "C" int paam_rta_end_to_end(paam_ctx *ctx, const paam_batch *b, int64_t n_e2e, const int64_t *e2e_off,
                                   const int64_t *e2e_chain, const int64_t *D_e2e, int64_t eps_prime_ns,
                                   const int64_t *R, const uint8_t *status, int64_t *R_e2e, uint8_t *status_e2e,
                                   void *stream_)
{
    if (!ctx || !b || n_e2e < 0) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    if (eps_prime_ns < 0 || eps_prime_ns > PAAM_MAX_OVERHEAD) return PAAM_E_RANGE;
    if (n_e2e == 0) return PAAM_OK;
    if (!e2e_off || !e2e_chain || !D_e2e || !R || !status || !R_e2e || !status_e2e) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t stream = (cudaStream_t)stream_;
    int32_t *err = nullptr;
    if (cudaMallocAsync(&err, sizeof(int32_t), stream) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    int rc = PAAM_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int32_t), stream) != cudaSuccess) rc = PAAM_E_CUDA;
    int64_t blocks = (n_e2e + 255) / 256;
    if (blocks > 16 * (int64_t)ctx->n_sm) blocks = 16 * (int64_t)ctx->n_sm;
    if (rc == PAAM_OK) {
        end_to_end_kernel<<<(unsigned)blocks, 256, 0, stream>>>(n_e2e, e2e_off, e2e_chain, D_e2e, eps_prime_ns,
                                                                b->n_chain, R, status, R_e2e, status_e2e, err);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
    }
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream) != cudaSuccess) rc = PAAM_E_CUDA;
    cudaFreeAsync(err, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    return rc;
}
