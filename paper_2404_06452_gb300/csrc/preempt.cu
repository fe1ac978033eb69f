// preempt.cu -- measurement of the device preemption cost kappa between two
// CUDA stream priorities, by the method of the paper's GPU preemption
// measurement (Sec. V, "GPU Preemption Delay with Multiple Buckets"): the same
// kernel is launched on a low-priority stream and, right after, on a
// high-priority stream; the high-priority kernel's event-timed duration minus
// its duration when run alone is the preemption delay of that iteration.
//
// The four kernel kinds are written here (no library code): a shared-memory
// tiled fp32 matrix multiply, a block-and-atomic sum reduction, a vector add
// and a 256-bin histogram with per-block shared-memory bins.  Their grids are
// sized to the data (thousands of short blocks, as benchmark kernels are), so
// a high-priority kernel gets SMs as the low-priority kernel's running blocks
// retire: the delay measured is the hand-over time of stream priority.  Each
// kernel is bounded, with no waits between threads of different blocks.
#include <vector>

#include "internal.cuh"

namespace {

constexpr int kMatN = 1024;          // MatMul: [N x N] x [N x N], fp32
constexpr int64_t kVecN = 1 << 24;   // VectorAdd: 16M floats
constexpr int64_t kRedN = 1 << 26;   // Reduction: 64M floats
constexpr int64_t kHistN = 1 << 26;  // Histogram: 64M bytes

__global__ void __launch_bounds__(256) matmul_kernel(const float *A, const float *B, float *C, int n)
{
    __shared__ float As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    float acc = 0.0f;
    for (int k0 = 0; k0 < n; k0 += 16) {
        As[ty][tx] = A[(size_t)row * n + k0 + tx];
        Bs[ty][tx] = B[(size_t)(k0 + ty) * n + col];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    C[(size_t)row * n + col] = acc;
}

__global__ void __launch_bounds__(256) reduce_kernel(const float *x, int64_t n, float *out)
{
    __shared__ float part[8];
    float s = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) s += x[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 8) {
        s = part[threadIdx.x];
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(0xffu, s, off);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

__global__ void __launch_bounds__(256) vadd_kernel(const float *a, const float *b, float *c, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) c[i] = a[i] + b[i];
}

__global__ void __launch_bounds__(256) hist_kernel(const uint8_t *x, int64_t n, unsigned *bins)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) atomicAdd(&h[x[i]], 1u);
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&bins[threadIdx.x], h[threadIdx.x]);
}

__global__ void fill_kernel(float *x, int64_t n, float v)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        x[i] = v + (float)(i & 1023) * 1e-3f;
}

// one set of buffers for one kernel kind
struct KernelSet {
    int kind = 0;
    float *a = nullptr, *b = nullptr, *c = nullptr;
    unsigned *bins = nullptr;
    int grid = 0;

    int alloc(int k, int n_sm)
    {
        kind = k;
        // blocks sized to the data: 16 (reduction), 4 (vector add) or 64 (histogram) elements per thread
        grid = k == 1 ? (int)(kRedN / (256 * 16)) : k == 2 ? (int)(kVecN / (256 * 4)) : (int)(kHistN / (256 * 64));
        (void)n_sm;
        size_t na = 0, nb = 0, nc = 0;
        if (k == 0) na = nb = nc = (size_t)kMatN * kMatN;
        else if (k == 1) na = kRedN, nc = 1;
        else if (k == 2) na = nb = nc = kVecN;
        else na = kHistN / 4, nc = 0;
        // on any failure the buffers taken so far are freed before returning
        if ((na && cudaMalloc(&a, 4 * na) != cudaSuccess) || (nb && cudaMalloc(&b, 4 * nb) != cudaSuccess) ||
            (nc && cudaMalloc(&c, 4 * nc) != cudaSuccess) ||
            (k == 3 && cudaMalloc(&bins, 256 * sizeof(unsigned)) != cudaSuccess)) {
            cudaGetLastError();
            release();
            return PAAM_E_NOMEM;
        }
        fill_kernel<<<1024, 256>>>(a, (int64_t)na, 0.5f);
        if (nb) fill_kernel<<<1024, 256>>>(b, (int64_t)nb, 0.25f);
        if (cudaGetLastError() != cudaSuccess) {
            release();
            return PAAM_E_CUDA;
        }
        return PAAM_OK;
    }

    void launch(cudaStream_t s) const
    {
        if (kind == 0)
            matmul_kernel<<<dim3(kMatN / 16, kMatN / 16), 256, 0, s>>>(a, b, c, kMatN);
        else if (kind == 1)
            reduce_kernel<<<grid, 256, 0, s>>>(a, kRedN, c);
        else if (kind == 2)
            vadd_kernel<<<grid, 256, 0, s>>>(a, b, c, kVecN);
        else
            hist_kernel<<<grid, 256, 0, s>>>((const uint8_t *)a, kHistN, bins);
    }

    void release()
    {
        cudaFree(a);
        cudaFree(b);
        cudaFree(c);
        cudaFree(bins);
        a = b = c = nullptr;
        bins = nullptr;
    }
};

} // namespace

extern "C" int paam_measure_preemption(int device, int kind, int iters, float *delay_us, float *base_us)
{
    if (kind < 0 || kind > 3 || iters < 1 || !delay_us) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(device));
    int n_sm = 0, lo = 0, hi = 0;
    PAAM_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
    PAAM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi)); // hi is the numerically smaller, higher priority
    cudaStream_t s_lo = nullptr, s_hi = nullptr;
    cudaEvent_t ev[4] = {};
    KernelSet low, high;
    int rc = PAAM_OK;
    if (cudaStreamCreateWithPriority(&s_lo, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s_hi, cudaStreamNonBlocking, hi) != cudaSuccess)
        rc = PAAM_E_CUDA;
    for (int i = 0; i < 4 && rc == PAAM_OK; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK) rc = low.alloc(kind, n_sm);
    if (rc == PAAM_OK) rc = high.alloc(kind, n_sm);
    if (rc == PAAM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PAAM_E_CUDA;
    // warm-up: both sets once on their streams
    if (rc == PAAM_OK) {
        low.launch(s_lo);
        high.launch(s_hi);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch(2);
    }
    for (int it = 0; it < iters && rc == PAAM_OK; ++it) {
        // the low-priority kernel first, then at once the same kernel on the high-priority stream
        low.launch(s_lo);
        cudaEventRecord(ev[0], s_hi);
        high.launch(s_hi);
        cudaEventRecord(ev[1], s_hi);
        if (cudaDeviceSynchronize() != cudaSuccess) {
            rc = PAAM_E_CUDA;
            break;
        }
        // the high-priority kernel alone: the baseline
        cudaEventRecord(ev[2], s_hi);
        high.launch(s_hi);
        cudaEventRecord(ev[3], s_hi);
        if (cudaStreamSynchronize(s_hi) != cudaSuccess) {
            rc = PAAM_E_CUDA;
            break;
        }
        paam_count_launch(3);
        float t_pre = 0.f, t_base = 0.f;
        cudaEventElapsedTime(&t_pre, ev[0], ev[1]);
        cudaEventElapsedTime(&t_base, ev[2], ev[3]);
        delay_us[it] = (t_pre - t_base) * 1e3f;
        if (base_us) base_us[it] = t_base * 1e3f;
    }
    if (cudaGetLastError() != cudaSuccess && rc == PAAM_OK) rc = PAAM_E_CUDA;
    cudaDeviceSynchronize();
    low.release();
    high.release();
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (s_lo) cudaStreamDestroy(s_lo);
    if (s_hi) cudaStreamDestroy(s_hi);
    return rc;
}
