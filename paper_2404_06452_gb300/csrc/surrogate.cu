// surrogate.cu -- the learned ranking model of the priority-assignment search.
//
// A multilayer perceptron 1024 -> 256 -> 256 -> 256 -> 64 with GELU hidden
// layers reads the 64 x 16 chain features of one (system, candidate) and
// predicts, per chain, the exact analysis' response time relative to the
// deadline (clip(R / D, 0, 2); 2 when not schedulable).  Weights are kept in
// fp32 (with AdamW moments) and used as bf16 copies by the tensor-core GEMMs
// (mlp_gemm.cu), which accumulate in fp32.  Training labels come from the
// exact analysis kernels; a candidate's score is its largest predicted
// R / D, and candidates are confirmed in increasing score by the exact search
// (paam_rta_search_ordered), so every admission stays exact.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mlp.cuh"

struct paam_model {
    paam_ctx *ctx;
    int64_t step;
    void *block;
    size_t block_bytes;
    float *W[4], *bias[4], *mW[4], *vW[4], *mb[4], *vb[4];
    float *gW[4], *gb[4]; // gradients of the last paam_surrogate_grad call
    __nv_bfloat16 *Wb[4], *WbT[4];
};

namespace {

constexpr int NL = 4;
constexpr int IN[NL] = {1024, 256, 256, 256};
constexpr int OUT[NL] = {256, 256, 256, 64};
constexpr int NCH = 64, NF = 16, XW = NCH * NF;

size_t n_params()
{
    size_t n = 0;
    for (int l = 0; l < NL; ++l) n += (size_t)IN[l] * OUT[l] + OUT[l];
    return n;
}

// ---- labels: clip(R / D, 0, 2) for schedulable chains, 2 otherwise, -1 for padding
__global__ void labels_kernel(BatchDev b, const int64_t *R, const uint8_t *status, float *L)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b.n_sys * NCH; i += stride) {
        const int64_t sys = i / NCH;
        const int c = (int)(i % NCH);
        const int64_t c0 = b.sys_chain_off[sys];
        const int n = (int)(b.sys_chain_off[sys + 1] - c0);
        float y = -1.0f;
        if (c < n) {
            const int64_t g = c0 + c;
            y = status[g] == PAAM_ST_SCHED ? fminf((float)((double)R[g] / (double)b.D[g]), 2.0f) : 2.0f;
        }
        L[i] = y;
    }
}

// ---- minibatch gather: rows idx[r] (-1 = padding) of X into Xb and, transposed,
// XbT ([1024][rows]), and of L into Lb; counts the valid labels into *count.
// One block per 64 x 64 tile (grid: 16 column tiles x rows / 64 row tiles):
// 16-byte loads and row-major stores, the transposed stores as 16-byte runs
// of 8 rows, read column-wise from a shared-memory copy of the tile.
constexpr int kTT = 64;
constexpr int kTP = kTT + 8; // row pitch of a shared tile (u16): 16-byte aligned rows

__device__ __forceinline__ void store_tile_t(const unsigned short (*t)[kTP], __nv_bfloat16 *out, int64_t ld,
                                             int64_t c0, int64_t r0)
{
    // out[(c0 + c) * ld + r0 + 8 rc + i] = t[8 rc + i][c]: a warp writes 32 columns
    for (int e = threadIdx.x; e < kTT * kTT / 8; e += blockDim.x) {
        const int c = e % kTT, rc = e / kTT;
        uint4 v;
        unsigned short *h = reinterpret_cast<unsigned short *>(&v);
#pragma unroll
        for (int i = 0; i < 8; ++i) h[i] = t[8 * rc + i][c];
        *reinterpret_cast<uint4 *>(out + (c0 + c) * ld + r0 + 8 * rc) = v;
    }
}

__global__ void __launch_bounds__(256) gather_kernel(const __nv_bfloat16 *X, const float *L, const int64_t *idx,
                                                     int rows, __nv_bfloat16 *Xb, __nv_bfloat16 *XbT, float *Lb,
                                                     float *count)
{
    __shared__ __align__(16) unsigned short t[kTT][kTP];
    static_assert(kTT * kTT / 8 == 2 * 256, "two 16-byte loads per thread");
    const int c0 = blockIdx.x * kTT, r0 = blockIdx.y * kTT;
    uint4 v[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int e = threadIdx.x + 256 * j, r = e / (kTT / 8), part = e % (kTT / 8);
        const int64_t src = idx[r0 + r];
        v[j] = src >= 0 ? *reinterpret_cast<const uint4 *>(X + src * XW + c0 + 8 * part) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int e = threadIdx.x + 256 * j, r = e / (kTT / 8), part = e % (kTT / 8);
        *reinterpret_cast<uint4 *>(Xb + (int64_t)(r0 + r) * XW + c0 + 8 * part) = v[j];
        *reinterpret_cast<uint4 *>(&t[r][8 * part]) = v[j];
    }
    if (XbT) {
        __syncthreads();
        store_tile_t(t, XbT, rows, c0, r0);
    }
    if (blockIdx.x != 0) return;
    // the tile's labels: 64 rows x 16 float4
    static_assert(kTT * NCH / 4 == 4 * 256, "four label loads per thread");
    float4 y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int e = threadIdx.x + 256 * j, r = e / (NCH / 4), q = e % (NCH / 4);
        const int64_t src = idx[r0 + r];
        y[j] = src >= 0 ? *reinterpret_cast<const float4 *>(L + src * NCH + 4 * q) : make_float4(-1.f, -1.f, -1.f, -1.f);
    }
    float cnt = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int e = threadIdx.x + 256 * j, r = e / (NCH / 4), q = e % (NCH / 4);
        *reinterpret_cast<float4 *>(Lb + (int64_t)(r0 + r) * NCH + 4 * q) = y[j];
        cnt += (y[j].x >= 0.0f) + (y[j].y >= 0.0f) + (y[j].z >= 0.0f) + (y[j].w >= 0.0f);
    }
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((threadIdx.x & 31) == 0 && cnt > 0.0f) atomicAdd(count, cnt);
}

// ---- masked mean-squared error and its gradient dY ([rows][64]) and dY^T
// ([64][rows]); one block per 64 rows
__global__ void __launch_bounds__(256) loss_kernel(const float *Y, const float *Lb, int rows, const float *count,
                                                   __nv_bfloat16 *dY, __nv_bfloat16 *dYT, float *loss_sum)
{
    __shared__ __align__(16) unsigned short t[kTT][kTP];
    __shared__ float part[8];
    static_assert(kTT * NCH / 4 == 4 * 256, "four float4 per thread");
    const int r0 = blockIdx.x * kTT;
    float4 yv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t i = (int64_t)r0 * NCH + 4 * (threadIdx.x + 256 * j);
        yv[j] = *reinterpret_cast<const float4 *>(Y + i);
        lv[j] = *reinterpret_cast<const float4 *>(Lb + i);
    }
    const float inv = 1.0f / fmaxf(*count, 1.0f);
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int e = threadIdx.x + 256 * j, r = e / (NCH / 4), c = 4 * (e % (NCH / 4));
        const float yy[4] = {yv[j].x, yv[j].y, yv[j].z, yv[j].w}, ll[4] = {lv[j].x, lv[j].y, lv[j].z, lv[j].w};
        unsigned short g[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float d = ll[q] >= 0.0f ? yy[q] - ll[q] : 0.0f;
            acc += d * d;
            g[q] = __bfloat16_as_ushort(__float2bfloat16_rn(2.0f * d * inv));
            t[r][c + q] = g[q];
        }
        uint2 w;
        w.x = (unsigned)g[0] | ((unsigned)g[1] << 16);
        w.y = (unsigned)g[2] | ((unsigned)g[3] << 16);
        *reinterpret_cast<uint2 *>(dY + (int64_t)(r0 + r) * NCH + c) = w;
    }
    __syncthreads();
    store_tile_t(t, dYT, rows, 0, r0);
    // one atomic per block: warp sums, then the block's warps
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
        atomicAdd(loss_sum, tot * inv);
    }
}

// ---- the gradients of one minibatch, and AdamW (decoupled weight decay on
// weights only) with a refresh of the bf16 copies.
// A weight gradient is the sum, in slice order, of the split-K slices its
// GEMM stored (deterministic, no atomics); a bias gradient is the row sum of
// the layer's transposed output gradient dT ([out][rows] bf16), taken by one
// block per bias (16-byte loads, a fixed shuffle tree per warp, the warps'
// sums in warp order).  Blocks [0, bias_blocks) take the biases, the others
// four weights per thread.
struct GradSegs {
    float *W[4], *m[4], *v[4], *g[4];  // weights [out][in] (and moments, gradient out)
    float *b[4], *mb[4], *vb[4], *gb[4];
    __nv_bfloat16 *Wb[4], *WbT[4];
    const float *part[4];              // [z][out * in] slices
    const __nv_bfloat16 *dT[4];        // [out][rows]
    int64_t woff[5];                   // weight index ranges in the concatenation (multiples of 4)
    int boff[5];                       // bias index ranges
    int z[4], rows_w[4], cols_w[4];
    int rows;                          // minibatch rows (a multiple of 8)
    int bias_blocks;
};

__device__ __forceinline__ float adam_step(float &w, float &m, float &v, float g, float lr, float b1, float b2,
                                           float eps, float c1, float c2, float wd)
{
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    w -= lr * ((m / c1) / (sqrtf(v / c2) + eps) + wd * w);
    return w;
}

// UPDATE: AdamW on every parameter; otherwise the gradients are stored into g / gb
template <bool UPDATE>
__global__ void __launch_bounds__(256) grad_adamw_kernel(GradSegs a, float lr, float b1, float b2, float eps,
                                                         float c1, float c2, float wd)
{
    if ((int)blockIdx.x < a.bias_blocks) {
        __shared__ float part[8];
        const int j = blockIdx.x, lane = threadIdx.x & 31;
        int k = 0;
        while (k < 3 && j >= a.boff[k + 1]) ++k;
        const int o = j - a.boff[k];
        const uint4 *row = reinterpret_cast<const uint4 *>(a.dT[k] + (int64_t)o * a.rows);
        float acc = 0.0f;
#pragma unroll 4
        for (int q = threadIdx.x; q < a.rows / 8; q += blockDim.x) {
            const uint4 v = row[q];
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 f = __bfloat1622float2(h[i]);
                acc += f.x + f.y;
            }
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float g = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) g += part[w];
            if (UPDATE)
                adam_step(a.b[k][o], a.mb[k][o], a.vb[k][o], g, lr, b1, b2, eps, c1, c2, 0.0f);
            else
                a.gb[k][o] = g;
        }
        return;
    }
    const int64_t stride = (int64_t)(gridDim.x - a.bias_blocks) * blockDim.x * 4;
    for (int64_t t = ((int64_t)(blockIdx.x - a.bias_blocks) * blockDim.x + threadIdx.x) * 4; t < a.woff[4];
         t += stride) {
        int k = 0;
        while (k < 3 && t >= a.woff[k + 1]) ++k;
        const int64_t i = t - a.woff[k], n = a.woff[k + 1] - a.woff[k];
        const float *pp = a.part[k] + i;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        const int z = a.z[k];
#pragma unroll 8
        for (int q = 0; q < z; ++q) {
            const float4 p4 = *reinterpret_cast<const float4 *>(pp + (int64_t)q * n);
            g.x += p4.x;
            g.y += p4.y;
            g.z += p4.z;
            g.w += p4.w;
        }
        if (!UPDATE) {
            *reinterpret_cast<float4 *>(a.g[k] + i) = g;
            continue;
        }
        float4 w = *reinterpret_cast<const float4 *>(a.W[k] + i);
        float4 mi = *reinterpret_cast<const float4 *>(a.m[k] + i);
        float4 vi = *reinterpret_cast<const float4 *>(a.v[k] + i);
        adam_step(w.x, mi.x, vi.x, g.x, lr, b1, b2, eps, c1, c2, wd);
        adam_step(w.y, mi.y, vi.y, g.y, lr, b1, b2, eps, c1, c2, wd);
        adam_step(w.z, mi.z, vi.z, g.z, lr, b1, b2, eps, c1, c2, wd);
        adam_step(w.w, mi.w, vi.w, g.w, lr, b1, b2, eps, c1, c2, wd);
        *reinterpret_cast<float4 *>(a.W[k] + i) = w;
        *reinterpret_cast<float4 *>(a.m[k] + i) = mi;
        *reinterpret_cast<float4 *>(a.v[k] + i) = vi;
        const __nv_bfloat16 wb[4] = {__float2bfloat16_rn(w.x), __float2bfloat16_rn(w.y), __float2bfloat16_rn(w.z),
                                     __float2bfloat16_rn(w.w)};
        uint2 pk;
        pk.x = (unsigned)__bfloat16_as_ushort(wb[0]) | ((unsigned)__bfloat16_as_ushort(wb[1]) << 16);
        pk.y = (unsigned)__bfloat16_as_ushort(wb[2]) | ((unsigned)__bfloat16_as_ushort(wb[3]) << 16);
        *reinterpret_cast<uint2 *>(a.Wb[k] + i) = pk;
        const int cols = a.cols_w[k], rw = a.rows_w[k];
#pragma unroll
        for (int q = 0; q < 4; ++q) a.WbT[k][((i + q) % cols) * rw + (i + q) / cols] = wb[q];
    }
}

__global__ void to_bf16_kernel(const float *W, int64_t n, int rows, int cols, __nv_bfloat16 *Wb,
                               __nv_bfloat16 *WbT)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const __nv_bfloat16 wb = __float2bfloat16_rn(W[i]);
        Wb[i] = wb;
        if (WbT) WbT[(i % cols) * rows + i / cols] = wb;
    }
}

// ---- per system: the top_k candidates in increasing score (ties: lower
// index), the first n_pinned candidate slots ahead of every scored one.  Row i
// of score is system i (with sys_list, system sys_list[i]); the picks after the
// first `skip` go to that system's row of ranked (row_len entries per row, 0:
// top_k - skip), followed, when row_len is longer, by the candidates not picked
// in index order.
__global__ void topk_kernel(const float *score, int64_t n_sys, int32_t K, int32_t n_pinned, int32_t top_k,
                            int32_t *ranked, const int32_t *sys_list = nullptr, int32_t skip = 0,
                            int32_t row_len = 0)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t sys = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (sys >= n_sys) return;
    const float *s = score + sys * K;
    const int64_t row = sys_list ? (int64_t)sys_list[sys] : sys;
    const int32_t len = row_len > 0 ? row_len : top_k - skip;
    int32_t *out = ranked + row * len;
    // pick repeatedly the smallest (score, index) above the previous pick
    float last_s = -INFINITY;
    int last_i = -1;
    for (int t = 0; t < top_k; ++t) {
        float best_s = INFINITY;
        int best_i = 0x7fffffff;
        for (int k = lane; k < K; k += 32) {
            const float v = k < n_pinned ? -INFINITY : (isnan(s[k]) ? INFINITY : s[k]);
            const bool after = v > last_s || (v == last_s && k > last_i);
            if (after && (v < best_s || (v == best_s && k < best_i))) {
                best_s = v;
                best_i = k;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, best_s, off);
            const int oi = __shfl_xor_sync(0xffffffffu, best_i, off);
            if (os < best_s || (os == best_s && oi < best_i)) {
                best_s = os;
                best_i = oi;
            }
        }
        if (lane == 0 && t >= skip) out[t - skip] = best_i;
        last_s = best_s;
        last_i = best_i;
    }
    if (len <= top_k - skip) return;
    // the rest: exactly the candidates above the last pick, in index order
    int base = top_k - skip;
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        bool rest = false;
        if (k < K) {
            const float v = k < n_pinned ? -INFINITY : (isnan(s[k]) ? INFINITY : s[k]);
            rest = v > last_s || (v == last_s && k > last_i);
        }
        const unsigned m = __ballot_sync(0xffffffffu, rest);
        const int at = base + __popc(m & ((1u << lane) - 1u));
        if (rest && at < len) out[at] = k;
        base += __popc(m);
    }
}

unsigned grid_for(int64_t n, int threads, int n_sm)
{
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = 16 * (int64_t)n_sm;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

} // namespace

// ---------------------------------------------------------------------------
// model lifecycle
// ---------------------------------------------------------------------------
namespace {

int model_alloc(paam_ctx *ctx, paam_model **out)
{
    paam_model *m = (paam_model *)calloc(1, sizeof(paam_model));
    if (!m) return PAAM_E_NOMEM;
    m->ctx = ctx;
    size_t bytes = 0;
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l], nb = OUT[l];
        bytes += 4 * (4 * nw + 4 * nb) + 2 * 2 * nw + 8 * 256;
    }
    if (cudaMalloc(&m->block, bytes) != cudaSuccess) {
        cudaGetLastError();
        free(m);
        return PAAM_E_NOMEM;
    }
    m->block_bytes = bytes;
    cudaMemset(m->block, 0, bytes);
    char *p = (char *)m->block;
    auto take = [&](size_t n) {
        char *q = p;
        p += (n + 255) & ~(size_t)255;
        return q;
    };
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l], nb = OUT[l];
        m->W[l] = (float *)take(4 * nw);
        m->mW[l] = (float *)take(4 * nw);
        m->vW[l] = (float *)take(4 * nw);
        m->gW[l] = (float *)take(4 * nw);
        m->bias[l] = (float *)take(4 * nb);
        m->mb[l] = (float *)take(4 * nb);
        m->vb[l] = (float *)take(4 * nb);
        m->gb[l] = (float *)take(4 * nb);
        m->Wb[l] = (__nv_bfloat16 *)take(2 * nw);
        m->WbT[l] = (__nv_bfloat16 *)take(2 * nw);
    }
    *out = m;
    return PAAM_OK;
}

int refresh_bf16(paam_model *m, cudaStream_t s)
{
    for (int l = 0; l < NL; ++l) {
        const int64_t nw = (int64_t)IN[l] * OUT[l];
        to_bf16_kernel<<<grid_for(nw, 256, m->ctx->n_sm), 256, 0, s>>>(m->W[l], nw, OUT[l], IN[l], m->Wb[l],
                                                                       m->WbT[l]);
        PAAM_CUDA_TRY(cudaGetLastError());
    }
    paam_count_launch(NL);
    return PAAM_OK;
}

// splitmix64-driven uniform in [-1, 1)
double unif_pm1(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

} // namespace

extern "C" int paam_model_create(paam_ctx *ctx, uint64_t seed, paam_model **out)
{
    if (!ctx || !out) return PAAM_E_INVAL;
    *out = nullptr;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    paam_model *m = nullptr;
    int rc = model_alloc(ctx, &m);
    if (rc != PAAM_OK) return rc;
    uint64_t x = seed;
    for (int l = 0; l < NL; ++l) { // uniform(-a, a), a = sqrt(6 / fan_in): keeps GELU activations in range
        const size_t nw = (size_t)IN[l] * OUT[l];
        const double a = sqrt(6.0 / IN[l]);
        std::vector<float> w(nw);
        for (size_t i = 0; i < nw; ++i) w[i] = (float)(a * unif_pm1(&x));
        if (cudaMemcpy(m->W[l], w.data(), 4 * nw, cudaMemcpyHostToDevice) != cudaSuccess) rc = PAAM_E_CUDA;
    }
    if (rc == PAAM_OK) rc = refresh_bf16(m, 0);
    if (rc == PAAM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc != PAAM_OK) {
        cudaFree(m->block);
        free(m);
        return rc;
    }
    *out = m;
    return PAAM_OK;
}

extern "C" void paam_model_free(paam_model *m)
{
    if (!m) return;
    cudaSetDevice(m->ctx->device);
    cudaFree(m->block);
    free(m);
}

extern "C" int64_t paam_model_num_params(void) { return (int64_t)n_params(); }

// host copy of the fp32 parameters: per layer W [out][in] row-major, then bias [out]
extern "C" int paam_model_get_params(const paam_model *m, float *host)
{
    if (!m || !host) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(m->ctx->device));
    size_t o = 0;
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l];
        PAAM_CUDA_TRY(cudaMemcpy(host + o, m->W[l], 4 * nw, cudaMemcpyDeviceToHost));
        o += nw;
        PAAM_CUDA_TRY(cudaMemcpy(host + o, m->bias[l], 4 * (size_t)OUT[l], cudaMemcpyDeviceToHost));
        o += OUT[l];
    }
    return PAAM_OK;
}

extern "C" int paam_model_set_params(paam_model *m, const float *host)
{
    if (!m || !host) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(m->ctx->device));
    size_t o = 0;
    for (int l = 0; l < NL; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l];
        PAAM_CUDA_TRY(cudaMemcpy(m->W[l], host + o, 4 * nw, cudaMemcpyHostToDevice));
        o += nw;
        PAAM_CUDA_TRY(cudaMemcpy(m->bias[l], host + o, 4 * (size_t)OUT[l], cudaMemcpyHostToDevice));
        o += OUT[l];
    }
    int rc = refresh_bf16(m, 0);
    if (rc == PAAM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PAAM_E_CUDA;
    return rc;
}

// ---------------------------------------------------------------------------
// one minibatch: forward, masked MSE, backward, AdamW
// ---------------------------------------------------------------------------
namespace {

// Rows of one inference chunk at most (about 2.3 KB of scratch per row for
// systems of up to 16 chains, 3.8 KB for 64)
constexpr int64_t kInferRows = (int64_t)1 << 22;

struct Work {
    int rows;
    void *block;
    __nv_bfloat16 *Xb, *XbT, *Z[3], *H[3], *HT[3], *dY, *dYT, *dZ[3], *dZT[3];
    float *Lb, *Y, *count, *loss;
    float *part[4]; // per layer, the split-K slices of its weight gradient (training)
    int z[4];       // slices per layer
    int32_t *err;
};

// Weight-gradient GEMMs dW = dT x in^T contract over the minibatch rows: K is
// split so that the tiles times the splits cover the SMs about once, with at
// least two 64-row steps per split; each split stores its own slice and the
// slices are summed in order (deterministic, no atomics).
struct DwPlan {
    int bn, splits, z; // column tile, splits asked for, slices the launch writes
};

DwPlan dw_plan(int out, int in, int rows, int n_sm)
{
    DwPlan d;
    d.bn = in >= 1024 ? 256 : 64;
    const int tiles = ((out + 127) / 128) * (in / d.bn);
    const int kb = rows / 64;
    int sp = n_sm / tiles;
    if (sp > kb / 2) sp = kb / 2;
    if (sp < 1) sp = 1;
    d.splits = sp;
    const int per = (kb + sp - 1) / sp;
    d.z = (kb + per - 1) / per;
    return d;
}

size_t dw_part_floats(int l, int rows, int n_sm)
{
    return (size_t)dw_plan(OUT[l], IN[l], rows, n_sm).z * OUT[l] * IN[l];
}

// xw: columns of the input buffer Xb (the full 1024 for training; inference
// stores only the columns its batch can fill)
int work_alloc(Work &w, int rows, bool train, cudaStream_t s, int xw = XW, int n_sm = 0)
{
    w = Work{};
    w.rows = rows;
    const size_t r = (size_t)rows;
    if (n_sm < 1) n_sm = 1;
    size_t part = 0;
    for (int l = 0; train && l < NL; ++l) part += 4 * dw_part_floats(l, rows, n_sm);
    size_t bytes = 2 * r * xw * (train ? 2 : 1) + 3 * 2 * r * 256 * (train ? 6 : 1) + 4 * r * 64 * (train ? 2 : 1) +
                   2 * 2 * r * 64 + 64 * 256 + part + 256;
    if (cudaMallocAsync(&w.block, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    char *p = (char *)w.block;
    auto take = [&](size_t n) {
        char *q = p;
        p += (n + 255) & ~(size_t)255;
        return q;
    };
    w.Xb = (__nv_bfloat16 *)take(2 * r * xw);
    if (train) w.XbT = (__nv_bfloat16 *)take(2 * r * xw);
    for (int l = 0; l < 3; ++l) {
        w.H[l] = (__nv_bfloat16 *)take(2 * r * 256);
        if (train) {
            w.Z[l] = (__nv_bfloat16 *)take(2 * r * 256);
            w.HT[l] = (__nv_bfloat16 *)take(2 * r * 256);
            w.dZ[l] = (__nv_bfloat16 *)take(2 * r * 256);
            w.dZT[l] = (__nv_bfloat16 *)take(2 * r * 256);
        }
    }
    w.Y = (float *)take(4 * r * 64);
    if (train) {
        w.Lb = (float *)take(4 * r * 64);
        w.dY = (__nv_bfloat16 *)take(2 * r * 64);
        w.dYT = (__nv_bfloat16 *)take(2 * r * 64);
    }
    for (int l = 0; train && l < NL; ++l) {
        w.part[l] = (float *)take(4 * dw_part_floats(l, rows, n_sm));
        w.z[l] = dw_plan(OUT[l], IN[l], rows, n_sm).z;
    }
    w.count = (float *)take(4);
    w.loss = (float *)take(4);
    w.err = (int32_t *)take(4);
    return PAAM_OK;
}

// Column tile for a minibatch GEMM: the widest that still gives every SM a
// tile (minibatches of a few thousand rows have few row tiles).
int bn_for(int M, int N, int n_sm)
{
    const int mt = (M + 127) / 128;
    for (int bn = 256; bn >= 64; bn /= 2)
        if (N % bn == 0 && mt * (N / bn) >= n_sm) return bn;
    return 64;
}

TcGemm gemm(const __nv_bfloat16 *A, int lda, int a_rows, const __nv_bfloat16 *B, int ldb, int b_rows, int K)
{
    TcGemm g = {};
    g.A = A;
    g.lda = lda;
    g.a_rows = a_rows;
    g.B = B;
    g.ldb = ldb;
    g.b_rows = b_rows;
    g.K = K;
    g.splits = 1;
    return g;
}

// Feature columns that can be non-zero in this batch: 16 per chain slot up to
// the largest system, rounded up to the GEMM's 64-column K step.
int input_width(const paam_batch *b)
{
    const int w = ((NF * (b->max_chains > 0 ? b->max_chains : 1)) + 63) / 64 * 64;
    return w < XW ? w : XW;
}

// X (rows of w.Xb, kx columns) through the network into w.Y; keeps Z, H, H^T
// when training.  kx < 1024 reads only the first kx input columns of layer 1:
// exact when the remaining feature columns are zero (chain slots past every
// system's chains), since their products add nothing to the fp32 sums.
// With score != NULL the output layer writes, per row, the largest
// prediction over the row's system's chains (at least 0) into score[row]
// (zeroed here) instead of all 64 outputs into w.Y; rows are candidates of
// systems sys0.. in groups of K.
struct ScoreOut {
    float *score;
    const int64_t *sys_off;
    int64_t sys0;
    int K;
    const int32_t *sys_list; // rows' systems through this list (NULL: consecutive from sys0)
};

int forward(const paam_model *m, Work &w, const __nv_bfloat16 *X, int kx, bool train, cudaStream_t s,
            const ScoreOut *so = nullptr)
{
    const int rows = w.rows;
    for (int l = 0; l < 3; ++l) {
        TcGemm g = l == 0 ? gemm(X, kx, rows, m->Wb[0], IN[0], OUT[0], kx)
                          : gemm(w.H[l - 1], IN[l], rows, m->Wb[l], IN[l], OUT[l], IN[l]);
        g.ep.mode = TC_EPI_BIAS_GELU;
        g.ep.M = rows;
        g.ep.N = OUT[l];
        g.ep.bias = m->bias[l];
        g.ep.Z = train ? w.Z[l] : nullptr;
        g.ep.ldz = OUT[l];
        g.ep.H = w.H[l];
        g.ep.ldh = OUT[l];
        g.ep.HT = train ? w.HT[l] : nullptr;
        g.ep.ldht = rows;
        if (train) g.bn = bn_for(rows, OUT[l], m->ctx->n_sm);
        int rc = tc_gemm(g, w.err, s);
        if (rc != PAAM_OK) return rc;
    }
    TcGemm g = gemm(w.H[2], IN[3], rows, m->Wb[3], IN[3], OUT[3], IN[3]);
    g.ep.mode = TC_EPI_BIAS_F32;
    g.ep.M = rows;
    g.ep.N = OUT[3];
    g.ep.bias = m->bias[3];
    g.ep.C = w.Y;
    g.ep.ldc = OUT[3];
    if (train) g.bn = bn_for(rows, OUT[3], m->ctx->n_sm);
    if (so) {
        PAAM_CUDA_TRY(cudaMemsetAsync(so->score, 0, 4 * (size_t)rows, s));
        g.ep.mode = TC_EPI_ROWMAX;
        g.ep.C = so->score;
        g.ep.sys_off = so->sys_off;
        g.ep.sys0 = so->sys0;
        g.ep.rows_per_sys = so->K;
        g.ep.sys_list = so->sys_list;
    }
    return tc_gemm(g, w.err, s);
}

// The masked MSE's gradients as the backward GEMMs leave them: per layer, the
// split-K slices of the weight gradient in w.part[l] and the transposed output
// gradient (dY^T, dZ^T) whose row sums are the bias gradient; grad_adamw
// finishes them.
int backward(paam_model *m, Work &w, cudaStream_t s)
{
    const int rows = w.rows, sm = m->ctx->n_sm;
    loss_kernel<<<rows / kTT, 256, 0, s>>>(w.Y, w.Lb, rows, w.count, w.dY, w.dYT, w.loss);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    // output layer: dW4 = dY^T H3, db4 = column sums of dY, dH3 = dY W4 (then the GELU derivative)
    const __nv_bfloat16 *dT = w.dYT; // [OUT[l]][rows]
    const __nv_bfloat16 *d = w.dY;   // [rows][OUT[l]]
    for (int l = 3; l >= 0; --l) {
        const __nv_bfloat16 *inT = l == 0 ? w.XbT : w.HT[l - 1];
        TcGemm g = gemm(dT, rows, OUT[l], inT, rows, IN[l], rows);
        const DwPlan dp = dw_plan(OUT[l], IN[l], rows, sm);
        g.ep.mode = TC_EPI_STORE_F32;
        g.ep.M = OUT[l];
        g.ep.N = IN[l];
        g.ep.C = w.part[l];
        g.ep.ldc = IN[l];
        g.ep.split_stride = (int64_t)OUT[l] * IN[l];
        g.splits = dp.splits;
        g.bn = dp.bn;
        int rc = tc_gemm(g, w.err, s);
        if (rc != PAAM_OK) return rc;
        if (l == 0) break;
        TcGemm h = gemm(d, OUT[l], rows, m->WbT[l], OUT[l], IN[l], OUT[l]);
        h.ep.mode = TC_EPI_DGELU;
        h.ep.M = rows;
        h.ep.N = IN[l];
        h.ep.Zin = w.Z[l - 1];
        h.ep.ldzin = IN[l];
        h.ep.H = w.dZ[l - 1];
        h.ep.ldh = IN[l];
        h.ep.HT = w.dZT[l - 1];
        h.ep.ldht = rows;
        h.bn = bn_for(rows, IN[l], sm);
        rc = tc_gemm(h, w.err, s);
        if (rc != PAAM_OK) return rc;
        dT = w.dZT[l - 1];
        d = w.dZ[l - 1];
    }
    return PAAM_OK;
}

// o != NULL: one AdamW step on the minibatch's gradients (bias corrections
// c1 = 1 - beta1^t, c2 = 1 - beta2^t); o == NULL: the gradients into m->gW, m->gb
int grad_adamw(paam_model *m, const Work &w, const paam_train_opts *o, float c1, float c2, cudaStream_t s)
{
    GradSegs a = {};
    int64_t off = 0;
    int boff = 0;
    for (int l = 0; l < NL; ++l) {
        a.W[l] = m->W[l], a.m[l] = m->mW[l], a.v[l] = m->vW[l], a.g[l] = m->gW[l];
        a.b[l] = m->bias[l], a.mb[l] = m->mb[l], a.vb[l] = m->vb[l], a.gb[l] = m->gb[l];
        a.Wb[l] = m->Wb[l], a.WbT[l] = m->WbT[l];
        a.part[l] = w.part[l];
        a.z[l] = w.z[l];
        a.dT[l] = l == 3 ? w.dYT : w.dZT[l];
        a.rows_w[l] = OUT[l], a.cols_w[l] = IN[l];
        a.woff[l] = off;
        a.boff[l] = boff;
        off += (int64_t)IN[l] * OUT[l];
        boff += OUT[l];
    }
    a.woff[NL] = off;
    a.boff[NL] = boff;
    a.rows = w.rows;
    a.bias_blocks = boff; // one block per bias
    const unsigned grid = (unsigned)a.bias_blocks + grid_for(off / 4, 256, m->ctx->n_sm);
    if (o)
        grad_adamw_kernel<true><<<grid, 256, 0, s>>>(a, o->lr, o->beta1, o->beta2, o->adam_eps, c1, c2,
                                                     o->weight_decay);
    else
        grad_adamw_kernel<false><<<grid, 256, 0, s>>>(a, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f, 1.0f, 0.0f);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}

// One training step: the minibatch gather (rows idx[0 .. rows)), forward,
// backward and AdamW.
int enqueue_step(paam_model *m, Work &w, const __nv_bfloat16 *X, const float *L, const int64_t *idx,
                 const paam_train_opts *o, float c1, float c2, cudaStream_t s)
{
    const int rows = w.rows;
    PAAM_CUDA_TRY(cudaMemsetAsync(w.count, 0, 4, s));
    gather_kernel<<<dim3(XW / kTT, rows / kTT), 256, 0, s>>>(X, L, idx, rows, w.Xb, w.XbT, w.Lb, w.count);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    int rc = forward(m, w, w.Xb, XW, true, s);
    if (rc == PAAM_OK) rc = backward(m, w, s);
    if (rc == PAAM_OK) rc = grad_adamw(m, w, o, c1, c2, s);
    return rc;
}

// The training step as a CUDA graph: captured once, then launched per step
// with two kernel arguments patched, the gather's index pointer and the
// AdamW bias corrections (launches already enqueued keep their own values).
struct StepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t gather = nullptr, adam = nullptr;
    cudaKernelNodeParams pg = {}, pa = {}; // as captured; the argument values live in the graph
    unsigned kernels = 0;
    ~StepGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

constexpr int kGatherArgs = 8, kAdamArgs = 8; // argument counts of gather_kernel, grad_adamw_kernel

int capture_step(StepGraph &g, paam_model *m, Work &w, const __nv_bfloat16 *X, const float *L, const int64_t *idx,
                 const paam_train_opts *o, float c1, float c2, cudaStream_t s)
{
    const uint64_t n0 = paam_launch_count();
    PAAM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(m, w, X, L, idx, o, c1, c2, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &g.graph);
    g.kernels = (unsigned)(paam_launch_count() - n0);
    paam_uncount_launch(g.kernels);
    if (rc != PAAM_OK || ce != cudaSuccess || !g.graph) {
        cudaGetLastError();
        return rc != PAAM_OK ? rc : PAAM_E_CUDA;
    }
    size_t n = 0;
    PAAM_CUDA_TRY(cudaGraphGetNodes(g.graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    PAAM_CUDA_TRY(cudaGraphGetNodes(g.graph, nodes.data(), &n));
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        PAAM_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        if (t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p = {};
        PAAM_CUDA_TRY(cudaGraphKernelNodeGetParams(nd, &p));
        if (p.func == (void *)gather_kernel) {
            g.gather = nd;
            g.pg = p;
        } else if (p.func == (void *)grad_adamw_kernel<true>) {
            g.adam = nd;
            g.pa = p;
        }
    }
    if (!g.gather || !g.adam || !g.pg.kernelParams || !g.pa.kernelParams) return PAAM_E_CUDA;
    PAAM_CUDA_TRY(cudaGraphInstantiate(&g.exec, g.graph, 0));
    return PAAM_OK;
}

int patch_step(StepGraph &g, const int64_t *idx, float c1, float c2)
{
    void *ag[kGatherArgs], *aa[kAdamArgs];
    for (int i = 0; i < kGatherArgs; ++i) ag[i] = g.pg.kernelParams[i];
    for (int i = 0; i < kAdamArgs; ++i) aa[i] = g.pa.kernelParams[i];
    ag[2] = (void *)&idx;
    aa[5] = (void *)&c1;
    aa[6] = (void *)&c2;
    cudaKernelNodeParams p = g.pg;
    p.kernelParams = ag;
    p.extra = nullptr;
    PAAM_CUDA_TRY(cudaGraphExecKernelNodeSetParams(g.exec, g.gather, &p));
    p = g.pa;
    p.kernelParams = aa;
    p.extra = nullptr;
    PAAM_CUDA_TRY(cudaGraphExecKernelNodeSetParams(g.exec, g.adam, &p));
    return PAAM_OK;
}

int check_train_opts(const paam_train_opts *o)
{
    if (!o || o->epochs < 0 || o->batch_rows < 128 || o->batch_rows % 128 || o->n_buckets < 1 || o->kappa_ns < 0 ||
        o->kappa_ns > PAAM_MAX_OVERHEAD || !(o->lr > 0.0f) || !(o->beta1 >= 0.0f && o->beta1 < 1.0f) ||
        !(o->beta2 >= 0.0f && o->beta2 < 1.0f) || !(o->adam_eps > 0.0f) || !(o->weight_decay >= 0.0f))
        return PAAM_E_INVAL;
    return PAAM_OK;
}

} // namespace

extern "C" int paam_surrogate_train(paam_ctx *ctx, const paam_batch *b, const int64_t *R, const uint8_t *status,
                                    const paam_train_opts *o, paam_model **model)
{
    if (!ctx || !b || !model || (b->n_chain > 0 && (!R || !status))) return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    int rc = check_train_opts(o);
    if (rc != PAAM_OK) return rc;
    if (b->max_chains > NCH) return PAAM_E_UNSUPPORTED;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    bool created = false;
    if (!*model) {
        rc = paam_model_create(ctx, o->seed, model);
        if (rc != PAAM_OK) return rc;
        created = true;
    } else if ((*model)->ctx != ctx) {
        return PAAM_E_STATE;
    }
    paam_model *m = *model;
    cudaStream_t s = ctx->capture_stream;
    const int64_t n = b->n_sys;
    const int rows = o->batch_rows;
    const int64_t steps = (n + rows - 1) / rows;
    void *data = nullptr;
    Work w;
    if (cudaMallocAsync(&data, (size_t)n * (2 * XW + 4 * NCH) + 8 * (size_t)steps * rows + 1024, s) != cudaSuccess) {
        cudaGetLastError();
        rc = PAAM_E_NOMEM;
    }
    if (rc == PAAM_OK) rc = work_alloc(w, rows, true, s, XW, ctx->n_sm);
    __nv_bfloat16 *X = (__nv_bfloat16 *)data;
    float *L = (float *)((char *)data + (size_t)n * 2 * XW);
    int64_t *idx_dev = (int64_t *)((char *)L + (size_t)n * 4 * NCH);
    if (rc == PAAM_OK) rc = paam_launch_features(b, nullptr, 1, 0, 0, n, o->n_buckets, o->kappa_ns, XW, X, s);
    if (rc == PAAM_OK) {
        labels_kernel<<<grid_for(n * NCH, 256, ctx->n_sm), 256, 0, s>>>(batch_dev(b), R, status, L);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
        if (cudaMemsetAsync(w.err, 0, 4, s) != cudaSuccess) rc = PAAM_E_CUDA;
    }
    std::vector<int64_t> idx((size_t)(steps * rows));
    StepGraph sg;
    uint64_t rng = o->seed ^ 0x5DEECE66DULL ^ (uint64_t)m->step;
    for (int e = 0; e < o->epochs && rc == PAAM_OK; ++e) {
        // minibatch order: a fresh permutation of the systems, padded with -1
        for (int64_t i = 0; i < (int64_t)idx.size(); ++i) idx[i] = i < n ? i : -1;
        for (int64_t i = n - 1; i > 0; --i) {
            const int64_t j = (int64_t)((unif_pm1(&rng) * 0.5 + 0.5) * (double)(i + 1)) % (i + 1);
            const int64_t t = idx[i];
            idx[i] = idx[j];
            idx[j] = t;
        }
        if (cudaMemcpyAsync(idx_dev, idx.data(), 8 * idx.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(w.loss, 0, 4, s) != cudaSuccess)
            rc = PAAM_E_CUDA;
        for (int64_t st = 0; st < steps && rc == PAAM_OK; ++st) {
            m->step += 1;
            const float c1 = 1.0f - powf(o->beta1, (float)m->step), c2 = 1.0f - powf(o->beta2, (float)m->step);
            const int64_t *ix = idx_dev + st * rows;
            rc = sg.exec ? patch_step(sg, ix, c1, c2) : capture_step(sg, m, w, X, L, ix, o, c1, c2, s);
            if (rc == PAAM_OK && cudaGraphLaunch(sg.exec, s) != cudaSuccess) rc = PAAM_E_CUDA;
            if (rc == PAAM_OK) paam_count_launch(sg.kernels);
        }
        float loss = 0.0f;
        if (rc == PAAM_OK && (cudaMemcpyAsync(&loss, w.loss, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                              cudaStreamSynchronize(s) != cudaSuccess))
            rc = PAAM_E_CUDA;
        if (rc == PAAM_OK && o->epoch_loss) o->epoch_loss[e] = loss / (float)steps;
    }
    int32_t herr = 0;
    if (w.block) cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s);
    if (w.block) cudaFreeAsync(w.block, s);
    if (data) cudaFreeAsync(data, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == PAAM_OK) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    if (rc != PAAM_OK && created) {
        paam_model_free(m);
        *model = nullptr;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// inference
// ---------------------------------------------------------------------------
namespace {

// Scores and ranks the K candidates of n_list systems: systems 0 .. n_list - 1,
// or with sys_list (device) the systems sys_list[0 .. n_list).  Each system's
// picks after the first `skip` go to its row of ranked (rows by system index,
// row_len entries; 0: top_k - skip), then the candidates not picked in index
// order (topk_kernel); scores (optional, device [n_list][K]) by list position.
int infer_rank(paam_ctx *ctx, const paam_model *m, const paam_batch *b, const int16_t *ranks, int32_t K,
               int32_t nmax, int32_t n_buckets, int64_t kappa_ns, int32_t n_pinned, int32_t top_k, int32_t skip,
               const int32_t *sys_list, int64_t n_list, int32_t *ranked, float *scores, cudaStream_t s,
               int32_t row_len = 0)
{
    if (n_list == 0) return PAAM_OK;
    // candidates are scored in equal chunks of whole systems of at most about
    // kInferRows rows: each chunk pays a fixed cost (launches, the weight load
    // of every persistent CTA, the last tile's epilogue running alone), so
    // chunks are as large as the scratch allows
    const int64_t total = n_list * (int64_t)K;
    const int64_t n_chunks = (total + kInferRows - 1) / kInferRows;
    const int64_t chunk = (n_list + n_chunks - 1) / n_chunks;
    const int rows = (int)(chunk * K);
    const int kx = input_width(b);
    Work w;
    int rc = work_alloc(w, rows, false, s, kx);
    if (rc != PAAM_OK) return rc;
    float *sc = scores;
    void *tmp = nullptr;
    if (!sc) {
        if (cudaMallocAsync(&tmp, 4 * (size_t)n_list * K, s) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(w.block, s);
            return PAAM_E_NOMEM;
        }
        sc = (float *)tmp;
    }
    if (cudaMemsetAsync(w.err, 0, 4, s) != cudaSuccess) rc = PAAM_E_CUDA;
    for (int64_t s0 = 0; s0 < n_list && rc == PAAM_OK; s0 += chunk) {
        const int64_t ns = (s0 + chunk <= n_list) ? chunk : n_list - s0;
        const int64_t items = ns * K;
        Work wc = w;
        wc.rows = (int)items;
        rc = paam_launch_features(b, ranks, K, nmax, s0, items, n_buckets, kappa_ns, kx, wc.Xb, s, sys_list);
        const ScoreOut so = {sc + s0 * K, b->sys_chain_off, s0, K, sys_list};
        if (rc == PAAM_OK) rc = forward(m, wc, wc.Xb, kx, false, s, &so);
    }
    if (rc == PAAM_OK) {
        topk_kernel<<<(unsigned)((n_list + 7) / 8), 256, 0, s>>>(sc, n_list, K, n_pinned, top_k, ranked, sys_list,
                                                                 skip, row_len);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
    }
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = PAAM_E_CUDA;
    cudaFreeAsync(w.block, s);
    if (tmp) cudaFreeAsync(tmp, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    return rc;
}

int check_infer_args(const paam_model *m, const paam_batch *b, int32_t K, int32_t nmax, int32_t n_buckets,
                     int64_t kappa_ns, int32_t n_pinned, int32_t top_k)
{
    if (K < 1 || top_k < 1 || top_k > K || n_pinned < 0 || n_pinned > K || nmax < b->max_chains || n_buckets < 1 ||
        kappa_ns < 0 || kappa_ns > PAAM_MAX_OVERHEAD)
        return PAAM_E_INVAL;
    if (b->max_chains > NCH) return PAAM_E_UNSUPPORTED;
    return PAAM_OK;
}

constexpr int32_t kGuidedPicks = 32; // candidates the guided search takes in the network's order

// identity slot order over the first np candidates of every system
__global__ void ident_order_kernel(int32_t *order, int64_t n_sys, int32_t np)
{
    const int64_t n = n_sys * np, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) order[i] = (int32_t)(i % np);
}

// systems without an admitted pinned candidate (fa < 0) go to list; first_ok gets
// -1 (nothing left to visit) for the others and Kr (no candidate yet) for these
__global__ void undecided_kernel(const int32_t *fa, int64_t n_sys, int32_t Kr, int32_t *list, int32_t *count,
                                 int32_t *first_ok)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sys; i += stride) {
        const bool open = fa[i] < 0;
        first_ok[i] = open ? Kr : -1;
        if (open) list[atomicAdd(count, 1)] = (int32_t)i;
    }
}

__global__ void combine_kernel(const int32_t *fa, int64_t n_sys, int32_t *first_ok)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sys; i += stride)
        if (fa[i] >= 0) first_ok[i] = fa[i];
}

} // namespace

extern "C" int paam_surrogate_infer(paam_ctx *ctx, const paam_model *m, const paam_batch *b, const int16_t *ranks,
                                    int32_t K, int32_t nmax, int32_t n_buckets, int64_t kappa_ns, int32_t n_pinned,
                                    int32_t top_k, int32_t *ranked, float *scores, void *stream_)
{
    if (!ctx || !m || !b || (b->n_sys > 0 && (!ranks || !ranked))) return PAAM_E_INVAL;
    if (m->ctx != ctx || b->ctx != ctx) return PAAM_E_STATE;
    int rc = check_infer_args(m, b, K, nmax, n_buckets, kappa_ns, n_pinned, top_k);
    if (rc != PAAM_OK) return rc;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    return infer_rank(ctx, m, b, ranks, K, nmax, n_buckets, kappa_ns, n_pinned, top_k, 0, nullptr, b->n_sys, ranked,
                      scores, (cudaStream_t)stream_);
}

// The exact search guided by the network: the pinned candidates of every system
// first, then, for the systems none of them admits, all other candidates in the
// network's order, stopping at the first admitted one.  Every visited candidate
// is analysed exactly, and a system's candidates are visited until one is
// admitted or none is left, so first_ok[s] >= 0 exactly when the exhaustive
// search admits a candidate of s.
extern "C" int paam_surrogate_search(paam_ctx *ctx, const paam_model *m, const paam_batch *b,
                                     const paam_analysis_opts *o, const int16_t *ranks, int32_t K, int32_t nmax,
                                     int32_t n_pinned, int32_t *first_ok, void *stream_)
{
    if (!ctx || !m || !b || !o || (b->n_sys > 0 && (!ranks || !first_ok))) return PAAM_E_INVAL;
    if (m->ctx != ctx || b->ctx != ctx) return PAAM_E_STATE;
    int rc = check_infer_args(m, b, K, nmax, o->n_buckets, o->kappa_ns, n_pinned, K);
    if (rc != PAAM_OK) return rc;
    if (b->n_sys * (int64_t)K > (int64_t)INT32_MAX) return PAAM_E_RANGE;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream_;
    const int64_t n = b->n_sys;
    const int32_t Kr = K - n_pinned; // candidates left after the pinned ones
    // scratch: pinned order or network order ([n][max(n_pinned, Kr)]), the pinned
    // phase's results, the list of open systems and its length
    const int32_t w = n_pinned > Kr ? n_pinned : Kr;
    void *blk = nullptr;
    const size_t ob = 4 * (size_t)n * (w > 0 ? w : 1);
    if (cudaMallocAsync(&blk, ob + 8 * (size_t)n + 256, s) != cudaSuccess) {
        cudaGetLastError();
        return PAAM_E_NOMEM;
    }
    int32_t *order = (int32_t *)blk;
    int32_t *fa = (int32_t *)((char *)blk + ob);
    int32_t *list = fa + n;
    int32_t *count = list + n;
    const unsigned grid = grid_for(n * (w > 0 ? w : 1), 256, ctx->n_sm);
    if (cudaMemsetAsync(count, 0, 4, s) != cudaSuccess) rc = PAAM_E_CUDA;
    // 1. the pinned candidates, in slot order, stopping at the first admitted one
    if (rc == PAAM_OK && n_pinned > 0) {
        ident_order_kernel<<<grid, 256, 0, s>>>(order, n, n_pinned);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
        if (rc == PAAM_OK) rc = paam_rta_search_ordered(ctx, b, o, ranks, K, nmax, order, n_pinned, 1, nullptr, fa, s);
    } else if (rc == PAAM_OK && cudaMemsetAsync(fa, 0xff, 4 * (size_t)n, s) != cudaSuccess) { // -1: none admitted
        rc = PAAM_E_CUDA;
    }
    // 2. the systems left open, and the network's order of their other candidates
    int32_t n_open = 0;
    if (rc == PAAM_OK) {
        undecided_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(fa, n, Kr, list, count, first_ok);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
        if (rc == PAAM_OK && (cudaMemcpyAsync(&n_open, count, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                              cudaStreamSynchronize(s) != cudaSuccess))
            rc = PAAM_E_CUDA;
    }
    if (rc == PAAM_OK && n_open > 0 && Kr > 0) {
        // every row valid (the closed systems' rows are never read: their slots are pruned)
        if (cudaMemsetAsync(order, 0, 4 * (size_t)n * Kr, s) != cudaSuccess) rc = PAAM_E_CUDA;
        // the network's kGuidedPicks best in increasing score, then the others in index
        // order (a full ranking costs a selection per candidate; an admissible system is
        // found among the best few, an inadmissible one needs every candidate anyway)
        const int32_t picks = Kr < kGuidedPicks ? Kr : kGuidedPicks;
        if (rc == PAAM_OK)
            rc = infer_rank(ctx, m, b, ranks, K, nmax, o->n_buckets, o->kappa_ns, n_pinned, n_pinned + picks,
                            n_pinned, list, n_open, order, nullptr, s, Kr);
        // 3. those candidates in that order, stopping at the first admitted one; the
        // closed systems (first_ok -1) are skipped before their set-up
        if (rc == PAAM_OK) rc = paam_search_ordered_from(ctx, b, o, ranks, K, nmax, order, Kr, first_ok, s);
    } else if (rc == PAAM_OK && n_open > 0) { // nothing left to visit
        if (cudaMemsetAsync(first_ok, 0xff, 4 * (size_t)n, s) != cudaSuccess) rc = PAAM_E_CUDA;
    }
    if (rc == PAAM_OK) {
        combine_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(fa, n, first_ok);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
    }
    cudaFreeAsync(blk, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == PAAM_OK) rc = PAAM_E_CUDA;
    return rc;
}

extern "C" int paam_surrogate_predict(paam_ctx *ctx, const paam_model *m, const paam_batch *b, int32_t n_buckets,
                                      int64_t kappa_ns, float *pred, void *stream_)
{
    if (!ctx || !m || !b || (b->n_sys > 0 && !pred)) return PAAM_E_INVAL;
    if (m->ctx != ctx || b->ctx != ctx) return PAAM_E_STATE;
    if (n_buckets < 1 || kappa_ns < 0 || kappa_ns > PAAM_MAX_OVERHEAD) return PAAM_E_INVAL;
    if (b->max_chains > NCH) return PAAM_E_UNSUPPORTED;
    if (b->n_sys == 0) return PAAM_OK;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream_;
    const int64_t n_chunks = (b->n_sys + kInferRows - 1) / kInferRows;
    const int64_t chunk = (b->n_sys + n_chunks - 1) / n_chunks;
    const int kx = input_width(b);
    Work w;
    int rc = work_alloc(w, (int)chunk, false, s, kx);
    if (rc != PAAM_OK) return rc;
    if (cudaMemsetAsync(w.err, 0, 4, s) != cudaSuccess) rc = PAAM_E_CUDA;
    for (int64_t s0 = 0; s0 < b->n_sys && rc == PAAM_OK; s0 += chunk) {
        Work wc = w;
        wc.rows = (int)((s0 + chunk <= b->n_sys) ? chunk : b->n_sys - s0);
        wc.Y = pred + s0 * NCH;
        rc = paam_launch_features(b, nullptr, 1, 0, s0, wc.rows, n_buckets, kappa_ns, kx, wc.Xb, s);
        if (rc == PAAM_OK) rc = forward(m, wc, wc.Xb, kx, false, s);
    }
    int32_t herr = 0;
    if (cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = PAAM_E_CUDA;
    cudaFreeAsync(w.block, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    return rc;
}

// Loss and gradients of one minibatch (rows a multiple of 128), no update.
extern "C" int paam_surrogate_grad(paam_ctx *ctx, paam_model *m, const void *X, const float *L, int32_t rows,
                                   float *grads_host, float *loss_host)
{
    if (!ctx || !m || !X || !L || !grads_host || rows < 128 || rows % 128) return PAAM_E_INVAL;
    if (m->ctx != ctx) return PAAM_E_STATE;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->capture_stream;
    Work w;
    int rc = work_alloc(w, rows, true, s, XW, ctx->n_sm);
    if (rc != PAAM_OK) return rc;
    int64_t *idx = nullptr;
    if (cudaMallocAsync((void **)&idx, 8 * (size_t)rows, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(w.block, s);
        return PAAM_E_NOMEM;
    }
    std::vector<int64_t> id(rows);
    for (int i = 0; i < rows; ++i) id[i] = i;
    if (cudaMemcpyAsync(idx, id.data(), 8 * (size_t)rows, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(w.err, 0, 4, s) != cudaSuccess || cudaMemsetAsync(w.count, 0, 4, s) != cudaSuccess ||
        cudaMemsetAsync(w.loss, 0, 4, s) != cudaSuccess)
        rc = PAAM_E_CUDA;
    if (rc == PAAM_OK) {
        gather_kernel<<<dim3(XW / kTT, rows / kTT), 256, 0, s>>>((const __nv_bfloat16 *)X, L, idx, rows, w.Xb,
                                                                 w.XbT, w.Lb, w.count);
        if (cudaGetLastError() != cudaSuccess) rc = PAAM_E_CUDA;
        paam_count_launch();
    }
    if (rc == PAAM_OK) rc = forward(m, w, w.Xb, XW, true, s);
    if (rc == PAAM_OK) rc = backward(m, w, s);
    if (rc == PAAM_OK) rc = grad_adamw(m, w, nullptr, 1.0f, 1.0f, s);
    size_t o = 0;
    for (int l = 0; l < NL && rc == PAAM_OK; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l];
        if (cudaMemcpyAsync(grads_host + o, m->gW[l], 4 * nw, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = PAAM_E_CUDA;
        o += nw;
        if (cudaMemcpyAsync(grads_host + o, m->gb[l], 4 * (size_t)OUT[l], cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = PAAM_E_CUDA;
        o += OUT[l];
    }
    float loss = 0.0f;
    int32_t herr = 0;
    cudaMemcpyAsync(&loss, w.loss, 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&herr, w.err, 4, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(idx, s);
    cudaFreeAsync(w.block, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = PAAM_E_CUDA;
    if (rc == PAAM_OK && herr != 0) rc = herr;
    if (loss_host) *loss_host = loss;
    return rc;
}

// ---------------------------------------------------------------------------
// checkpoints: magic, version, step, parameter count, then per layer the fp32
// weights, biases and both AdamW moments
// ---------------------------------------------------------------------------
extern "C" int paam_model_save(const paam_model *m, const char *path)
{
    if (!m || !path) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(m->ctx->device));
    FILE *f = fopen(path, "wb");
    if (!f) return PAAM_E_INVAL;
    const char magic[8] = {'P', 'A', 'A', 'M', 'S', 'U', 'R', '1'};
    const int64_t hdr[2] = {m->step, (int64_t)n_params()};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, 8, 2, f) == 2;
    for (int l = 0; l < NL && ok; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l], nb = OUT[l];
        const float *parts[6] = {m->W[l], m->bias[l], m->mW[l], m->vW[l], m->mb[l], m->vb[l]};
        const size_t sizes[6] = {nw, nb, nw, nw, nb, nb};
        for (int k = 0; k < 6 && ok; ++k) {
            std::vector<float> h(sizes[k]);
            ok = cudaMemcpy(h.data(), parts[k], 4 * sizes[k], cudaMemcpyDeviceToHost) == cudaSuccess &&
                 fwrite(h.data(), 4, sizes[k], f) == sizes[k];
        }
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? PAAM_OK : PAAM_E_CUDA;
}

extern "C" int paam_model_load(paam_ctx *ctx, const char *path, paam_model **out)
{
    if (!ctx || !path || !out) return PAAM_E_INVAL;
    *out = nullptr;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    FILE *f = fopen(path, "rb");
    if (!f) return PAAM_E_INVAL;
    char magic[8];
    int64_t hdr[2];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "PAAMSUR1", 8) == 0 && fread(hdr, 8, 2, f) == 2 &&
              hdr[1] == (int64_t)n_params();
    paam_model *m = nullptr;
    if (ok && model_alloc(ctx, &m) != PAAM_OK) ok = false;
    for (int l = 0; l < NL && ok; ++l) {
        const size_t nw = (size_t)IN[l] * OUT[l], nb = OUT[l];
        float *parts[6] = {m->W[l], m->bias[l], m->mW[l], m->vW[l], m->mb[l], m->vb[l]};
        const size_t sizes[6] = {nw, nb, nw, nw, nb, nb};
        for (int k = 0; k < 6 && ok; ++k) {
            std::vector<float> h(sizes[k]);
            ok = fread(h.data(), 4, sizes[k], f) == sizes[k] &&
                 cudaMemcpy(parts[k], h.data(), 4 * sizes[k], cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    fclose(f);
    if (ok) {
        m->step = hdr[0];
        ok = refresh_bf16(m, 0) == PAAM_OK && cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        if (m) paam_model_free(m);
        return PAAM_E_INVAL;
    }
    *out = m;
    return PAAM_OK;
}

// Surrogate input features of every (system, candidate) into X ([n_sys * K][1024] bf16, device);
// ranks NULL (K = 1) takes the systems' own priorities.
extern "C" int paam_surrogate_features(paam_ctx *ctx, const paam_batch *b, const int16_t *ranks, int32_t K,
                                       int32_t nmax, int32_t n_buckets, int64_t kappa_ns, void *X, void *stream)
{
    if (!ctx || !b || (b->n_sys > 0 && !X) || n_buckets < 1 || kappa_ns < 0 || kappa_ns > PAAM_MAX_OVERHEAD)
        return PAAM_E_INVAL;
    if (b->ctx != ctx) return PAAM_E_STATE;
    if (b->max_chains > NCH) return PAAM_E_UNSUPPORTED;
    if (ranks ? (K < 1 || nmax < b->max_chains) : K != 1) return PAAM_E_INVAL;
    PAAM_CUDA_TRY(cudaSetDevice(ctx->device));
    return paam_launch_features(b, ranks, K, nmax, 0, b->n_sys * (int64_t)K, n_buckets, kappa_ns, XW,
                                (__nv_bfloat16 *)X, (cudaStream_t)stream);
}
