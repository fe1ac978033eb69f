// mlp_gemm.cu -- BF16 tensor-core GEMM with fused epilogues for the surrogate
// network (tcgen05 + TMA + TMEM on sm_103a).
//
//   C[M, N] = A[M, K] * B[N, K]^T      A, B bf16 row-major (K contiguous),
//                                      fp32 accumulation in tensor memory.
//
// One CTA computes a 128 x BN output tile (BN = 64, 128 or 256) over a range
// of K in 64-wide blocks (split-K along grid z for the weight gradients).
// Warp 0 streams A and B tiles with TMA into a 4-stage ring of 128-byte-
// swizzled shared-memory buffers; warp 1 owns the tensor memory and one of
// its threads issues tcgen05.mma (128 x BN x 16 per instruction); warps 2-5
// drain the accumulator with tcgen05.ld (warp w reads TMEM lanes 32 (w % 4)
// ..) and apply the epilogue to their rows.
#include <mutex>

#include "mlp.cuh"
#include "tc.cuh"

namespace {

constexpr int BM = 128, BK = 64, STAGES = 4;
constexpr uint64_t kWaitNs = 2000000000ull; // 2 s: far above any legitimate wait

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// 32 consecutive accumulator columns col0.. of one output row
__device__ __forceinline__ void epilogue_chunk(const TcEpilogue &ep, int row, int col0, const uint32_t (&v)[32])
{
    if (row >= ep.M) return;
    float a[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) a[i] = __uint_as_float(v[i]);
    const bool full = col0 + 32 <= ep.N;
    switch (ep.mode) {
    case TC_EPI_STORE_F32:
    case TC_EPI_BIAS_F32: {
        if (ep.mode == TC_EPI_BIAS_F32)
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] += (col0 + i < ep.N) ? ep.bias[col0 + i] : 0.0f;
        float *c = ep.C + (size_t)row * ep.ldc + col0;
        if (full) {
#pragma unroll
            for (int i = 0; i < 32; i += 4) *(float4 *)(c + i) = make_float4(a[i], a[i + 1], a[i + 2], a[i + 3]);
        } else {
            for (int i = 0; i < 32; ++i)
                if (col0 + i < ep.N) c[i] = a[i];
        }
        break;
    }
    case TC_EPI_ATOMIC_F32: {
        float *c = ep.C + (size_t)row * ep.ldc + col0;
        for (int i = 0; i < 32; ++i)
            if (col0 + i < ep.N) atomicAdd(c + i, a[i]);
        break;
    }
    case TC_EPI_BIAS_GELU:
    case TC_EPI_DGELU: {
        __nv_bfloat16 out[32];
        if (ep.mode == TC_EPI_BIAS_GELU) {
            __nv_bfloat16 zb[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                zb[i] = __float2bfloat16_rn(a[i] + ((col0 + i < ep.N) ? ep.bias[col0 + i] : 0.0f));
                out[i] = __float2bfloat16_rn(gelu(__bfloat162float(zb[i])));
            }
            if (ep.Z && full) {
                uint4 *z = (uint4 *)(ep.Z + (size_t)row * ep.ldz + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) z[i] = ((const uint4 *)zb)[i];
            }
        } else {
            const __nv_bfloat16 *zin = ep.Zin + (size_t)row * ep.ldzin + col0;
            __nv_bfloat16 zb[32];
            if (full) {
#pragma unroll
                for (int i = 0; i < 4; ++i) ((uint4 *)zb)[i] = ((const uint4 *)zin)[i];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) out[i] = __float2bfloat16_rn(a[i] * gelu_grad(__bfloat162float(zb[i])));
        }
        if (full) {
            uint4 *h = (uint4 *)(ep.H + (size_t)row * ep.ldh + col0);
#pragma unroll
            for (int i = 0; i < 4; ++i) h[i] = ((const uint4 *)out)[i];
            if (ep.HT) // one column at a time: the warp's 32 consecutive rows are contiguous
#pragma unroll
                for (int i = 0; i < 32; ++i) ep.HT[(size_t)(col0 + i) * ep.ldht + row] = out[i];
        }
        break;
    }
    default:
        break;
    }
}

template <int BN>
struct GemmSmem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TILES = STAGES * STAGE;
    static constexpr int TOTAL = TILES + 256 + 1024; // barriers and flags, alignment slack
};

template <int BN>
__global__ void __launch_bounds__(192) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int kb_total,
                                                      int kb_per_split, TcEpilogue ep, int32_t *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023); // swizzled tiles
    using L = GemmSmem<BN>;
    uint64_t *full = (uint64_t *)(smem + L::TILES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kb_per_split;
    const int kb1 = min(kb0 + kb_per_split, kb_total);
    const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        *issued = 0;
        tc::fence_barrier_init();
        tc::prefetch_tmap(&tmA);
        tc::prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, kCols);
        tc::tmem_relinquish();
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) { // ---- TMA producer
        int i = 0;
        for (; i < nkb && !*abort_flag; ++i) {
            const int s = i % STAGES, r = i / STAGES;
            if (r > 0 && !tc::mbar_wait(&empty[s], (r - 1) & 1, kWaitNs)) {
                *abort_flag = 1;
                atomicExch(err, PAAM_E_TIMEOUT);
                break;
            }
            uint8_t *a = smem + s * L::STAGE;
            uint8_t *b = a + L::A_BYTES;
            tc::mbar_expect_tx(&full[s], L::STAGE);
            tc::tma_load_2d(a, &tmA, &full[s], (kb0 + i) * BK, m0);
            tc::tma_load_2d(b, &tmB, &full[s], (kb0 + i) * BK, n0);
        }
        *issued = i;
    } else if (warp == 1 && lane == 0) { // ---- MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16(BM, BN);
        bool ok = nkb > 0;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES, r = i / STAGES;
            if (*abort_flag || !tc::mbar_wait(&full[s], r & 1, kWaitNs)) {
                *abort_flag = 1;
                atomicExch(err, PAAM_E_TIMEOUT);
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(smem + s * L::STAGE);
            const uint32_t b = a + L::A_BYTES;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) // K = 16 per instruction: step 32 bytes inside the swizzle atom
                tc::mma_bf16(tmem, tc::desc_sw128(a + 32 * j), tc::desc_sw128(b + 32 * j), idesc,
                             (i > 0 || j > 0) ? 1u : 0u);
            tc::mma_commit(&empty[s]); // frees the stage once these MMAs have read it
        }
        if (ok) tc::mma_commit(done);
    } else if (warp >= 2) { // ---- epilogue: one output row per thread
        const int q = warp & 3; // the TMEM lane quadrant this warp may access
        const int row = m0 + 32 * q + lane;
        bool ok = nkb > 0;
        if (ok && !tc::mbar_wait(done, 0, kWaitNs)) {
            ok = false;
            *abort_flag = 1;
            atomicExch(err, PAAM_E_TIMEOUT);
        }
        tc::fence_after_sync();
        if (ok) {
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * c), v);
                tc::tmem_wait_ld();
                epilogue_chunk(ep, row, n0 + 32 * c, v);
            }
        }
        tc::fence_before_sync();
    }
    __syncthreads();
    if (warp == 0 && lane == 0 && *abort_flag) {
        // let TMA copies already issued land before this CTA's shared memory is released
        const int n_issued = *issued;
        for (int s = 0; s < STAGES && s < n_issued; ++s) {
            const int last = ((n_issued - 1 - s) / STAGES) * STAGES + s;
            tc::mbar_wait(&full[s], (last / STAGES) & 1, kWaitNs / 4);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kCols);
    }
}

// ---- host side -------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// bf16 row-major matrix [rows][ld], tile box_rows x 64, 128-byte swizzle, zeros outside
bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
int launch_bn(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.a_rows, g.K, g.lda, BM) || !make_map(&mb, g.B, g.b_rows, g.K, g.ldb, BN))
        return PAAM_E_CUDA;
    const int kb_total = g.K / BK;
    const int splits = g.splits < 1 ? 1 : (g.splits > kb_total ? kb_total : g.splits);
    const int per = (kb_total + splits - 1) / splits;
    const dim3 grid((unsigned)((g.ep.M + BM - 1) / BM), (unsigned)(g.ep.N / BN), (unsigned)((kb_total + per - 1) / per));
    const int smem = GemmSmem<BN>::TOTAL;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    tc_gemm_kernel<BN><<<grid, 192, smem, stream>>>(ma, mb, kb_total, per, g.ep, err);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}

} // namespace

int tc_gemm(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    if (g.K <= 0 || g.K % BK || g.lda % 8 || g.ldb % 8 || g.ep.N % 64 || g.ep.M <= 0) return PAAM_E_INVAL;
    if (g.splits > 1 && g.ep.mode != TC_EPI_ATOMIC_F32) return PAAM_E_INVAL;
    if (g.ep.N % 256 == 0) return launch_bn<256>(g, err, stream);
    if (g.ep.N % 128 == 0) return launch_bn<128>(g, err, stream);
    return launch_bn<64>(g, err, stream);
}

// C[M, N] fp32 = A[M, K] * B[N, K]^T (bf16, device, row-major, ld = K).
extern "C" int paam_tc_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, int32_t *err,
                                 void *stream)
{
    if (!A || !B || !C || !err || M <= 0 || N <= 0) return PAAM_E_INVAL;
    TcGemm g = {};
    g.A = (const __nv_bfloat16 *)A;
    g.lda = K;
    g.a_rows = M;
    g.B = (const __nv_bfloat16 *)B;
    g.ldb = K;
    g.b_rows = N;
    g.K = K;
    g.splits = 1;
    g.ep.mode = TC_EPI_STORE_F32;
    g.ep.M = M;
    g.ep.N = N;
    g.ep.C = C;
    g.ep.ldc = N;
    return tc_gemm(g, err, (cudaStream_t)stream);
}
