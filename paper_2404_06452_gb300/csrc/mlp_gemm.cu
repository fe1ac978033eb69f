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

#include "gelu.cuh"
#include "mlp.cuh"
#include "tc.cuh"

namespace {
using namespace paam_gelu;

constexpr int BM = 128, BK = 64;
constexpr uint64_t kWaitNs = 2000000000ull; // 2 s: far above any legitimate wait

// a[i] += bias[col0 + i] (columns past N get nothing); bias is 16-byte aligned
__device__ __forceinline__ void add_bias(const TcEpilogue &ep, int col0, bool full, float (&a)[32])
{
    if (full) {
        const float4 *b4 = reinterpret_cast<const float4 *>(ep.bias + col0);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 v = __ldg(b4 + i);
            a[4 * i] += v.x;
            a[4 * i + 1] += v.y;
            a[4 * i + 2] += v.z;
            a[4 * i + 3] += v.w;
        }
    } else {
        for (int i = 0; i < 32; ++i) a[i] += (col0 + i < ep.N) ? ep.bias[col0 + i] : 0.0f;
    }
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
        if (ep.mode == TC_EPI_BIAS_F32) add_bias(ep, col0, full, a);
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
    case TC_EPI_ROWMAX: {
        const int64_t sys = ep.sys_list ? (int64_t)ep.sys_list[ep.sys0 + row / ep.rows_per_sys]
                                        : ep.sys0 + row / ep.rows_per_sys;
        const int n = (int)(ep.sys_off[sys + 1] - ep.sys_off[sys]);
        if (col0 >= n) break;
        add_bias(ep, col0, full, a);
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (col0 + i < n) m = fmaxf(m, a[i]); // a NaN prediction is ignored
        atomicMax(reinterpret_cast<int *>(ep.C) + row, __float_as_int(m));
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
            add_bias(ep, col0, full, a);
            if (ep.Z && full) { // the pre-activation, kept for the backward pass
                __nv_bfloat162 zb[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) zb[i] = __floats2bfloat162_rn(a[2 * i], a[2 * i + 1]);
                uint4 *z = (uint4 *)(ep.Z + (size_t)row * ep.ldz + col0);
#pragma unroll
                for (int i = 0; i < 4; ++i) z[i] = ((const uint4 *)zb)[i];
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
                ((__nv_bfloat162 *)out)[i] = __floats2bfloat162_rn(gelu(a[2 * i]), gelu(a[2 * i + 1]));
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

template <int BN, int STAGES>
struct GemmSmem {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TILES = STAGES * STAGE;
    static constexpr int TOTAL = TILES + 256 + 1024; // barriers and flags, alignment slack
};

// Warp roles: 0 TMA producer, 1 TMEM owner and MMA issuer, 2..9 epilogue (two
// warps per TMEM lane quadrant, one per half of the tile's columns).
constexpr int kGemmThreads = 320;

template <int BN, int STAGES>
__global__ void __launch_bounds__(kGemmThreads, 2) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int kb_total,
                                                      int kb_per_split, TcEpilogue ep, int32_t *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023); // swizzled tiles
    using L = GemmSmem<BN, STAGES>;
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
    } else if (warp >= 2) { // ---- epilogue: one output row per thread, half the columns per warp
        const int q = warp & 3; // the TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;
        const int row = m0 + 32 * q + lane;
        bool ok = nkb > 0;
        if (ok && !tc::mbar_wait(done, 0, kWaitNs)) {
            ok = false;
            *abort_flag = 1;
            atomicExch(err, PAAM_E_TIMEOUT);
        }
        tc::fence_after_sync();
        if (ok) {
            TcEpilogue e = ep; // a split of a split-K product stores into its own slice
            if (ep.split_stride) e.C = ep.C + (int64_t)blockIdx.z * ep.split_stride;
#pragma unroll 1
            for (int c = half * (BN / 64); c < (half + 1) * (BN / 64); ++c) {
                uint32_t v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * c), v);
                tc::tmem_wait_ld();
                epilogue_chunk(e, row, n0 + 32 * c, v);
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

// ---- persistent, weight-stationary layer -------------------------------------------
// For K <= 256 and one column tile (N = BN) the whole B operand (a layer's
// weights, at most 256 x 256 bf16 = 128 KB) stays in shared memory; each CTA
// loops over row tiles, A tiles stream through a 4-stage TMA ring, and the
// accumulator is double-buffered in TMEM (2 x BN columns) so the epilogue of
// row tile i (16 warps, four per TMEM lane quadrant) overlaps the loads and
// MMAs of tile i + 1.
constexpr int kPersistThreads = 576; // warp 0 TMA, warp 1 TMEM + MMA, warps 2..17 epilogue
constexpr int kPersistEpiWarps = kPersistThreads / 32 - 2;
constexpr int kPersistStages = 4;

// Output staging of the TMA-store epilogue: one 32 x 32 bf16 block per
// epilogue warp (its 32 rows, 32 columns), 64-byte swizzled.
constexpr int kStageBytes = 32 * 32 * 2;

template <int BN>
struct PersistSmem {
    static constexpr int W_BYTES = 256 * BN * 2; // K up to 256
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int STAGE_BYTES = kPersistEpiWarps * kStageBytes;
    static constexpr int BIAS_BYTES = BN * 4;
    static constexpr int TILES = W_BYTES + kPersistStages * A_BYTES + STAGE_BYTES + BIAS_BYTES;
    static constexpr int TOTAL = TILES + 256 + 1024;
};

// Bias, GELU and bf16 packing of 32 accumulator columns col0.. of this
// thread's row, then the row's 64 bytes into the warp's staging block: the
// 16-byte piece k of row r sits at piece k ^ ((r >> 1) & 3), the 64-byte
// swizzle the tensor map of the store names.
__device__ __forceinline__ void stage_gelu_row(const float *bias_s, int col0, const uint32_t (&v)[32],
                                               uint8_t *stage, int lane)
{
    uint32_t packed[16];
    const float2 *b2 = reinterpret_cast<const float2 *>(bias_s + col0);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float2 bb = b2[i];
        const __nv_bfloat162 h =
            __floats2bfloat162_rn(gelu(__uint_as_float(v[2 * i]) + bb.x), gelu(__uint_as_float(v[2 * i + 1]) + bb.y));
        packed[i] = *reinterpret_cast<const uint32_t *>(&h);
    }
    uint8_t *row = stage + lane * 64;
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        *reinterpret_cast<uint4 *>(row + ((k ^ sw) << 4)) =
            make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
}

// TMA_OUT: the epilogue is bias + GELU into H through the staging blocks and
// TMA stores (every column of the tile valid); otherwise epilogue_chunk.
template <int BN, bool TMA_OUT>
__global__ void __launch_bounds__(kPersistThreads, 1)
    tc_layer_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                               const __grid_constant__ CUtensorMap tmH, int kb_total, int m_tiles, TcEpilogue ep,
                               int32_t *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    using L = PersistSmem<BN>;
    uint8_t *wsm = smem;               // kb_total blocks of [BN][64] bf16, 128-byte swizzled
    uint8_t *asm_a = smem + L::W_BYTES; // A ring
    uint8_t *stage_all = asm_a + kPersistStages * L::A_BYTES; // epilogue output blocks (1024-byte aligned)
    float *bias_s = (float *)(stage_all + L::STAGE_BYTES);
    uint64_t *full = (uint64_t *)(smem + L::TILES);
    uint64_t *empty = full + kPersistStages;
    uint64_t *acc_full = empty + kPersistStages;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *wbar = acc_empty + 2;
    uint64_t *fin = wbar + 1;
    uint32_t *tmem_slot = (uint32_t *)(fin + 1);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    volatile int *issued = abort_flag + 1;
    constexpr uint32_t kCols = 2 * BN; // BN in {64, 128, 256}: a power of two >= 32
    constexpr int W_BLOCK = BN * BK * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPersistStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], kPersistEpiWarps);
        }
        tc::mbar_init(wbar, 1);
        tc::mbar_init(fin, 1);
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
    if constexpr (TMA_OUT) // the bias, once per CTA (the TMA-store epilogue reads it from here)
        for (int i = threadIdx.x; i < BN; i += blockDim.x) bias_s[i] = ep.bias[i];
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) { // ---- TMA producer: W once, then A tiles
        tc::mbar_expect_tx(wbar, (uint32_t)(kb_total * W_BLOCK));
        for (int kb = 0; kb < kb_total; ++kb) tc::tma_load_2d(wsm + kb * W_BLOCK, &tmB, wbar, kb * BK, 0);
        int it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < m_tiles; tile += gridDim.x) {
            for (int kb = 0; kb < kb_total; ++kb) {
                const int s = it % kPersistStages, r = it / kPersistStages;
                if (*abort_flag || (r > 0 && !tc::mbar_wait(&empty[s], (r - 1) & 1, kWaitNs))) {
                    *abort_flag = 1;
                    atomicExch(err, PAAM_E_TIMEOUT);
                    ok = false;
                    break;
                }
                tc::mbar_expect_tx(&full[s], L::A_BYTES);
                tc::tma_load_2d(asm_a + s * L::A_BYTES, &tmA, &full[s], kb * BK, tile * BM);
                ++it;
            }
        }
        *issued = it;
    } else if (warp == 1 && lane == 0) { // ---- MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16(BM, BN);
        bool ok = tc::mbar_wait(wbar, 0, kWaitNs);
        int it = 0, i = 0;
        for (int tile = blockIdx.x; ok && tile < m_tiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            if (*abort_flag || (i >= 2 && !tc::mbar_wait(&acc_empty[b], ((i >> 1) - 1) & 1, kWaitNs))) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t d = tmem + (uint32_t)(b * BN);
            for (int kb = 0; kb < kb_total; ++kb, ++it) {
                const int s = it % kPersistStages, r = it / kPersistStages;
                if (*abort_flag || !tc::mbar_wait(&full[s], r & 1, kWaitNs)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a = tc::smem_u32(asm_a + s * L::A_BYTES);
                const uint32_t w = tc::smem_u32(wsm + kb * W_BLOCK);
#pragma unroll
                for (int j = 0; j < BK / 16; ++j)
                    tc::mma_bf16(d, tc::desc_sw128(a + 32 * j), tc::desc_sw128(w + 32 * j), idesc,
                                 (kb > 0 || j > 0) ? 1u : 0u);
                tc::mma_commit(&empty[s]);
            }
            if (!ok) break;
            tc::mma_commit(&acc_full[b]);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, PAAM_E_TIMEOUT);
        }
        // every MMA this thread issued has completed before TMEM can be released
        tc::mma_commit(fin);
        tc::mbar_wait(fin, 0, kWaitNs);
    } else if (warp >= 2) { // ---- epilogue: one output row per thread, a quarter of the columns per warp
        const int q = warp & 3, cg = (warp - 2) >> 2;
        uint8_t *stage = stage_all + (warp - 2) * kStageBytes;
        int i = 0;
        for (int tile = blockIdx.x; tile < m_tiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            if (*abort_flag || !tc::mbar_wait(&acc_full[b], (i >> 1) & 1, kWaitNs)) {
                *abort_flag = 1;
                atomicExch(err, PAAM_E_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            const int row0 = tile * BM + 32 * q;
#pragma unroll 1
            for (int c = cg; c < BN / 32; c += 4) {
                uint32_t v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * BN + 32 * c), v);
                tc::tmem_wait_ld();
                if constexpr (TMA_OUT) {
                    // the warp's previous store has read its staging block
                    if (lane == 0) tc::bulk_wait_read_all();
                    __syncwarp();
                    stage_gelu_row(bias_s, 32 * c, v, stage, lane);
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0 && row0 < ep.M) { // rows past M are clipped by the tensor map
                        tc::tma_store_2d(&tmH, stage, 32 * c, row0);
                        tc::bulk_commit();
                    }
                } else {
                    epilogue_chunk(ep, row0 + lane, 32 * c, v);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
        }
        if (TMA_OUT && lane == 0) tc::bulk_wait_all(); // stores complete before shared memory is released
    }
    __syncthreads();
    if (warp == 0 && lane == 0 && *abort_flag) {
        // let TMA copies already issued land before this CTA's shared memory is released
        tc::mbar_wait(wbar, 0, kWaitNs / 4);
        const int n_issued = *issued;
        for (int s = 0; s < kPersistStages && s < n_issued; ++s) {
            const int last = ((n_issued - 1 - s) / kPersistStages) * kPersistStages + s;
            tc::mbar_wait(&full[s], (last / kPersistStages) & 1, kWaitNs / 4);
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

template <int BN, int STAGES>
int launch_bn(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.a_rows, g.K, g.lda, BM) || !make_map(&mb, g.B, g.b_rows, g.K, g.ldb, BN))
        return PAAM_E_CUDA;
    const int kb_total = g.K / BK;
    const int splits = g.splits < 1 ? 1 : (g.splits > kb_total ? kb_total : g.splits);
    const int per = (kb_total + splits - 1) / splits;
    const dim3 grid((unsigned)((g.ep.M + BM - 1) / BM), (unsigned)(g.ep.N / BN), (unsigned)((kb_total + per - 1) / per));
    const int smem = GemmSmem<BN, STAGES>::TOTAL;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    tc_gemm_kernel<BN, STAGES><<<grid, kGemmThreads, smem, stream>>>(ma, mb, kb_total, per, g.ep, err);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}

// Short K (at most 4 steps of 64) needs no deeper ring than 2 stages; the
// smaller footprint lets 2 CTAs share an SM, so one CTA's epilogue overlaps
// the other's loads and MMAs (TMEM: 2 x 256 columns at most).
template <int BN>
int launch_bn_depth(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    const int per = g.splits > 1 ? (g.K / BK + g.splits - 1) / g.splits : g.K / BK;
    if (per <= 4) return launch_bn<BN, 2>(g, err, stream);
    return launch_bn<BN, 4>(g, err, stream);
}

} // namespace

static int sm_count()
{
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev];
}

// bf16 row-major output [rows][ld] with cols valid columns, 32 x 32 boxes,
// 64-byte swizzle (the epilogue's staging layout); rows past `rows` are not written
bool make_store_map(CUtensorMap *m, const __nv_bfloat16 *base, int rows, int cols, int ld)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
int launch_persistent(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    CUtensorMap ma, mb, mh;
    if (!make_map(&ma, g.A, g.a_rows, g.K, g.lda, BM) || !make_map(&mb, g.B, g.b_rows, g.K, g.ldb, BN))
        return PAAM_E_CUDA;
    // the TMA-store epilogue: bias + GELU into H only, every column of the tile valid, H 16-byte aligned rows
    int tma_out = g.ep.mode == TC_EPI_BIAS_GELU && !g.ep.Z && !g.ep.HT && g.ep.H && g.ep.bias && g.ep.N == BN &&
                  g.ep.ldh % 8 == 0 && ((uintptr_t)g.ep.H & 15) == 0;
    if (tma_out && !make_store_map(&mh, g.ep.H, g.ep.M, g.ep.N, g.ep.ldh)) tma_out = 0;
    if (!tma_out) mh = ma; // unused
    const int m_tiles = (g.ep.M + BM - 1) / BM;
    const int n_sm = sm_count();
    const int grid = m_tiles < n_sm ? m_tiles : (n_sm > 0 ? n_sm : 1);
    const int smem = PersistSmem<BN>::TOTAL;
    auto kern = tma_out ? tc_layer_persistent_kernel<BN, true> : tc_layer_persistent_kernel<BN, false>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    kern<<<grid, kPersistThreads, smem, stream>>>(ma, mb, mh, g.K / BK, m_tiles, g.ep, err);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}

int tc_gemm(const TcGemm &g, int32_t *err, cudaStream_t stream)
{
    if (g.K <= 0 || g.K % BK || g.lda % 8 || g.ldb % 8 || g.ep.N % 64 || g.ep.M <= 0) return PAAM_E_INVAL;
    if (g.splits > 1 && g.ep.mode != TC_EPI_ATOMIC_F32 && !(g.ep.mode == TC_EPI_STORE_F32 && g.ep.split_stride > 0))
        return PAAM_E_INVAL;
    if (g.ep.split_stride && (g.ep.mode != TC_EPI_STORE_F32 || g.splits < 1)) return PAAM_E_INVAL;
    if (g.bn && ((g.bn != 64 && g.bn != 128 && g.bn != 256) || g.ep.N % g.bn)) return PAAM_E_INVAL;
    if (g.bn == 64) return launch_bn_depth<64>(g, err, stream);
    if (g.bn == 128) return launch_bn_depth<128>(g, err, stream);
    // one column tile, short K, many row tiles: weights stay resident, epilogue overlaps MMA
    if (g.splits <= 1 && g.K <= 256 && g.b_rows == g.ep.N && g.ep.M >= 4 * BM * sm_count()) {
        if (g.ep.N == 256) return launch_persistent<256>(g, err, stream);
        if (g.ep.N == 128) return launch_persistent<128>(g, err, stream);
        if (g.ep.N == 64) return launch_persistent<64>(g, err, stream);
    }
    if (g.ep.N % 256 == 0) return launch_bn_depth<256>(g, err, stream);
    if (g.ep.N % 128 == 0) return launch_bn_depth<128>(g, err, stream);
    return launch_bn_depth<64>(g, err, stream);
}

namespace {
using namespace paam_gelu;
__global__ void diag_gelu_kernel(const float *z, float *g, float *d, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (g) g[i] = gelu(z[i]);
        if (d) d[i] = gelu_grad(z[i]);
    }
}
} // namespace

extern "C" int paam_diag_gelu(const float *z, float *gelu_out, float *grad_out, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && !z)) return PAAM_E_INVAL;
    if (n == 0) return PAAM_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    diag_gelu_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(z, gelu_out, grad_out, n);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
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
