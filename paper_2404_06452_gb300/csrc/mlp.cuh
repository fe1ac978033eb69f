// mlp.cuh -- shared declarations of the surrogate network's GPU code.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

// Epilogue applied to each fp32 accumulator tile of the tensor-core GEMM.
enum TcEpiMode {
    TC_EPI_STORE_F32 = 0,  // C = acc (with split_stride: split z writes C + z * split_stride)
    TC_EPI_BIAS_GELU = 1,  // Z = bf16(acc + bias); H = bf16(gelu(Z)); HT = H^T (optional)
    TC_EPI_BIAS_F32 = 2,   // C = acc + bias
    TC_EPI_DGELU = 3,      // H = bf16(acc * gelu'(Zin)); HT = H^T (optional)
    TC_EPI_ATOMIC_F32 = 4, // C += acc (split-K partial sums)
    TC_EPI_ROWMAX = 5,     // C[row] = max(C[row], 0, max over the row's valid columns of acc + bias)
};

struct TcEpilogue {
    int mode, M, N;                // valid output rows and columns
    float *C;
    int ldc;
    const float *bias;             // [N]
    const __nv_bfloat16 *Zin;      // pre-activation read by TC_EPI_DGELU
    int ldzin;
    __nv_bfloat16 *Z;              // pre-activation written by TC_EPI_BIAS_GELU
    int ldz;
    __nv_bfloat16 *H;              // activation (BIAS_GELU) or input gradient (DGELU), row-major
    int ldh;
    __nv_bfloat16 *HT;             // H transposed ([N][M]), optional
    int ldht;
    // TC_EPI_ROWMAX: row r belongs to system sys0 + r / rows_per_sys (with
    // sys_list, to system sys_list[sys0 + r / rows_per_sys]), whose chain count
    // (sys_off[s + 1] - sys_off[s]) is the number of valid columns; C[r] must
    // start non-negative (the maximum is taken on the float bits)
    const int64_t *sys_off;
    int64_t sys0;
    int rows_per_sys;
    const int32_t *sys_list;
    // TC_EPI_STORE_F32 with splits > 1: each split stores its partial product
    // into its own [M][ldc] slice, C + split * split_stride (summed afterwards
    // in a fixed order, so the result does not depend on scheduling)
    int64_t split_stride;
};

// C[M, N] (epilogue) = A[M, K] * B[N, K]^T with A, B bf16 row-major, lda/ldb in
// elements; a_rows / b_rows are the allocated rows of A and B (tiles past them
// read zeros).  K must be a multiple of 64, lda and ldb multiples of 8, the
// output N a multiple of 64.  splits > 1 divides K over grid z and needs
// TC_EPI_ATOMIC_F32, or TC_EPI_STORE_F32 with a split_stride.  bn (0: chosen
// from N) asks for a column-tile width of 64, 128 or 256 dividing N.  err
// receives PAAM_E_TIMEOUT if a bounded wait expired.
struct TcGemm {
    const __nv_bfloat16 *A;
    int lda, a_rows;
    const __nv_bfloat16 *B;
    int ldb, b_rows;
    int K, splits;
    TcEpilogue ep;
    int bn;
};

int tc_gemm(const TcGemm &g, int32_t *err, cudaStream_t stream);





// Surrogate input features (features.cu): rows item = (system - sys0) * K +
// candidate for items [0, n_items) of systems starting at sys0 (with sys_list,
// of systems sys_list[sys0 ..]); ranks NULL = the systems' own priorities (K = 1).  X is [n_items][width] bf16 with width =
// 16 x (chain slots), a multiple of 16 of at least 16 x the batch's largest
// chain count and at most 1024; slots past a system's chains are zero, so a
// first layer may read only the first width columns of its 1024-wide input.
int paam_launch_features(const paam_batch *b, const int16_t *ranks, int32_t K, int32_t nmax, int64_t sys0,
                         int64_t n_items, int32_t n_buckets, int64_t kappa, int32_t width, __nv_bfloat16 *X,
                         cudaStream_t stream, const int32_t *sys_list = nullptr);
