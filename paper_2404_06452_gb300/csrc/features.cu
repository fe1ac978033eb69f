// features.cu -- input features of the surrogate network.
//
// For every (system, candidate priority order) the network sees 64 chain
// slots of 16 features (zero for slots past the system's chains), all
// dimensionless ratios of the quantities the analysis uses (Sec. II-C and
// Sec. IV-F), with priorities taken from the candidate and executor
// priorities derived from them (criticality-as-priority):
//
//   0 E/T             1 S*/T            2 D/T           3 log2(T/Tmin)/4
//   4 rank/n          5 min(delta,16)/16  6 Emax/D      7 M*/D
//   8 sum_hp (E+S*)/T 9 sum_hpp E/T     10 sum_hps S*/T 11 B/D
//  12 blk/D           13 (E+S*)/D       14 sum_{hp,hpp} (E+S*)/D   15 1
//
// (E: CPU WCET sum, S*: sum of A + 2 kappa, M*: largest A + 2 kappa, B: the
// Lemma 4 blocking term, blk: the same-bucket accelerator blocking term;
// hp, hpp, hps as in Theorem 1 and Eq. 3.)  Each value is clipped to [0, 8]
// and stored as bf16.  One warp computes one item.
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace {

constexpr int NCH = 64, NF = 16;

struct FeatSmem {
    float T[NCH], D[NCH], E[NCH], Emax[NCH], S[NCH], M[NCH];
    int32_t prio[NCH], ep[NCH], exec[NCH], core[NCH], dl[NCH], bucket[NCH];
};

__global__ void __launch_bounds__(256) features_kernel(BatchDev b, const int16_t *ranks, int32_t K, int32_t nmax,
                                                       int64_t sys0, int64_t n_items, int32_t n_buckets,
                                                       int64_t kappa, __nv_bfloat16 *X)
{
    __shared__ FeatSmem sm[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FeatSmem &s = sm[warp];
    const int64_t gw = (int64_t)blockIdx.x * 8 + warp, nw = (int64_t)gridDim.x * 8;
    for (int64_t item = gw; item < n_items; item += nw) {
        const int64_t sys = sys0 + item / K;
        const int32_t cand = (int32_t)(item % K);
        const int64_t c0 = b.sys_chain_off[sys];
        const int n = (int)(b.sys_chain_off[sys + 1] - c0);
        const int64_t x0 = b.sys_exec_off[sys];
        const int16_t *row = ranks ? ranks + (sys * K + cand) * nmax : nullptr;
        unsigned users = 0, users_hi = 0;
        for (int c = lane; c < n; c += 32) {
            const int64_t g = c0 + c;
            const int x = b.exec[g];
            s.T[c] = (float)b.T[g];
            s.D[c] = (float)b.D[g];
            s.prio[c] = row ? (n - 1 - row[c]) : b.prio[g];
            s.exec[c] = x;
            s.core[c] = b.exec_core[x0 + x];
            s.ep[c] = (!row && b.exec_prio) ? b.exec_prio[x0 + x] : INT32_MIN;
            const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
            double E = 0, Emax = 0, S = 0, M = 0;
            for (int64_t cb = cb0; cb < cb1; ++cb) {
                const double e = (double)b.E[cb];
                E += e;
                Emax = e > Emax ? e : Emax;
            }
            const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
            for (int64_t q = q0; q < q1; ++q) {
                const double a = (double)b.A[q] + 2.0 * (double)kappa;
                S += a;
                M = a > M ? a : M;
            }
            s.E[c] = (float)E;
            s.Emax[c] = (float)Emax;
            s.S[c] = (float)S;
            s.M[c] = (float)M;
            s.dl[c] = (int32_t)(q1 - q0);
            if (q1 > q0) {
                if (c < 32) users |= 1u << c;
                else users_hi |= 1u << (c - 32);
            }
        }
        users = __reduce_or_sync(0xffffffffu, users);
        users_hi = __reduce_or_sync(0xffffffffu, users_hi);
        const int n_users = __popc(users) + __popc(users_hi);
        __syncwarp();
        if (row || !b.exec_prio) // criticality-as-priority
            for (int c = lane; c < n; c += 32) {
                int32_t best = INT32_MIN;
                for (int k = 0; k < n; ++k)
                    if (s.exec[k] == s.exec[c] && s.prio[k] > best) best = s.prio[k];
                s.ep[c] = best;
            }
        float Tmin = 3.4e38f;
        for (int c = lane; c < n; c += 32) Tmin = fminf(Tmin, s.T[c]);
        for (int off = 16; off > 0; off >>= 1) Tmin = fminf(Tmin, __shfl_xor_sync(0xffffffffu, Tmin, off));
        __syncwarp();
        for (int c = lane; c < n; c += 32) { // bucket: rank among accelerator users (R2)
            int r = 0;
            for (int k = 0; k < n; ++k) r += (s.dl[k] > 0 && s.prio[k] > s.prio[c]) ? 1 : 0;
            s.bucket[c] = s.dl[c] > 0 ? (int32_t)((int64_t)r * n_buckets / n_users) : -1;
        }
        __syncwarp();
        __nv_bfloat16 *out = X + item * (int64_t)(NCH * NF);
        for (int c = lane; c < NCH; c += 32) {
            float f[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) f[i] = 0.0f;
            if (c < n) {
                const float T = s.T[c], D = s.D[c], E = s.E[c], S = s.S[c];
                const int32_t pc = s.prio[c], xc = s.exec[c], kc = s.core[c], ec = s.ep[c], bc = s.bucket[c];
                int rank = 0;
                float hp_u = 0, hpp_u = 0, hps_u = 0, hpx_d = 0, B = 0, blk = 0;
                for (int h = 0; h < n; ++h) {
                    if (h == c) continue;
                    const bool hi = s.prio[h] > pc;
                    rank += hi ? 1 : 0;
                    if (s.exec[h] == xc) {
                        if (hi) {
                            hp_u += (s.E[h] + s.S[h]) / s.T[h];
                            hpx_d += s.E[h] + s.S[h];
                        } else {
                            B = fmaxf(B, s.Emax[h]);
                        }
                    } else if (s.core[h] == kc && s.ep[h] > ec) {
                        hpp_u += s.E[h] / s.T[h];
                        hpx_d += s.E[h] + s.S[h];
                    }
                    if (s.dl[h] > 0 && hi) hps_u += s.S[h] / s.T[h];
                    if (bc >= 0 && s.dl[h] > 0 && !hi && s.bucket[h] == bc) blk = fmaxf(blk, s.M[h]);
                }
                f[0] = E / T;
                f[1] = S / T;
                f[2] = D / T;
                f[3] = log2f(T / Tmin) * 0.25f;
                f[4] = (float)rank / (float)n;
                f[5] = (float)min(s.dl[c], 16) * (1.0f / 16.0f);
                f[6] = s.Emax[c] / D;
                f[7] = s.M[c] / D;
                f[8] = hp_u;
                f[9] = hpp_u;
                f[10] = hps_u;
                f[11] = B / D;
                f[12] = blk / D;
                f[13] = (E + S) / D;
                f[14] = hpx_d / D;
                f[15] = 1.0f;
#pragma unroll
                for (int i = 0; i < NF; ++i) f[i] = fminf(fmaxf(f[i], 0.0f), 8.0f);
            }
            __nv_bfloat16 v[NF];
#pragma unroll
            for (int i = 0; i < NF; ++i) v[i] = __float2bfloat16_rn(f[i]);
            uint4 *o = (uint4 *)(out + c * NF);
            o[0] = ((const uint4 *)v)[0];
            o[1] = ((const uint4 *)v)[1];
        }
        __syncwarp();
    }
}

} // namespace

int paam_launch_features(const paam_batch *b, const int16_t *ranks, int32_t K, int32_t nmax, int64_t sys0,
                         int64_t n_items, int32_t n_buckets, int64_t kappa, __nv_bfloat16 *X, cudaStream_t stream)
{
    if (n_items <= 0) return PAAM_OK;
    int64_t blocks = (n_items + 7) / 8;
    if (blocks > 32 * (int64_t)b->ctx->n_sm) blocks = 32 * (int64_t)b->ctx->n_sm;
    features_kernel<<<(unsigned)blocks, 256, 0, stream>>>(batch_dev(b), ranks, K < 1 ? 1 : K, nmax, sys0, n_items,
                                                          n_buckets, kappa, X);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}
