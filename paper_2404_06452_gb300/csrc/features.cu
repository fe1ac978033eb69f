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
                                                       int64_t kappa, int32_t slots, __nv_bfloat16 *X,
                                                       const int32_t *sys_list)
{
    __shared__ FeatSmem sm[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FeatSmem &s = sm[warp];
    const int64_t gw = (int64_t)blockIdx.x * 8 + warp, nw = (int64_t)gridDim.x * 8;
    for (int64_t item = gw; item < n_items; item += nw) {
        const int64_t sys = sys_list ? (int64_t)sys_list[sys0 + item / K] : sys0 + item / K;
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
        __nv_bfloat16 *out = X + item * (int64_t)(slots * NF);
        for (int c = lane; c < slots; c += 32) {
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

// ---------------------------------------------------------------------------
// Candidate mode: one CTA per system; a segment of L lanes (16 or 32, at least
// the system's chain count) per candidate order.
//
// The candidate-independent half of each chain's features (0-3, 5-7, 13, 15)
// and the per-executor sums are computed once per system into shared memory.
// For a candidate, lane k of the segment takes the chain at priority position
// k (rank k, 0 = highest), so "higher priority" is "lower lane":
//   - hp sums and B (Lemma 4) run over the lanes of the same executor below /
//     above (a __match_any_sync mask); an executor's priority is that of its
//     lowest lane (criticality-as-priority), and the hpp sums add the
//     per-executor demand of the executors on the core whose lowest lane comes
//     first;
//   - hps is an exclusive prefix sum over the accelerator users; the bucket of
//     a user is floor(rank among users * n_buckets / |U|), non-decreasing
//     along the lanes, so blk (largest M* of a lower user in the same bucket)
//     is a segmented suffix maximum whose segments are contiguous.
// Sums run in priority order rather than chain order; the fp32 results differ
// from the per-item kernel only by rounding.  A rank row that is not a
// permutation of 0..n-1 gets an all-zero feature row.
constexpr int CF_THREADS = 128;

struct CandSmem {
    uint4 tmpl[32][2]; // 16 bf16 features, candidate-independent ones filled in
    float uEpS[32], uE[32], uS[32], EpS[32], Emax[32], M[32], D[32];
    uint8_t x[32], lc[32], user[32];
    float UcpuX[32], EpSX[32];
    float invD[32];                   // 1 / D per chain
    int32_t bkt[32];                  // bucket of the accelerator user of rank r (R2)
    float inv_n;
    uint8_t ord[CF_THREADS / 16][16]; // per 16-lane segment: chain at position k
    uint8_t ord_hi[CF_THREADS / 32][16]; // positions 16..31 of 32-lane segments
};

__device__ __forceinline__ uint32_t bf16_bits(float v)
{
    v = fminf(fmaxf(v, 0.0f), 8.0f);
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

template <int L>
__global__ void __launch_bounds__(CF_THREADS) cand_features_kernel(BatchDev b, const int16_t *ranks, int32_t K,
                                                                   int32_t nmax, int64_t sys0, int64_t n_systems,
                                                                   int32_t n_buckets, int64_t kappa, int32_t slots,
                                                                   __nv_bfloat16 *X, const int32_t *sys_list)
{
    __shared__ CandSmem s;
    constexpr int SEGS = CF_THREADS / L;
    const int t = threadIdx.x, lane = t & 31;
    const int sg = t / L, k = t % L;                               // segment in the block, position in it
    const unsigned full = 0xffffffffu;
    const unsigned segmask = L == 32 ? full : (0xffffu << (lane & 16));
    const unsigned lt = (1u << lane) - 1u;                        // lanes under this one in the warp
    const unsigned gt = ~lt & ~(1u << lane);
    for (int64_t si = blockIdx.x; si < n_systems; si += gridDim.x) {
        const int64_t sys = sys_list ? (int64_t)sys_list[sys0 + si] : sys0 + si;
        const int64_t c0 = b.sys_chain_off[sys];
        const int n = (int)(b.sys_chain_off[sys + 1] - c0);
        const int64_t x0 = b.sys_exec_off[sys];
        const int nx = (int)(b.sys_exec_off[sys + 1] - x0);
        __syncthreads(); // the previous system's tables are no longer read
        // ---- candidate-independent part: thread c < n (all in warp 0) handles chain c
        if (t < 32) {
            float T = 1.0f, Dc = 1.0f, E = 0.0f, S = 0.0f, Em = 0.0f, Mc = 0.0f, tmin = 3.4e38f;
            int dl = 0;
            if (t < n) {
                const int64_t g = c0 + t;
                T = (float)b.T[g];
                Dc = (float)b.D[g];
                tmin = T;
                const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
                double e = 0, emax = 0, sa = 0, m = 0;
                for (int64_t cb = cb0; cb < cb1; ++cb) {
                    const double v = (double)b.E[cb];
                    e += v;
                    emax = v > emax ? v : emax;
                }
                const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
                for (int64_t q = q0; q < q1; ++q) {
                    const double a = (double)b.A[q] + 2.0 * (double)kappa;
                    sa += a;
                    m = a > m ? a : m;
                }
                E = (float)e;
                Em = (float)emax;
                S = (float)sa;
                Mc = (float)m;
                dl = (int)(q1 - q0);
                const int xc = b.exec[g];
                s.uEpS[t] = (E + S) / T;
                s.uE[t] = E / T;
                s.uS[t] = S / T;
                s.EpS[t] = E + S;
                s.Emax[t] = Em;
                s.M[t] = Mc;
                s.D[t] = Dc;
                s.invD[t] = 1.0f / Dc;
                s.x[t] = (uint8_t)xc;
                s.user[t] = dl > 0 ? 1 : 0;
                const int kc = b.exec_core[x0 + xc]; // local core: lowest executor on the same core
                int lcx = xc;
                for (int y = 0; y < xc; ++y)
                    if (b.exec_core[x0 + y] == kc) {
                        lcx = y;
                        break;
                    }
                s.lc[t] = (uint8_t)lcx;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) tmin = fminf(tmin, __shfl_xor_sync(full, tmin, off));
            if (t < n) {
                uint32_t w[8];
                w[0] = bf16_bits(E / T) | bf16_bits(S / T) << 16;
                w[1] = bf16_bits(Dc / T) | bf16_bits(log2f(T / tmin) * 0.25f) << 16;
                w[2] = bf16_bits((float)min(dl, 16) * (1.0f / 16.0f)) << 16;
                w[3] = bf16_bits(Em / Dc) | bf16_bits(Mc / Dc) << 16;
                w[4] = 0;
                w[5] = 0;
                w[6] = bf16_bits((E + S) / Dc) << 16;
                w[7] = bf16_bits(1.0f) << 16;
                s.tmpl[t][0] = make_uint4(w[0], w[1], w[2], w[3]);
                s.tmpl[t][1] = make_uint4(w[4], w[5], w[6], w[7]);
            }
            __syncwarp();
            if (t < nx) { // per executor, in chain order: CPU utilisation and total demand
                float u = 0.0f, es = 0.0f;
                for (int c = 0; c < n; ++c)
                    if (s.x[c] == t) {
                        u += s.uE[c];
                        es += s.EpS[c];
                    }
                s.UcpuX[t] = u;
                s.EpSX[t] = es;
            }
        }
        __syncthreads();
        int n_users = 0;
        for (int c = 0; c < n; ++c) n_users += s.user[c];
        if (t < n_users) s.bkt[t] = (int32_t)((int64_t)t * n_buckets / n_users);
        if (t == 0) s.inv_n = 1.0f / (float)n;
        __syncthreads();
        const float inv_n = s.inv_n;
        // ---- one candidate per segment ---------------------------------------------
        // lane k reads chain k's rank; the next candidate's row is fetched one
        // iteration ahead so its latency overlaps this candidate's work
        const int16_t *rrow = ranks + (sys * K + sg) * (int64_t)nmax + k; // this lane's entry, candidate sg
        const int64_t rstep = (int64_t)SEGS * nmax;
        int r_next = (sg < K && k < n) ? *rrow : -1;
        for (int cand0 = 0; cand0 < K; cand0 += SEGS) {
            const int cand = cand0 + sg;
            const bool live = cand < K; // whole segments are live or not
            const int r = r_next;
            rrow += rstep;
            r_next = (cand + SEGS < K && k < n) ? *rrow : -1;
            const bool in = r >= 0 && r < n;
            unsigned bits = (k < n && in) ? (1u << r) : 0u;
#pragma unroll
            for (int off = L / 2; off > 0; off >>= 1) bits |= __shfl_xor_sync(full, bits, off);
            const unsigned want = n >= 32 ? full : ((1u << n) - 1u);
            const bool valid = live && bits == want;
            // scatter: chain k goes to position r (a permutation: no two lanes collide)
            if (valid && k < n) {
                if (r < 16)
                    s.ord[(sg * L) / 16][r] = (uint8_t)k;
                else
                    s.ord_hi[(sg * L) / 32][r - 16] = (uint8_t)k;
            }
            __syncwarp();
            const int c = (valid && k < n) ? (int)(k < 16 ? s.ord[(sg * L) / 16][k] : s.ord_hi[(sg * L) / 32][k - 16])
                                           : 0;
            __syncwarp();
            const bool act = valid && k < n;
            // this lane's chain (position k)
            const int x = act ? s.x[c] : 255;
            const int lcx = act ? s.lc[c] : 255;
            const bool user = act && s.user[c];
            const float uEpS = act ? s.uEpS[c] : 0.0f, EpS = act ? s.EpS[c] : 0.0f;
            const float Emax = act ? s.Emax[c] : 0.0f, Mc = act ? s.M[c] : 0.0f, iD = act ? s.invD[c] : 1.0f;
            const float uS = act ? s.uS[c] : 0.0f;
            // same executor / same core within this segment
            const unsigned same = __match_any_sync(full, (unsigned)(x | (sg << 8))) & segmask;
            const unsigned samecore = __match_any_sync(full, (unsigned)(lcx | (sg << 8))) & segmask;
            const int first = __ffs(same) - 1;                       // executor's highest-priority lane
            const unsigned firsts = __ballot_sync(full, act && first == lane) & segmask;
            // hp: same executor, higher priority (lower lanes); B: same executor, lower priority
            float hpU = 0.0f, hpE = 0.0f, B = 0.0f;
            unsigned mlow = act ? (same & lt) : 0u, mhigh = act ? (same & gt) : 0u;
            while (__any_sync(full, mlow | mhigh)) {
                const int jl = mlow ? __ffs(mlow) - 1 : lane;
                const int jh = mhigh ? __ffs(mhigh) - 1 : lane;
                const float vU = __shfl_sync(full, uEpS, jl), vE = __shfl_sync(full, EpS, jl);
                const float vB = __shfl_sync(full, Emax, jh);
                if (mlow) {
                    hpU += vU;
                    hpE += vE;
                    mlow &= mlow - 1;
                }
                if (mhigh) {
                    B = fmaxf(B, vB);
                    mhigh &= mhigh - 1;
                }
            }
            // hpp: executors on the core whose highest-priority lane precedes this executor's
            const float ux = act ? s.UcpuX[x] : 0.0f, ex = act ? s.EpSX[x] : 0.0f;
            float hppU = 0.0f, hppE = 0.0f;
            unsigned mx = act ? (firsts & samecore & ((1u << first) - 1u)) : 0u;
            while (__any_sync(full, mx)) {
                const int jx = mx ? __ffs(mx) - 1 : lane;
                const float vU = __shfl_sync(full, ux, jx), vE = __shfl_sync(full, ex, jx);
                if (mx) {
                    hppU += vU;
                    hppE += vE;
                    mx &= mx - 1;
                }
            }
            // hps: exclusive prefix sum over users; user rank and bucket
            float incl = user ? uS : 0.0f;
#pragma unroll
            for (int off = 1; off < L; off <<= 1) {
                const float v = __shfl_up_sync(full, incl, off, L);
                if (k >= off) incl += v;
            }
            float hps = __shfl_up_sync(full, incl, 1, L);
            if (k == 0) hps = 0.0f;
            const unsigned users = __ballot_sync(full, user) & segmask;
            const int urank = __popc(users & lt);
            const int key = urank < n_users ? s.bkt[urank] : 0x7fffffff;
            // blk: segmented suffix maximum of M* over users with the same key
            float acc = user ? Mc : 0.0f;
#pragma unroll
            for (int off = 1; off < L; off <<= 1) {
                const float v = __shfl_down_sync(full, acc, off, L);
                const int kk = __shfl_down_sync(full, key, off, L);
                if (k + off < n && kk == key) acc = fmaxf(acc, v);
            }
            const float nxt = __shfl_down_sync(full, acc, 1, L);
            const int nkey = __shfl_down_sync(full, key, 1, L);
            const float blk = (user && k + 1 < n && nkey == key) ? nxt : 0.0f;
            // the row: chain c's slot gets the template patched with this candidate's terms
            if (live) {
                uint4 *out = reinterpret_cast<uint4 *>(X + ((si * K + cand) * (int64_t)(slots * NF)));
                if (act) {
                    uint4 lo = s.tmpl[c][0], hi = s.tmpl[c][1];
                    lo.z |= bf16_bits((float)k * inv_n);                       // 4: rank / n
                    hi.x = bf16_bits(hpU) | bf16_bits(hppU) << 16;             // 8, 9
                    hi.y = bf16_bits(hps) | bf16_bits(B * iD) << 16;           // 10, 11
                    hi.z |= bf16_bits(blk * iD);                               // 12
                    hi.w |= bf16_bits((hpE + hppE) * iD);                      // 14
                    out[2 * c] = lo;
                    out[2 * c + 1] = hi;
                }
                const int first_pad = valid ? n : 0;
                for (int q = first_pad + k; q < slots; q += L) {
                    out[2 * q] = make_uint4(0, 0, 0, 0);
                    out[2 * q + 1] = make_uint4(0, 0, 0, 0);
                }
            }
        }
    }
}

} // namespace

int paam_launch_features(const paam_batch *b, const int16_t *ranks, int32_t K, int32_t nmax, int64_t sys0,
                         int64_t n_items, int32_t n_buckets, int64_t kappa, int32_t width, __nv_bfloat16 *X,
                         cudaStream_t stream, const int32_t *sys_list)
{
    if (n_items <= 0) return PAAM_OK;
    if (width % NF || width / NF < b->max_chains || width > NCH * NF) return PAAM_E_INVAL;
    const int slots = width / NF;
    K = K < 1 ? 1 : K;
    if (ranks && b->max_chains <= 32 && b->max_exec <= 32 && n_items % K == 0) {
        const int64_t n_systems = n_items / K;
        // one wave of resident CTAs, each taking every so-many-th system: a grid
        // above residency leaves a partial second wave behind the first
        const bool l16 = b->max_chains <= 16;
        static int resident[2] = {0, 0};
        int &per_sm = resident[l16 ? 0 : 1];
        if (per_sm == 0) {
            int r = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &r, l16 ? cand_features_kernel<16> : cand_features_kernel<32>, CF_THREADS, 0) != cudaSuccess ||
                r < 1) {
                cudaGetLastError();
                r = 8;
            }
            per_sm = r;
        }
        int64_t blocks = n_systems;
        if (blocks > (int64_t)per_sm * b->ctx->n_sm) blocks = (int64_t)per_sm * b->ctx->n_sm;
        if (l16)
            cand_features_kernel<16><<<(unsigned)blocks, CF_THREADS, 0, stream>>>(
                batch_dev(b), ranks, K, nmax, sys0, n_systems, n_buckets, kappa, slots, X, sys_list);
        else
            cand_features_kernel<32><<<(unsigned)blocks, CF_THREADS, 0, stream>>>(
                batch_dev(b), ranks, K, nmax, sys0, n_systems, n_buckets, kappa, slots, X, sys_list);
    } else {
        int64_t blocks = (n_items + 7) / 8;
        if (blocks > 32 * (int64_t)b->ctx->n_sm) blocks = 32 * (int64_t)b->ctx->n_sm;
        features_kernel<<<(unsigned)blocks, 256, 0, stream>>>(batch_dev(b), ranks, K, nmax, sys0, n_items,
                                                              n_buckets, kappa, slots, X, sys_list);
    }
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}
