// analyze_wide.cu -- exact int64 analysis of PAAM (Sec. IV-F, Theorem 1) for
// systems whose times do not fit the 32-bit fast path (analyze_fast.cu).
//
// A group of G lanes analyses one system at a time.  The system's chain table
// lives in shared memory.  Set-up work is spread over chains (lane c handles
// chains c, c+G, ...): per-chain aggregates, bucket map, blocking terms and
// the per-segment handling-time fixed points (Lemma 2), which are independent
// across chains.  The chain recurrences of Theorem 1 then run one chain at a
// time in an order where every needed H*_h is final; inside each iteration
// the lanes split the interfering chains and combine partial sums with warp
// shuffles.
#include "internal.cuh"

namespace {

constexpr int64_t kInf = INT64_MAX;

template <int MAXN>
struct SysSmem {
    int64_t T[MAXN], D[MAXN], E[MAXN], S[MAXN], Hs[MAXN], B[MAXN], blk[MAXN], Hseg[MAXN];
    int64_t Emax[MAXN], M[MAXN], seglo[MAXN], hold[MAXN];
    int32_t prio[MAXN], eprio[MAXN], delta[MAXN], core[MAXN], exec[MAXN], bucket[MAXN];
    uint8_t spin[MAXN], status[MAXN], order[MAXN];
};

template <int G>
__device__ __forceinline__ unsigned group_mask()
{
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

template <int G>
__device__ __forceinline__ int64_t group_sum(int64_t v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

template <int G>
__device__ __forceinline__ int group_or(int v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(mask, v, off);
    return v;
}

// Lemma 1 (Eq. 2): arrivals in a window t >= 0 are at most ceil(t / T) + 1
__device__ __forceinline__ int64_t arrivals(int64_t t, int64_t T) { return (t + T - 1) / T + 1; }

template <int G, int MAXN>
__device__ void analyze_system(const BatchDev &b, const AnalysisParams &p, int64_t item,
                               SysSmem<MAXN> &s, int lane, unsigned gmask, int64_t *__restrict__ R_out,
                               uint8_t *__restrict__ st_out, uint8_t *__restrict__ verdict)
{
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int base_lane = (int)(threadIdx.x & 31u) & ~(G - 1);
        if (__shfl_sync(gmask, cand_pruned(p, sys, cand) ? 1 : 0, base_lane)) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    const int64_t x0 = b.sys_exec_off[sys];
    const int64_t kappa2 = 2 * p.kappa, eps = p.eps;
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority

    // ---- chain aggregates (Sec. II-C; A* = A + 2 kappa) -------------------
    int rank_bad = 0;
    unsigned long long rbits = 0;
    for (int c = lane; c < n; c += G) {
        const int64_t g = c0 + c;
        s.T[c] = b.T[g];
        s.D[c] = b.D[g];
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[c];
            if (r < 0 || r >= n) rank_bad = 1;
            else rbits |= 1ull << r;
            s.prio[c] = n - 1 - r;
        } else {
            s.prio[c] = b.prio[g];
        }
        const int x = b.exec[g];
        s.exec[c] = x;
        s.spin[c] = b.spin[g];
        s.core[c] = b.exec_core[x0 + x];
        s.eprio[c] = xprio ? xprio[x0 + x] : 0;
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        int64_t E = 0, Emax = 0, S = 0, M = 0;
        for (int64_t cb = cb0; cb < cb1; ++cb) {
            const int64_t e = b.E[cb];
            E += e;
            Emax = e > Emax ? e : Emax;
        }
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        for (int64_t q = q0; q < q1; ++q) {
            const int64_t a = b.A[q] + kappa2;
            S += a;
            M = a > M ? a : M;
        }
        s.E[c] = E;
        s.Emax[c] = Emax;
        s.S[c] = S;
        s.M[c] = M;
        s.delta[c] = (int32_t)(q1 - q0);
        s.seglo[c] = q0;
    }
    __syncwarp(gmask);
    if (rank_row) { // a candidate must be a permutation of 0..n-1
        rank_bad = group_or<G>(rank_bad, gmask);
        for (int off = G / 2; off > 0; off >>= 1) rbits |= __shfl_xor_sync(gmask, rbits, off);
        const unsigned long long all = n >= 64 ? ~0ull : ((1ull << n) - 1);
        if (rank_bad || rbits != all) {
            if (lane == 0) {
                atomicExch(p.err, PAAM_E_INVAL);
                if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = 0;
            }
            __syncwarp(gmask);
            return;
        }
    }

    // ---- executor priorities, buckets (R2), blocking terms ----------------
    int n_users = 0;
    for (int k = 0; k < n; ++k) n_users += s.delta[k] > 0;
    for (int c = lane; c < n; c += G) {
        if (!xprio) { // criticality-as-priority: highest chain priority on the executor
            int32_t best = INT32_MIN;
            for (int k = 0; k < n; ++k)
                if (s.exec[k] == s.exec[c] && s.prio[k] > best) best = s.prio[k];
            s.eprio[c] = best;
        }
        // bucket of c: rank among accelerator users, split into n evenly sized groups
        int32_t bucket = -1;
        if (s.delta[c] > 0) {
            int r = 0;
            for (int k = 0; k < n; ++k) r += (s.delta[k] > 0 && s.prio[k] > s.prio[c]);
            bucket = (int32_t)((int64_t)r * p.n_buckets / n_users);
        }
        s.bucket[c] = bucket;
    }
    __syncwarp(gmask);
    for (int c = lane; c < n; c += G) {
        const int32_t bucket_c = s.bucket[c];
        int64_t blk = 0, B = 0;
        for (int l = 0; l < n; ++l) {
            if (s.prio[l] >= s.prio[c]) continue;
            if (s.exec[l] == s.exec[c] && s.Emax[l] > B) B = s.Emax[l]; // Lemma 4
            if (bucket_c >= 0 && s.bucket[l] == bucket_c && s.M[l] > blk) blk = s.M[l]; // R2-R3
        }
        s.blk[c] = blk;
        s.B[c] = B;
        // position in an order that puts every needed H*_h first:
        // executor priority, then chain priority, both descending
        int pos = 0;
        for (int k = 0; k < n; ++k)
            pos += (s.eprio[k] > s.eprio[c]) || (s.eprio[k] == s.eprio[c] && s.prio[k] > s.prio[c]);
        s.order[pos] = (uint8_t)c;
    }
    __syncwarp(gmask);

    // ---- Lemma 2 (Eq. 3): per-segment handling times, chains in parallel ---
    // Safe blocking (blocking_mode 1) also needs, per chain, its longest
    // callback with every request: hold = max_i E_i + sum over i's segments
    // of (Lemma 2 bound + eps), infinite when a segment has no bound.
    const bool safe = p.blocking_mode == 1;
    for (int c = lane; c < n; c += G) {
        int64_t Hseg = 0, hold = 0;
        const int64_t Dc = s.D[c], blk = s.blk[c];
        const int32_t pc = s.prio[c];
        const int64_t g = c0 + c;
        const int64_t cb1 = b.chain_cb_off[g + 1];
        for (int64_t cb = b.chain_cb_off[g]; cb < cb1 && Hseg != kInf; ++cb) {
            int64_t t = b.E[cb];
            const int64_t q1 = b.cb_seg_off[cb + 1];
            for (int64_t q = b.cb_seg_off[cb]; q < q1 && Hseg != kInf; ++q) {
                const int64_t a = b.A[q] + kappa2;
                int64_t h = a + blk;
                for (;;) {
                    if (h > Dc) {
                        Hseg = kInf;
                        break;
                    }
                    int64_t nh = a + blk;
                    for (int k = 0; k < n; ++k)
                        if (s.delta[k] > 0 && s.prio[k] > pc) nh += arrivals(h, s.T[k]) * s.S[k];
                    if (nh == h) break; // each step raises some ceil(h/T_k): at most n*(D/Tmin+1) steps
                    h = nh;
                }
                if (Hseg != kInf) {
                    Hseg += h;
                    t += h + eps;
                }
            }
            if (safe && t > hold) hold = t;
        }
        s.Hseg[c] = Hseg;
        s.hold[c] = Hseg == kInf ? kInf : hold;
    }
    __syncwarp(gmask);
    if (safe) { // B_c: the longest hold of a lower-priority chain on the same executor
        for (int c = lane; c < n; c += G) {
            int64_t B = 0;
            for (int l = 0; l < n; ++l)
                if (s.exec[l] == s.exec[c] && s.prio[l] < s.prio[c] && s.hold[l] > B) B = s.hold[l];
            s.B[c] = B;
        }
        __syncwarp(gmask);
    }

    // ---- Theorem 1 (Eq. 6) chain by chain ----------------------------------
    for (int k = 0; k < n; ++k) {
        const int c = s.order[k];
        const int32_t pc = s.prio[c], ec = s.exec[c], ep = s.eprio[c], cc = s.core[c];
        // dependencies: H* of hp(c) and of spinning hpp(c) chains
        int dep_bad = 0;
        for (int h = lane; h < n; h += G) {
            if (h == c) continue;
            const bool hp = s.exec[h] == ec && s.prio[h] > pc;
            const bool hpp_spin = s.exec[h] != ec && s.core[h] == cc && s.eprio[h] > ep && s.spin[h];
            if ((hp || hpp_spin) && s.status[h] != PAAM_ST_SCHED) dep_bad = 1;
        }
        dep_bad = group_or<G>(dep_bad, gmask);
        int64_t R = -1;
        uint8_t st = PAAM_ST_DEP;
        int64_t hs_final = 0;
        if (!dep_bad && s.B[c] == kInf) { // unbounded safe blocking
            st = PAAM_ST_OVERRUN;
        } else if (!dep_bad) {
            const int64_t Dc = s.D[c], Bc = s.B[c], Ec = s.E[c], Sc = s.S[c], Hseg = s.Hseg[c];
            const int64_t dc = s.delta[c];
            const int64_t own = Sc + dc * s.blk[c];
            const int64_t deps = dc * eps;
            // start: B + E + H* with the interference part of Eq. 4 empty
            int64_t Rc = Bc + Ec + (dc > 0 ? (Hseg < own ? Hseg : own) + deps : 0);
            st = PAAM_ST_OVERRUN;
            for (;;) {
                if (Rc > Dc) break;
                int64_t cpu = 0, acc = 0;
                for (int h = lane; h < n; h += G) {
                    if (h == c) continue;
                    const int64_t m = arrivals(Rc, s.T[h]);
                    if (s.exec[h] == ec) {
                        if (s.prio[h] > pc) cpu += m * (s.E[h] + s.Hs[h]); // hp(c)
                    } else if (s.core[h] == cc && s.eprio[h] > ep) {          // hpp(c)
                        cpu += m * (s.E[h] + (s.spin[h] ? s.Hs[h] : (int64_t)s.delta[h] * eps));
                    }
                    if (s.delta[h] > 0 && s.prio[h] > pc) acc += m * s.S[h]; // Eq. 4
                }
                cpu = group_sum<G>(cpu, gmask);
                acc = group_sum<G>(acc, gmask);
                int64_t hs = 0;
                if (dc > 0) {
                    const int64_t hch = own + acc;
                    hs = (Hseg < hch ? Hseg : hch) + deps; // Eq. 1 with min(Eq. 3, Eq. 4)
                }
                const int64_t Rn = Bc + Ec + hs + cpu;
                if (Rn == Rc) {
                    st = PAAM_ST_SCHED;
                    hs_final = hs;
                    break;
                }
                Rc = Rn;
            }
            R = st == PAAM_ST_SCHED ? Rc : -1;
        }
        if (lane == 0) {
            s.status[c] = st;
            s.Hs[c] = hs_final;
        }
        __syncwarp(gmask);
        if (lane == 0 && !rank_row) {
            R_out[c0 + c] = R;
            st_out[c0 + c] = st;
        }
    }
    int ok = 1;
    for (int c = lane; c < n; c += G) ok &= s.status[c] == PAAM_ST_SCHED;
    for (int off = G / 2; off > 0; off >>= 1) ok &= __shfl_xor_sync(gmask, ok, off);
    if (lane == 0) {
        if (rank_row) {
            if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = (uint8_t)ok;
            if (ok) atomicMin(p.first_ok + sys, cand);
        } else if (verdict) {
            verdict[sys] = (uint8_t)ok;
        }
    }
    __syncwarp(gmask);
}

// Systems are either all of the batch (list == nullptr) or the list
// list[0 .. *count).
template <int G, int MAXN>
__global__ void __launch_bounds__(256) analyze_wide_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                           uint8_t *st, uint8_t *verdict,
                                                           const int32_t *list, const int32_t *count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    SysSmem<MAXN> &s = reinterpret_cast<SysSmem<MAXN> *>(smem_raw)[grp];
    const unsigned gmask = group_mask<G>();
    const int64_t n = list ? (int64_t)*count : (p.K > 0 ? b.n_sys * p.K : b.n_sys);
    for (int64_t i = (int64_t)blockIdx.x * groups + grp; i < n; i += (int64_t)gridDim.x * groups) {
        const int64_t item = list ? (int64_t)list[i] : i;
        analyze_system<G, MAXN>(b, p, item, s, lane, gmask, R, st, verdict);
    }
}

} // namespace

int paam_launch_wide(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st,
                     uint8_t *verdict, const int32_t *list, const int32_t *count, int64_t max_items,
                     cudaStream_t stream)
{
    constexpr int G = 32, MAXN = 64;
    const int threads = 256;
    const int groups = threads / G;
    const size_t smem = sizeof(SysSmem<MAXN>) * groups;
    auto kern = analyze_wide_kernel<G, MAXN>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, list, count);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}
