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

// NACC accelerators (rule R1: one server each, analysed on its own); the
// per-accelerator tables hold, for each chain, its requests to that
// accelerator only.  delta is the chain's total number of segments.
template <int MAXN, int NACC>
struct SysSmem {
    int64_t T[MAXN], D[MAXN], E[MAXN], Hs[MAXN], B[MAXN];
    int64_t Emax[MAXN], seglo[MAXN], hold[MAXN];
    uint8_t cap[MAXN]; // 1: a segment recurrence of the chain reached kIterCap evaluations
    int64_t S[MAXN][NACC], M[MAXN][NACC], blk[MAXN][NACC], Hseg[MAXN][NACC];
    int32_t prio[MAXN], eprio[MAXN], delta[MAXN], core[MAXN], exec[MAXN];
    int32_t dA[MAXN][NACC], bucket[MAXN][NACC];
    uint8_t spin[MAXN], status[MAXN], order[MAXN];
    // ceil(t / T) by multiply and shift when the system's periods and deadlines
    // are below 2^30 (every window the loops test is at most a deadline)
    uint32_t tm1[MAXN], mg[MAXN];
    uint8_t sh[MAXN];
};

// accelerator of segment q (indices were checked against PAAM_MAX_ACC at load)
template <int NACC>
__device__ __forceinline__ int acc_of(const BatchDev &b, int64_t q)
{
    if constexpr (NACC == 1) {
        return 0;
    } else {
        const int u = b.acc ? b.acc[q] : 0;
        return u < NACC ? u : NACC - 1;
    }
}

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
__device__ __forceinline__ int group_and(int v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v &= __shfl_xor_sync(mask, v, off);
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

// The same for 0 <= t <= D < 2^30 and T < 2^30: t + T - 1 < 2^31, and with
// m = ceil(2^(31 + l) / T), l = ceil(log2 T), floor(x / T) = (x m) >> (31 + l)
// for every x < 2^31 (Granlund and Montgomery 1994, Theorem 4.2 with N = 31).
template <int MAXN, int NACC>
__device__ __forceinline__ int64_t arrivals_of(const SysSmem<MAXN, NACC> &s, int k, int64_t t, bool fast)
{
    if (fast) return (int64_t)((((uint64_t)((uint32_t)t + s.tm1[k])) * s.mg[k]) >> s.sh[k]) + 1;
    return arrivals(t, s.T[k]);
}

template <int G, int MAXN, int NACC>
__device__ void analyze_system(const BatchDev &b, const AnalysisParams &p, int64_t item,
                               SysSmem<MAXN, NACC> &s, int lane, unsigned gmask, int64_t *__restrict__ R_out,
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
    // target mode: the candidate's verdict is the status of this one chain
    const int tgt = (p.K > 0 && p.target) ? (int)p.target[sys * p.Kc + cand_of(p, sys, cand)] : -1;
    if (p.K > 0 && p.target && (tgt < 0 || tgt >= n)) return;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority

    // ---- chain aggregates (Sec. II-C; A* = A + 2 kappa) -------------------
    int rank_bad = 0;
    unsigned long long rbits = 0;
    int small = 1; // every period and deadline of the system below 2^30
    for (int c = lane; c < n; c += G) {
        const int64_t g = c0 + c;
        s.T[c] = b.T[g];
        s.D[c] = b.D[g];
        if (b.T[g] < (1ll << 30) && b.D[g] < (1ll << 30)) {
            const uint32_t Tu = (uint32_t)b.T[g];
            const uint32_t l = Tu > 1 ? 32u - (uint32_t)__clz(Tu - 1u) : 0u;
            s.mg[c] = (uint32_t)(((1ull << (31 + l)) + Tu - 1u) / Tu);
            s.sh[c] = (uint8_t)(31 + l);
            s.tm1[c] = Tu - 1u;
        } else {
            small = 0;
        }
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
        int64_t E = 0, Emax = 0;
        for (int64_t cb = cb0; cb < cb1; ++cb) {
            const int64_t e = b.E[cb];
            E += e;
            Emax = e > Emax ? e : Emax;
        }
        int64_t S[NACC], M[NACC];
        int32_t dl[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) S[a] = M[a] = dl[a] = 0;
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        for (int64_t q = q0; q < q1; ++q) {
            const int64_t a = b.A[q] + kappa2;
            const int u = acc_of<NACC>(b, q);
            S[u] += a;
            M[u] = a > M[u] ? a : M[u];
            dl[u] += 1;
        }
        s.E[c] = E;
        s.Emax[c] = Emax;
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            s.S[c][a] = S[a];
            s.M[c][a] = M[a];
            s.dA[c][a] = dl[a];
        }
        s.delta[c] = (int32_t)(q1 - q0);
        s.seglo[c] = q0;
    }
    __syncwarp(gmask);
    const bool fast = group_and<G>(small, gmask) != 0;
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
    int n_users[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
        n_users[a] = 0;
        for (int k = 0; k < n; ++k) n_users[a] += s.dA[k][a] > 0;
    }
    for (int c = lane; c < n; c += G) {
        if (!xprio) { // criticality-as-priority: highest chain priority on the executor
            int32_t best = INT32_MIN;
            for (int k = 0; k < n; ++k)
                if (s.exec[k] == s.exec[c] && s.prio[k] > best) best = s.prio[k];
            s.eprio[c] = best;
        }
        // bucket of c at each accelerator: rank among that accelerator's users,
        // split into n evenly sized groups
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            int32_t bucket = -1;
            if (s.dA[c][a] > 0) {
                int r = 0;
                for (int k = 0; k < n; ++k) r += (s.dA[k][a] > 0 && s.prio[k] > s.prio[c]);
                bucket = (int32_t)((int64_t)r * p.n_buckets / n_users[a]);
            }
            s.bucket[c][a] = bucket;
        }
    }
    __syncwarp(gmask);
    for (int c = lane; c < n; c += G) {
        int64_t blk[NACC], B = 0;
#pragma unroll
        for (int a = 0; a < NACC; ++a) blk[a] = 0;
        for (int l = 0; l < n; ++l) {
            if (s.prio[l] >= s.prio[c]) continue;
            if (s.exec[l] == s.exec[c] && s.Emax[l] > B) B = s.Emax[l]; // Lemma 4
#pragma unroll
            for (int a = 0; a < NACC; ++a) { // R2-R3, at each accelerator
                const int32_t bucket_c = s.bucket[c][a];
                if (bucket_c >= 0 && s.bucket[l][a] == bucket_c && s.M[l][a] > blk[a]) blk[a] = s.M[l][a];
            }
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a) s.blk[c][a] = blk[a];
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
        int64_t Hseg[NACC], hold = 0;
        bool any_inf = false; // some segment of the chain has no bound
        bool capped = false;
#pragma unroll
        for (int a = 0; a < NACC; ++a) Hseg[a] = 0;
        const int64_t Dc = s.D[c];
        const int32_t pc = s.prio[c];
        const int64_t g = c0 + c;
        const int64_t cb1 = b.chain_cb_off[g + 1];
        // with one accelerator nothing after an unbounded segment matters
        for (int64_t cb = b.chain_cb_off[g]; cb < cb1 && !(NACC == 1 && any_inf); ++cb) {
            int64_t t = b.E[cb];
            const int64_t q1 = b.cb_seg_off[cb + 1];
            for (int64_t q = b.cb_seg_off[cb]; q < q1; ++q) {
                const int u = acc_of<NACC>(b, q);
                if (Hseg[u] == kInf) { // this accelerator's sum is already unbounded
                    any_inf = true;
                    continue;
                }
                const int64_t a = b.A[q] + kappa2, blk = s.blk[c][u];
                int64_t h = a + blk;
                bool inf = false;
                uint32_t ev = 0;
                for (;;) {
                    if (h > Dc) {
                        inf = true;
                        break;
                    }
                    if (ev++ == kIterCap) {
                        inf = capped = true;
                        break;
                    }
                    int64_t nh = a + blk;
                    for (int k = 0; k < n; ++k) // hps at this segment's accelerator
                        if (s.dA[k][u] > 0 && s.prio[k] > pc) nh += arrivals_of(s, k, h, fast) * s.S[k][u];
                    if (nh == h) break; // each step raises some ceil(h/T_k): at most n*(D/Tmin+1) steps
                    h = nh;
                }
                if (inf) {
                    Hseg[u] = kInf;
                    any_inf = true;
                } else {
                    Hseg[u] += h;
                    t += h + eps;
                }
            }
            if (safe && t > hold) hold = t;
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a) s.Hseg[c][a] = Hseg[a];
        s.hold[c] = any_inf ? kInf : hold;
        s.cap[c] = capped ? 1 : 0;
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
            const int64_t Dc = s.D[c], Bc = s.B[c], Ec = s.E[c];
            const int64_t dc = s.delta[c];
            const int64_t deps = dc * eps;
            int64_t own[NACC], h0 = 0;
            bool uses[NACC]; // accelerators chain c requests (the same in every lane of the group)
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
                uses[a] = s.dA[c][a] > 0;
                own[a] = s.S[c][a] + (int64_t)s.dA[c][a] * s.blk[c][a];
                if (uses[a]) h0 += s.Hseg[c][a] < own[a] ? s.Hseg[c][a] : own[a];
            }
            // start: B + E + H* with the interference parts of Eq. 4 empty
            int64_t Rc = Bc + Ec + (dc > 0 ? h0 + deps : 0);
            st = PAAM_ST_OVERRUN;
            uint32_t ev = 0;
            for (;;) {
                if (Rc > Dc) break;
                if (ev++ == kIterCap) {
                    st = PAAM_ST_ITERCAP;
                    break;
                }
                int64_t cpu = 0, acc[NACC];
#pragma unroll
                for (int a = 0; a < NACC; ++a) acc[a] = 0;
                for (int h = lane; h < n; h += G) {
                    if (h == c) continue;
                    const int64_t m = arrivals_of(s, h, Rc, fast);
                    if (s.exec[h] == ec) {
                        if (s.prio[h] > pc) cpu += m * (s.E[h] + s.Hs[h]); // hp(c)
                    } else if (s.core[h] == cc && s.eprio[h] > ep) {          // hpp(c)
                        cpu += m * (s.E[h] + (s.spin[h] ? s.Hs[h] : (int64_t)s.delta[h] * eps));
                    }
                    if (s.prio[h] > pc)
#pragma unroll
                        for (int a = 0; a < NACC; ++a)
                            if (uses[a] && s.dA[h][a] > 0) acc[a] += m * s.S[h][a]; // Eq. 4 at accelerator a
                }
                cpu = group_sum<G>(cpu, gmask);
                int64_t hs = 0;
#pragma unroll
                for (int a = 0; a < NACC; ++a) {
                    if (uses[a]) { // Eq. 1 with min(Eq. 3, Eq. 4), summed over accelerators (R1)
                        acc[a] = group_sum<G>(acc[a], gmask);
                        const int64_t hch = own[a] + acc[a];
                        hs += s.Hseg[c][a] < hch ? s.Hseg[c][a] : hch;
                    }
                }
                if (dc > 0) hs += deps;
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
        if (s.cap[c] && st != PAAM_ST_DEP) { // a segment bound was cut short
            st = PAAM_ST_ITERCAP;
            R = -1;
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
        if (c == tgt) break; // chains after the target cannot change its result
    }
    if (tgt >= 0) {
        if (lane == 0) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = (uint8_t)(s.status[tgt] == PAAM_ST_SCHED);
        __syncwarp(gmask);
        return;
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
template <int G, int MAXN, int NACC>
__global__ void __launch_bounds__(256) analyze_wide_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                           uint8_t *st, uint8_t *verdict,
                                                           const int32_t *list, const int32_t *count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    SysSmem<MAXN, NACC> &s = reinterpret_cast<SysSmem<MAXN, NACC> *>(smem_raw)[grp];
    const unsigned gmask = group_mask<G>();
    const int64_t n = list ? (int64_t)*count : (p.K > 0 ? b.n_sys * p.K : b.n_sys);
    for_each_item<G>(p, n, grp, groups, lane, gmask, [&](int64_t i) {
        const int64_t item = list ? (int64_t)list[i] : i;
        analyze_system<G, MAXN, NACC>(b, p, item, s, lane, gmask, R, st, verdict);
    });
}

} // namespace

namespace {

template <int G, int MAXN, int NACC>
int launch_wide_g(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, cudaStream_t stream)
{
    const int threads = 256;
    const int groups = threads / G;
    const size_t smem = sizeof(SysSmem<MAXN, NACC>) * groups;
    auto kern = analyze_wide_kernel<G, MAXN, NACC>;
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

// batches of at most 16 chains per system: 16 lanes and 16-chain tables, so
// that no lane idles in the loops over chains
template <int NACC>
int launch_wide_n(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, cudaStream_t stream)
{
    if (bt->max_chains <= 16)
        return launch_wide_g<16, 16, NACC>(bt, p, R, st, verdict, list, count, max_items, stream);
    return launch_wide_g<32, 64, NACC>(bt, p, R, st, verdict, list, count, max_items, stream);
}

} // namespace

int paam_launch_wide(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st,
                     uint8_t *verdict, const int32_t *list, const int32_t *count, int64_t max_items,
                     cudaStream_t stream)
{
    // tables for as many accelerators as the batch uses (validation recorded the largest index)
    const unsigned long long used = bt->acc ? bt->stats[ST_ACCMAX] + 1 : 1;
    static_assert(PAAM_MAX_ACC == 4, "instantiations below cover 1..4 accelerators");
    if (used >= 4) return launch_wide_n<4>(bt, p, R, st, verdict, list, count, max_items, stream);
    if (used == 3) return launch_wide_n<3>(bt, p, R, st, verdict, list, count, max_items, stream);
    if (used == 2) return launch_wide_n<2>(bt, p, R, st, verdict, list, count, max_items, stream);
    return launch_wide_n<1>(bt, p, R, st, verdict, list, count, max_items, stream);
}
