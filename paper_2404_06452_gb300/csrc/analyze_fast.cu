// analyze_fast.cu -- the analysis kernels of the hot path (Sec. IV-F).
//
// Every system is analysed exactly; this file holds the fast path for systems
// whose periods, deadlines and per-chain CPU and accelerator sums stay below
// 2^30 ns (about one second).  Under that bound every window t of the fixed
// points fits 31 bits, so the arrival count ceil(t / T) of Lemma 1 is an exact
// 32x32->64 multiply and shift (division by an invariant integer, Granlund &
// Montgomery 1994, Theorem 4.2 with N = 31), products mu * C fit 64 bits and
// sums never overflow (the batch passed the int64 range check at load time).
// Systems outside the bound go to the int64 kernel (analyze_wide.cu); systems
// with more chains than the configuration's table go to a wider configuration.
//
// Work split: a group of G lanes owns one system; its chain table sits in
// shared memory.  Set-up runs lanes over chains: aggregates (Sec. II-C),
// interferer sets as bitmasks -- hp and hpp (Lemma 4, Theorem 1) and hps
// (Eq. 3) --, bucket (rank among accelerator users = popcount of hps, R2),
// blocking (Eq. 3, Lemma 4) and the per-segment fixed points of Lemma 2.  The
// chain recurrences of Theorem 1 then run in an order where every needed H*_h
// is final; within an iteration the lanes split the interferer set and add
// their partial sums with warp shuffles.
#include "internal.cuh"

namespace {

constexpr uint64_t kFit = 1ull << 30; // fast-path bound on times and per-chain sums
constexpr uint32_t kInf32 = 0xFFFFFFFFu;

template <int MAXN>
struct MaskOf {
    using type = uint64_t;
};
template <>
struct MaskOf<16> {
    using type = uint32_t;
};
template <>
struct MaskOf<32> {
    using type = uint32_t;
};

template <int MAXN>
struct FastSmem {
    using Mask = typename MaskOf<MAXN>::type;
    // interferer records, read inside the fixed-point loops
    uint2 tm[MAXN];      // {T - 1, magic} for ceil(t / T)
    uint32_t S[MAXN];    // S*_h: accelerator demand per job (sum of A + 2 kappa)
    uint32_t Ehp[MAXN];  // E_h + H*_h (H* added once h is analysed)
    uint32_t Ehpp[MAXN]; // E_h + spin(h): H*_h if h spins, else delta_h eps
    uint8_t sh[MAXN];    // shift of the magic division
    uint8_t order[MAXN]; // analysis order
    uint8_t spin[MAXN];
    uint8_t cap[MAXN];   // 1: a segment recurrence reached kIterCap evaluations
    // per chain: interferer sets and the terms of its own recurrence
    Mask hp[MAXN], hpp[MAXN], hps[MAXN];
    uint32_t D[MAXN], B[MAXN], E[MAXN], blk[MAXN], Hseg[MAXN], R[MAXN], dlt[MAXN];
    uint32_t seg0[MAXN]; // first segment, relative to the system's first segment
    // set-up only
    int2 pe[MAXN];             // {chain priority, executor priority}
    int2 xk[MAXN];             // {executor, core}
    Mask lower_x[MAXN];        // lower-priority chains on the same executor
    int32_t bucket[MAXN];      // server bucket of an accelerator user (R2), else -1
    uint32_t Emax[MAXN], M[MAXN], Amin[MAXN];
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

template <int G, typename V>
__device__ __forceinline__ V group_sum(V v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

template <int G, typename V>
__device__ __forceinline__ V group_or(V v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(mask, v, off);
    return v;
}

template <typename Mask>
__device__ __forceinline__ int popc(Mask m)
{
    if constexpr (sizeof(Mask) == 8)
        return __popcll(m);
    else
        return __popc(m);
}

template <typename Mask>
__device__ __forceinline__ int lowest(Mask m)
{
    if constexpr (sizeof(Mask) == 8)
        return __ffsll((long long)m) - 1;
    else
        return __ffs((int)m) - 1;
}

// warp lane of the first lane of this thread's group
template <int G>
__device__ __forceinline__ int lane_base_of()
{
    return (int)(threadIdx.x & 31u) & ~(G - 1);
}

template <int G>
__device__ __forceinline__ unsigned group_and(unsigned v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v &= __shfl_xor_sync(mask, v, off);
    return v;
}

// bits h with h = lane (mod G)
template <int G, typename Mask>
__device__ __forceinline__ Mask lane_bits(int lane)
{
    Mask m = 0;
#pragma unroll
    for (int h = 0; h < (int)(8 * sizeof(Mask)); h += G) m |= (Mask)1 << h;
    return m << lane;
}

// Lemma 1 (Eq. 2): mu(t) = ceil(t / T) + 1, with t < 2^30 and T < 2^30.
__device__ __forceinline__ uint32_t arrivals(uint32_t t, uint2 tm, uint32_t sh)
{
    const uint64_t x = (uint64_t)(t + tm.x) * tm.y;
    return (uint32_t)(x >> sh) + 1u;
}

template <int G, int MAXN>
__device__ void fast_system(const BatchDev &b, const AnalysisParams &p, int64_t item, FastSmem<MAXN> &s,
                            int lane, unsigned gmask, int64_t *__restrict__ R_out,
                            uint8_t *__restrict__ st_out, uint8_t *__restrict__ verdict,
                            int32_t *big_list, int32_t *big_count, int32_t *wide_list,
                            int32_t *wide_count)
{
    using Mask = typename MaskOf<MAXN>::type;
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int pruned = __shfl_sync(gmask, cand_pruned(p, sys, cand) ? 1 : 0, lane_base_of<G>());
        if (pruned) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    if (n > MAXN) { // a wider configuration takes it
        if (lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;

    // ---- per-chain aggregates (Sec. II-C) and division magics ---------------
    int fits = 1;
    unsigned rank_ok = 1;
    Mask users = 0, spins = 0, rbits = 0;
    for (int c = lane; c < n; c += G) {
        const int64_t g = c0 + c;
        const int64_t T = b.T[g], D = b.D[g];
        const int x = b.exec[g];
        const uint8_t sp = b.spin[g];
        s.spin[c] = sp;
        int32_t pc;
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[c];
            rank_ok &= (r >= 0 && r < n) ? 1u : 0u;
            rbits |= (r >= 0 && r < n) ? (Mask)1 << r : 0;
            pc = n - 1 - r;
        } else {
            pc = b.prio[g];
        }
        s.pe[c] = make_int2(pc, xprio ? xprio[x0 + x] : 0);
        s.xk[c] = make_int2(x, b.exec_core[x0 + x]);
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        uint64_t E = 0, Emax = 0, S = 0, M = 0, Amin = ~0ull;
        for (int64_t cb = cb0; cb < cb1; ++cb) {
            const uint64_t e = (uint64_t)b.E[cb];
            E += e;
            Emax = e > Emax ? e : Emax;
        }
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        for (int64_t q = q0; q < q1; ++q) {
            const uint64_t a = (uint64_t)b.A[q] + kappa2; // A* = A + 2 kappa
            S += a;
            M = a > M ? a : M;
            Amin = a < Amin ? a : Amin;
        }
        const uint64_t dl = (uint64_t)(q1 - q0);
        const bool fit_c = (uint64_t)T < kFit && (uint64_t)D < kFit && E < kFit && S < kFit && dl < kFit &&
                           (eps == 0 || dl <= (kFit - 1) / eps);
        fits &= fit_c ? 1 : 0;
        uint32_t l = 0, m = 0;
        if (fit_c) { // m = ceil(2^(31+l) / T), l = ceil(log2 T): exact for every dividend below 2^31
            const uint32_t Tu = (uint32_t)T;
            l = Tu > 1 ? 32u - (uint32_t)__clz(Tu - 1u) : 0u;
            m = (uint32_t)(((1ull << (31 + l)) + Tu - 1u) / Tu);
        }
        s.tm[c] = make_uint2((uint32_t)T - 1u, m);
        s.sh[c] = (uint8_t)(31 + l);
        s.S[c] = (uint32_t)S;
        s.E[c] = (uint32_t)E;
        s.Emax[c] = (uint32_t)Emax;
        s.M[c] = (uint32_t)M;
        s.Amin[c] = (uint32_t)(Amin < kFit ? Amin : 0);
        s.D[c] = (uint32_t)D;
        s.dlt[c] = (uint32_t)dl;
        s.seg0[c] = (uint32_t)(q0 - seg_base);
        users |= (Mask)(dl > 0 ? 1 : 0) << c;
        spins |= (Mask)(sp ? 1 : 0) << c;
    }
    fits = group_and<G>((unsigned)fits, gmask);
    users = group_or<G>(users, gmask);
    spins = group_or<G>(spins, gmask);
    const Mask all = n >= (int)(8 * sizeof(Mask)) ? ~(Mask)0 : (((Mask)1 << n) - 1);
    if (rank_row) { // a candidate must be a permutation of 0..n-1
        rank_ok = group_and<G>(rank_ok, gmask);
        rbits = group_or<G>(rbits, gmask);
        if (!rank_ok || rbits != all) {
            if (lane == 0) {
                atomicExch(p.err, PAAM_E_INVAL);
                if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = 0;
            }
            __syncwarp(gmask);
            return;
        }
    }
    if (!fits) { // outside the 32-bit bound: the int64 kernel takes it
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        __syncwarp(gmask);
        return;
    }
    __syncwarp(gmask);
    if (!xprio) { // criticality-as-priority: highest chain priority on the executor
        for (int c = lane; c < n; c += G) {
            const int xc = s.xk[c].x;
            int32_t best = INT32_MIN;
            for (int k = 0; k < n; ++k)
                if (s.xk[k].x == xc && s.pe[k].x > best) best = s.pe[k].x;
            s.pe[c].y = best;
        }
        __syncwarp(gmask);
    }

    // ---- interferer sets, buckets, analysis order ----------------------------
    const int n_users = popc(users);
    const Mask valid = n >= (int)(8 * sizeof(Mask)) ? ~(Mask)0 : (((Mask)1 << n) - 1);
    for (int c = lane; c < n; c += G) {
        const int2 pec = s.pe[c], xkc = s.xk[c];
        Mask higher = 0, same_x = 0, hpp = 0;
        int pos = 0;
        for (int h = 0; h < n; ++h) {
            const int2 peh = s.pe[h], xkh = s.xk[h];
            const Mask bit = (Mask)1 << h;
            const bool hi = peh.x > pec.x;
            const bool sx = xkh.x == xkc.x;
            higher |= hi ? bit : 0;
            same_x |= sx ? bit : 0;
            hpp |= (!sx && xkh.y == xkc.y && peh.y > pec.y) ? bit : 0; // hpp(c), Lemma 4
            pos += (peh.y > pec.y) || (peh.y == pec.y && hi); // executor priority, then chain priority
        }
        const Mask cbit = (Mask)1 << c;
        s.hp[c] = higher & same_x;                        // hp(c), Lemma 4
        s.hpp[c] = hpp;
        s.hps[c] = higher & users;                        // hps(c), Eq. 3
        s.lower_x[c] = same_x & ~higher & ~cbit & valid;  // lp(c)
        s.order[pos] = (uint8_t)c;
        // bucket = floor(rank * n_buckets / |U|), rank = number of higher-priority users (R2)
        s.bucket[c] = (users & cbit) ? (int32_t)((uint32_t)popc(higher & users) * (uint32_t)p.n_buckets /
                                                 (uint32_t)n_users)
                                     : -1;
    }
    __syncwarp(gmask);

    // ---- blocking terms and per-segment fixed points (Lemma 2) --------------
    for (int c = lane; c < n; c += G) {
        const Mask cbit = (Mask)1 << c;
        const Mask hps = s.hps[c];
        const Mask lower_users = users & ~hps & ~cbit;
        uint32_t B = 0, blk = 0;
        for (Mask mm = s.lower_x[c]; mm; mm &= mm - 1) { // Lemma 4: one LP callback on the executor
            const int l = lowest(mm);
            B = s.Emax[l] > B ? s.Emax[l] : B;
        }
        const int32_t bc = s.bucket[c];
        if (bc >= 0)
            for (Mask mm = lower_users; mm; mm &= mm - 1) { // one LP request of the same bucket (R2-R3)
                const int l = lowest(mm);
                if (s.bucket[l] == bc && s.M[l] > blk) blk = s.M[l];
            }
        s.blk[c] = blk;
        s.B[c] = B;
        const uint32_t Dc = s.D[c];
        const uint32_t dl = s.dlt[c];
        uint32_t Hseg = kInf32;
        bool capped = false;
        if (dl > 0) {
            // Eq. 4 can take at most own + sum_h mu_h(D) S_h for any window R <= D.  Every
            // segment's Lemma 2 fixed point is at least x + sum_h mu_h(x) S_h >= x + f sum_h S_h
            // with x = A* + blk and f = 2 when x >= 1 (1 otherwise).  If the per-segment sum
            // cannot fall below Eq. 4 at D, the minimum of the two bounds is Eq. 4 at every
            // R <= D and the per-segment sum is not needed (recorded as infinite).
            const uint64_t own = (uint64_t)s.S[c] + (uint64_t)dl * blk;
            uint64_t hch_d = 0, sum_s = 0;
            for (Mask mm = hps; mm; mm &= mm - 1) {
                const int k = lowest(mm);
                hch_d += (uint64_t)arrivals(Dc, s.tm[k], s.sh[k]) * s.S[k];
                sum_s += s.S[k];
            }
            const uint64_t f = ((uint64_t)s.Amin[c] + blk) >= 1 ? 2 : 1;
            if (f * dl * sum_s < hch_d) {
                uint64_t limit = own + hch_d; // the per-segment sum matters only below this
                if (limit > (uint64_t)Dc + 1) limit = (uint64_t)Dc + 1;
                uint64_t Hsum = 0;
                bool inf = false;
                for (uint32_t j = 0; j < dl && !inf; ++j) {
                    const uint64_t base = (uint64_t)b.A[seg_base + s.seg0[c] + j] + kappa2 + blk;
                    uint64_t h = base; // the recurrence starts with the first two terms
                    uint32_t ev = 0;
                    for (;;) {
                        if (h > Dc || Hsum + h >= limit) {
                            inf = true;
                            break;
                        }
                        if (ev++ == kIterCap) {
                            inf = capped = true;
                            break;
                        }
                        uint64_t nh = base;
                        for (Mask mm = hps; mm; mm &= mm - 1) {
                            const int k = lowest(mm);
                            nh += (uint64_t)arrivals((uint32_t)h, s.tm[k], s.sh[k]) * s.S[k];
                        }
                        if (nh == h) break; // strictly increasing until here, bounded by D
                        h = nh;
                    }
                    Hsum += h;
                }
                if (!inf) Hseg = (uint32_t)Hsum;
            }
        }
        s.Hseg[c] = Hseg;
        s.cap[c] = capped ? 1 : 0;
        s.Ehp[c] = s.E[c];
        s.Ehpp[c] = s.E[c] + (s.spin[c] ? 0u : (uint32_t)((uint64_t)dl * eps));
    }
    __syncwarp(gmask);

    // ---- Theorem 1 (Eq. 6), chain by chain ----------------------------------
    const Mask mine = lane_bits<G, Mask>(lane);
    Mask sched = 0, dep = 0;
    Mask capm = 0; // chains whose chain recurrence reached kIterCap evaluations
    for (int k = 0; k < n; ++k) {
        const int c = s.order[k];
        const Mask hp = s.hp[c], hpp = s.hpp[c], hps = s.hps[c];
        const Mask cbit = (Mask)1 << c;
        if ((hp | (hpp & spins)) & ~sched) { // a needed H*_h is not available
            dep |= cbit;
            if (rank_row) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        if (s.cap[c]) { // a segment recurrence was cut short: no bound (PAAM_ST_ITERCAP)
            if (rank_row) break;
            continue;
        }
        const uint64_t Dc = s.D[c];
        const uint64_t base = (uint64_t)s.B[c] + s.E[c];
        const uint64_t dl = s.dlt[c];
        const uint64_t own = (uint64_t)s.S[c] + dl * s.blk[c];
        const uint64_t deps = dl * eps;
        const uint64_t Hseg = s.Hseg[c] == kInf32 ? ~0ull : (uint64_t)s.Hseg[c];
        const Mask todo = (hp | hpp | hps) & mine;
        // start: B + E + H* with the interference part of Eq. 4 empty
        uint64_t R = base + (dl ? (Hseg < own ? Hseg : own) + deps : 0);
        uint64_t hs = 0;
        bool ok = false;
        uint32_t ev = 0;
        while (R <= Dc) {
            if (ev++ == kIterCap) {
                capm |= cbit;
                break;
            }
            uint64_t cpu = 0, acc = 0;
            const uint32_t t = (uint32_t)R;
            for (Mask mm = todo; mm; mm &= mm - 1) {
                const int h = lowest(mm);
                const Mask bit = (Mask)1 << h;
                const uint64_t mu = arrivals(t, s.tm[h], s.sh[h]);
                const uint32_t ccpu = (hp & bit) ? s.Ehp[h] : ((hpp & bit) ? s.Ehpp[h] : 0u);
                const uint32_t cacc = (hps & bit) ? s.S[h] : 0u;
                cpu += mu * ccpu;
                acc += mu * cacc;
            }
            cpu = group_sum<G>(cpu, gmask);
            acc = group_sum<G>(acc, gmask);
            hs = 0;
            if (dl) {
                const uint64_t hch = own + acc; // Eq. 4
                hs = (Hseg < hch ? Hseg : hch) + deps; // Eq. 1 with min(Eq. 3, Eq. 4)
            }
            const uint64_t Rn = base + hs + cpu;
            if (Rn == R) {
                ok = true;
                break;
            }
            R = Rn; // strictly increasing until convergence, bounded by D
        }
        if (ok) {
            sched |= cbit;
            if (lane == 0) {
                s.R[c] = (uint32_t)R;
                s.Ehp[c] = s.E[c] + (uint32_t)hs;
                if (s.spin[c]) s.Ehpp[c] = s.E[c] + (uint32_t)hs;
            }
        }
        __syncwarp(gmask);
        if (!ok && rank_row) break;
    }

    // ---- outputs --------------------------------------------------------------
    if (rank_row) {
        if (lane == 0) {
            const bool ok = sched == all;
            if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = ok ? 1 : 0;
            if (ok) atomicMin(p.first_ok + sys, cand);
        }
        __syncwarp(gmask);
        return;
    }
    for (int c = lane; c < n; c += G) {
        const Mask bit = (Mask)1 << c;
        const bool ok = sched & bit;
        R_out[c0 + c] = ok ? (int64_t)s.R[c] : -1;
        st_out[c0 + c] = ok ? PAAM_ST_SCHED
                            : (((capm & bit) || s.cap[c]) ? PAAM_ST_ITERCAP : ((dep & bit) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
    }
    if (lane == 0 && verdict) verdict[sys] = sched == all ? 1 : 0;
    __syncwarp(gmask);
}

// Systems are all of the batch (list == nullptr) or list[0 .. *count).
template <int G, int MAXN>
__global__ void __launch_bounds__(256) analyze_fast_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                           uint8_t *st, uint8_t *verdict,
                                                           const int32_t *list, const int32_t *count,
                                                           int32_t *big_list, int32_t *big_count,
                                                           int32_t *wide_list, int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    FastSmem<MAXN> &s = reinterpret_cast<FastSmem<MAXN> *>(smem_raw)[grp];
    const unsigned gmask = group_mask<G>();
    const int64_t n_items = list ? (int64_t)*count : (p.K > 0 ? b.n_sys * p.K : b.n_sys);
    for_each_item<G>(p, n_items, grp, groups, lane, gmask, [&](int64_t i) {
        const int64_t item = list ? (int64_t)list[i] : i;
        fast_system<G, MAXN>(b, p, item, s, lane, gmask, R, st, verdict, big_list, big_count, wide_list,
                             wide_count);
    });
}

template <int G, int MAXN>
int launch_fast(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                const int32_t *list, const int32_t *count, int64_t max_items, int threads,
                cudaStream_t stream)
{
    if (threads % G != 0 || threads > 256) return PAAM_E_INVAL;
    int groups = threads / G;
    // fit the CTA's tables into the opt-in shared memory, keeping whole warps
    const int fit = bt->ctx->max_smem_optin / (int)sizeof(FastSmem<MAXN>);
    if (groups > fit) {
        const int per_warp = G >= 32 ? 1 : 32 / G;
        groups = fit / per_warp * per_warp;
        if (groups < 1) return PAAM_E_UNSUPPORTED;
        threads = groups * G;
    }
    const size_t smem = sizeof(FastSmem<MAXN>) * groups;
    auto kern = analyze_fast_kernel<G, MAXN>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, list, count,
                                                      bt->list_big, bt->counts, bt->list_wide,
                                                      bt->counts + 1);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

bool batch_fits_32(const paam_batch *b, const AnalysisParams &p)
{
    const unsigned long long F = kFit;
    const unsigned long long dmax = b->stats[ST_DELTAMAX];
    const unsigned long long k2 = 2ull * (unsigned long long)p.kappa;
    if (b->stats[ST_TMAX] >= F || b->stats[ST_DMAX] >= F || b->stats[ST_ECMAX] >= F || dmax >= F) return false;
    if (k2 > 0 && dmax > (F - 1) / k2) return false;
    if (b->stats[ST_SCMAX] + dmax * k2 >= F) return false;
    if (p.eps > 0 && dmax > (F - 1) / (unsigned long long)p.eps) return false;
    return true;
}

using LaunchFn = int (*)(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                         const int32_t *, const int32_t *, int64_t, int, cudaStream_t);

struct Variant {
    int impl, G, maxn;
    LaunchFn fn;
};

// Every (family, group width, table size) the library instantiates.
const Variant kVariants[] = {
    {0, 1, 16, launch_fast<1, 16>},   {0, 2, 16, launch_fast<2, 16>},   {0, 4, 16, launch_fast<4, 16>},
    {0, 8, 16, launch_fast<8, 16>},   {0, 2, 32, launch_fast<2, 32>},   {0, 4, 32, launch_fast<4, 32>},
    {0, 8, 32, launch_fast<8, 32>},   {0, 16, 32, launch_fast<16, 32>}, {0, 4, 64, launch_fast<4, 64>},
    {0, 8, 64, launch_fast<8, 64>},   {0, 16, 64, launch_fast<16, 64>}, {0, 32, 64, launch_fast<32, 64>},
    {1, 4, 16, launch_reg<4, 4>},     {1, 8, 16, launch_reg<8, 2>},     {1, 16, 16, launch_reg<16, 1>},
    {1, 16, 32, launch_reg<16, 2>},   {1, 32, 32, launch_reg<32, 1>},   {1, 32, 64, launch_reg<32, 2>},
    {2, 16, 16, launch_lazy<4>}, {3, 16, 16, launch_lazy<5>}, {4, 16, 16, launch_lazy<6>},
};

LaunchFn find_variant(int impl, int G, int maxn)
{
    for (const Variant &v : kVariants)
        if (v.impl == impl && v.G == G && v.maxn == maxn) return v.fn;
    return nullptr;
}

} // namespace

// Candidate launch configurations the autotuner times (kDefaultLaunchCfg is
// the one a batch starts with).
const LaunchCfg kLaunchCfgs[] = {
    {1, 8, 16, 0, 16, 256, 0},  {0, 8, 16, 0, 16, 256, 0},  {0, 16, 32, 0, 16, 256, 0}, {1, 16, 16, 0, 16, 256, 0},
    {1, 4, 16, 0, 16, 256, 0},  {1, 16, 32, 1, 32, 256, 0}, {1, 32, 32, 1, 32, 256, 0}, {1, 8, 16, 1, 32, 256, 0},
    {0, 4, 16, 0, 16, 256, 0},  {0, 8, 32, 0, 32, 256, 0},  {1, 16, 32, 0, 16, 256, 0}, {1, 4, 16, 1, 32, 128, 0},
    // the same shapes pulling from the work queue, 2 items per fetch
    {1, 16, 16, 0, 16, 256, 2}, {1, 8, 16, 0, 16, 256, 2},  {0, 8, 16, 0, 16, 256, 2},  {1, 16, 32, 1, 32, 256, 2},
    {1, 32, 32, 1, 32, 256, 2},
    // the queue shapes again, handing systems out by increasing chain count
    {1, 16, 16, 0, 16, 256, 2, 1}, {1, 32, 32, 1, 32, 256, 2, 1}, {1, 8, 16, 0, 16, 256, 2, 1},
    // register tables with lazy per-chain work (analyze_lazy.cu): static shares, queue, queue by size
    {2, 16, 16, 1, 32, 256, 0, 0}, {2, 16, 16, 1, 32, 256, 2, 0}, {2, 16, 16, 1, 32, 256, 2, 1},
    // the same with 5 and 6 resident blocks per SM (fewer registers per thread)
    {3, 16, 16, 1, 32, 256, 2, 1}, {4, 16, 16, 1, 32, 256, 2, 1}, {3, 16, 16, 1, 32, 256, 2, 0},
    // the same first passes with the 32-lane lazy kernel over the deferral list
    {4, 16, 16, kImplBigLazy32, 32, 256, 2, 1}, {2, 16, 16, kImplBigLazy32, 32, 256, 2, 1},
    {3, 16, 16, kImplBigLazy32, 32, 256, 2, 1},
};
const int kNumLaunchCfgs = (int)(sizeof(kLaunchCfgs) / sizeof(kLaunchCfgs[0]));
static_assert(kDefaultLaunchCfg < (int)(sizeof(kLaunchCfgs) / sizeof(kLaunchCfgs[0])), "default configuration");

int paam_enqueue_analysis(const paam_batch *b, const AnalysisParams &p, const LaunchCfg &cfg, int64_t *R,
                          uint8_t *status, uint8_t *verdict, cudaStream_t stream, int *n_kernels)
{
    LaunchFn small = find_variant(cfg.impl_small, cfg.g_small, cfg.maxn_small);
    LaunchFn bigfn = cfg.impl_big == kImplBigLazy32 ? launch_reg<32, 2> : find_variant(cfg.impl_big, cfg.g_big, 64);
    if (!small || !bigfn) return PAAM_E_INVAL;
    int k = 0;
    const int64_t items = p.K > 0 ? b->n_sys * (int64_t)p.K : b->n_sys;
    // the safe blocking term with several accelerators: the int64 kernel for every system
    if (p.blocking_mode == 1 && b->acc) {
        AnalysisParams pw = p; // the configuration's work distribution and order apply here too
        pw.queue_batch = 0;
        pw.sys_order = cfg.binned ? b->sys_order : nullptr;
        if (cfg.queue > 0 && b->queue) {
            PAAM_CUDA_TRY(cudaMemsetAsync(b->queue, 0, sizeof(unsigned long long), stream));
            pw.queue = b->queue;
            pw.queue_batch = cfg.queue;
        }
        const int rc = paam_launch_wide(b, pw, R, status, verdict, nullptr, nullptr, items, stream);
        if (n_kernels) *n_kernels = 1;
        return rc;
    }
    PAAM_CUDA_TRY(cudaMemsetAsync(b->counts, 0, 2 * sizeof(int32_t), stream));
    // per pass: its own work-queue counter, or static shares
    AnalysisParams pm = p, pb = p, pw = p;
    pm.queue_batch = pb.queue_batch = pw.queue_batch = 0;
    pm.sys_order = pb.sys_order = pw.sys_order = cfg.binned ? b->sys_order : nullptr;
    if (cfg.queue > 0 && b->queue) {
        PAAM_CUDA_TRY(cudaMemsetAsync(b->queue, 0, 3 * sizeof(unsigned long long), stream));
        pm.queue = b->queue;
        pb.queue = b->queue + 1;
        pw.queue = b->queue + 2;
        pm.queue_batch = pb.queue_batch = pw.queue_batch = cfg.queue;
    }
    if (p.blocking_mode == 1) { // the safe blocking term in the lazy kernel, the int64 kernel for the rest
        int rc = paam_launch_lazy_safe(b, pm, R, status, verdict, items, stream);
        if (rc == PAAM_OK) rc = paam_launch_wide(b, pw, R, status, verdict, b->list_wide, b->counts + 1, items, stream);
        if (n_kernels) *n_kernels = 2;
        return rc;
    }
    if (b->acc) { // several accelerators: per-accelerator register tables, the int64 kernel for the rest
        int rc = paam_launch_lazy_acc(b, pm, R, status, verdict, items, stream);
        if (rc == PAAM_OK) rc = paam_launch_wide(b, pw, R, status, verdict, b->list_wide, b->counts + 1, items, stream);
        if (n_kernels) *n_kernels = 2;
        return rc;
    }
    int rc = small(b, pm, R, status, verdict, nullptr, nullptr, items, cfg.threads, stream);
    if (rc != PAAM_OK) return rc;
    ++k;
    // the lazy kernel also defers systems inside the 32-bit bound that are not narrow
    const bool lazy_defers = cfg.impl_small >= 2 && b->stats[ST_DMAX] >= kLazyNarrowD;
    const bool lazy_passes = (b->max_chains > cfg.maxn_small || lazy_defers) && cfg.impl_big == kImplBigLazy32;
    if (lazy_passes) {
        // 17..32 chains in the 32-lane lazy kernel, then the rest of the list (over 32
        // chains) in the 64-chain lazy kernel, one system per fetch from the work queue
        // (the first pass's counter, reset: that pass is done)
        rc = launch_lazy32<6>(b, pb, R, status, verdict, b->list_big, b->counts, items, cfg.threads, stream);
        if (rc != PAAM_OK) return rc;
        ++k;
        if (b->max_chains > 32) {
            AnalysisParams ph = pb;
            ph.queue_batch = 0;
            if (cfg.queue > 0 && b->queue) {
                PAAM_CUDA_TRY(cudaMemsetAsync(b->queue, 0, sizeof(unsigned long long), stream));
                ph.queue = b->queue;
                ph.queue_batch = 1;
            }
            ph.min_chains = 33;
            rc = launch_lazy64(b, ph, R, status, verdict, b->list_big, b->counts, items, cfg.threads, stream);
            if (rc != PAAM_OK) return rc;
            ++k;
        }
    } else if (b->max_chains > cfg.maxn_small || lazy_defers) {
        rc = bigfn(b, pb, R, status, verdict, b->list_big, b->counts, items, cfg.threads, stream);
        if (rc != PAAM_OK) return rc;
        ++k;
    }
    // the int64 kernel for the systems outside the 32-bit bound, and (the 32-lane lazy
    // pass sends them there) for the deferred systems inside it that are not narrow
    if (!batch_fits_32(b, p) || (lazy_passes && b->stats[ST_DMAX] >= kLazyDeferWideD)) {
        rc = paam_launch_wide(b, pw, R, status, verdict, b->list_wide, b->counts + 1, items, stream);
        if (rc != PAAM_OK) return rc;
        ++k;
    }
    if (n_kernels) *n_kernels = k;
    return PAAM_OK;
}
