// analyze_lazy.cu -- the register-table analysis with lazy per-chain work.
//
// Same mathematics as analyze_reg.cu (Theorem 1, Eq. 6, with Eqs. 1-5): one
// system per group of 16 lanes, one chain per lane, Lemma 1's arrival counts
// by exact multiply-shift division, and the 32-bit narrow sums (every
// deadline below 2^27 - 16; a capped partial sum already exceeds every
// deadline, so it decides each comparison with D as the true sum would).  It
// differs in where the work goes:
//
//  - Relations cost one pass of a few instructions per chain pair: the
//    same-executor and same-core sets come from __match_any_sync, lower- and
//    higher-priority sets from one comparison each, and CPU blocking (Lemma 4)
//    from the few lower-priority chains of the executor.
//  - The test that decides whether Lemma 2's per-segment sum can beat Eq. 4
//    below the deadline, and the exact per-segment fixed points it calls for,
//    run when the chain's own recurrence is reached, with the lanes over the
//    chain's higher-priority accelerator users.  A chain that turns out
//    dependent on an unschedulable chain (the DEP rule) never pays for them;
//    only its own recurrence reads a per-segment sum, so results are those of
//    the eager order.
//
// Systems with more than 16 chains, or that fit the 32-bit bound but not the
// narrow one, go to b.list_big (the 32-lane pass of this kernel over that list,
// then analyze_lazy64.cu for those above 32 chains); systems outside the 32-bit
// bound to b.list_wide (the int64 kernel).  One accelerator: Lemma 4 as printed
// (blocking_mode 0) in analysis, candidate and target mode, and the safe reading
// (blocking_mode 1, 16 lanes; its larger systems go to the int64 kernel); several
// accelerators keep their kernel (analyze_lazy_acc.cu).
#include "reg_common.cuh"

namespace {
using namespace paam_reg;

// LG lanes per system = its largest chain count: 16 (the first pass over every
// system) or 32 (a pass over the first pass's deferral list, for systems of 17
// to 32 chains; larger ones are left on the list for the 64-chain kernel, and
// systems that are not narrow go to the int64 kernel)

// per chain, stored at the chain's position in the analysis order
constexpr int kPrefetchSlice = 256; // systems per L2 prefetch (a divisor of kBinWindow)

template <int LG>
struct LazySmem {
    uint4 rel[LG];    // {hp, hpp, hps, needs = hp and the spinning hpp: all must be schedulable (DEP rule)}
    uint4 rec[LG];    // {D, base = B + E, own = S* + delta blk (capped at D + 1), deps = delta eps}
    uint4 seg[LG];    // {chain index, lb (Lemma 2's lower bound, below), blk, delta}
    uint32_t emax[LG]; // longest callback, for Lemma 4's blocking
    uint32_t m[LG];    // M*, for the same-bucket blocking with several buckets
    uint32_t msort[LG]; // M* of the users (0 for the others) by chain-priority rank, one bucket
    uint32_t ssort[LG]; // S* of the users (0 for the others, capped at 2^27 - 1) by chain-priority rank
    uint32_t inv[LG];   // by priority value (values below LG): the chain of that priority
    uint32_t exm[LG];   // by executor priority value: the chains of that executor priority
    uint32_t seg0[LG];  // by analysis position: first segment, relative to the system's first
    uint32_t needs[LG]; // by chain: its DEP-rule set, read again for the status
    int32_t bucket[LG];
    int64_t c0, sys, seg_base; // kept here across the chain steps, not in registers
    int32_t cand;
};

// The safe reading of Lemma 4 (blocking_mode 1) also bounds every segment of the
// system, one per lane, from these tables (systems of up to kSafeSegs segments).
constexpr int kSafeSegs = 128;
template <int LG>
struct LazySafeExt {
    uint4 dv[LG];             // by chain: {2 (T - 1), magic, l, S*} (the interferer's term)
    uint4 ch[LG];             // by chain: {hps, D, blk, 0}
    uint32_t hq[kSafeSegs];   // by segment (relative to the system's first): its bound; kInfR none, kCapR cut short
    uint8_t segc[kSafeSegs];  // by segment: its chain
};
template <int LG>
struct LazySafeSmem : LazySmem<LG> {
    LazySafeExt<LG> x;
};

// a term of a segment's recurrence, capped: any term above every deadline (all
// below 2^27 here) decides the comparison with D as the exact one does
constexpr uint64_t kSafeTermCap = 1ull << 40;
// a hold without a bound, and any hold at or above it: every deadline is below it
constexpr uint32_t kHoldInf = (uint32_t)kFitR;

// ceil(t / T) + 1 (Lemma 1) times c, capped at 2^27 - 1 so that 16 lanes' sum fits 32 bits
__device__ __forceinline__ uint32_t capped_term(uint32_t t, uint32_t tm2, uint32_t mg, uint32_t lg, uint32_t c)
{
    const uint64_t v = (uint64_t)rarrivals(t, tm2, mg, lg) * c;
    return v < kNarrow - 1 ? (uint32_t)v : kNarrow - 1;
}

// The aggregates of chain g (Sec. II-C), which do not depend on the priorities:
// sums and extremes in 32 bits over values capped at 2^30 (a capped value takes
// the chain's sum to the 32-bit bound, and its system to the int64 kernel).
struct ChainAgg {
    uint32_t tm2, mg, lg, D, E, S, Emax, M, Amin, dl;
    int64_t q0;
    unsigned fit;
};

__device__ __forceinline__ void chain_aggregates(const BatchDev &b, int64_t g, uint64_t kappa2, uint64_t eps,
                                                 ChainAgg &a)
{
    const int64_t T = b.T[g], D = b.D[g];
    const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
    const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
    const int64_t *Ep = b.E + cb0;
    const int ncb = (int)(cb1 - cb0);
    uint32_t E = 0, Emax = 0, S = 0, M = 0, Amin = 0xFFFFFFFFu;
#pragma unroll 4
    for (int i = 0; i < ncb; ++i) {
        const uint32_t e = (uint64_t)Ep[i] < kFitR ? (uint32_t)Ep[i] : (uint32_t)kFitR;
        E = umin(E + e, (uint32_t)kFitR);
        Emax = umax(Emax, e);
    }
    const int64_t *Ap = b.A + q0;
    const int nq = (int)(q1 - q0);
    const uint32_t k2c = kappa2 < kFitR ? (uint32_t)kappa2 : (uint32_t)kFitR;
#pragma unroll 4
    for (int i = 0; i < nq; ++i) {
        const uint32_t v = ((uint64_t)Ap[i] < kFitR ? (uint32_t)Ap[i] : (uint32_t)kFitR) + k2c; // A* = A + 2 kappa
        S = umin(S + v, (uint32_t)kFitR);
        M = umax(M, v);
        Amin = umin(Amin, v);
    }
    const uint64_t dl = (uint64_t)nq;
    a.fit = ((uint64_t)T < kFitR && (uint64_t)D < kFitR && E < kFitR && S < kFitR && dl < kFitR &&
             (eps == 0 || dl <= (kFitR - 1) / eps))
                ? 1u
                : 0u;
    a.tm2 = a.mg = a.lg = 0;
    if (a.fit) rdivisor((uint32_t)T, a.tm2, a.mg, a.lg);
    a.D = (uint32_t)D;
    a.E = E;
    a.S = S;
    a.Emax = Emax;
    a.M = M;
    a.Amin = dl ? (Amin < kFitR ? Amin : 0u) : 0u;
    a.dl = (uint32_t)dl;
    a.q0 = q0;
}

// REC: the aggregates come from p.chain_recs (candidate mode).  TGT (target mode,
// the Audsley-style seed; see AnalysisParams.target): candidate (system, c) is
// decided by chain p.target[system * Kc + c] alone (-1: no trial in the slot), the
// chains are analysed up to that one's step and no failure ends a candidate early.
// SAFE (16 lanes, aggregates computed here): the safe reading of Lemma 4
// (blocking_mode 1): every segment's Lemma 2 bound is computed (one segment per
// lane), each chain's longest callback hold E_i + sum over its segments of (bound
// + eps), B_c as the longest hold of a lower-priority chain on c's executor, and
// Eq. 3's exact sum in every recurrence; systems of more than kSafeSegs segments
// go to the int64 kernel's list.
template <int LG, bool REC = false, bool TGT = false, bool SAFE = false>
__device__ void lazy_system(const BatchDev &b, const AnalysisParams &p, int64_t item, LazySmem<LG> &s,
                            LazySafeExt<LG> *sx, int lane,
                            unsigned gm, int64_t *__restrict__ R_out, uint8_t *__restrict__ st_out,
                            uint8_t *__restrict__ verdict, int32_t *big_list, int32_t *big_count,
                            int32_t *wide_list, int32_t *wide_count)
{
    using Mask = uint32_t;
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int pruned = __shfl_sync(gm, cand_pruned(p, sys, cand) ? 1 : 0, 0, LG);
        if (pruned) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    int tgt = -1;
    if constexpr (TGT) {
        tgt = p.target[sys * p.Kc + cand_of(p, sys, cand)];
        if (tgt < 0 || tgt >= n) return; // no trial in this slot
    }
    if (n > LG) { // the 64-chain kernel's; the first pass appends it to its list
        if (LG == 16 && lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;
    const int j = lane;
    const Mask jbit = 1u << j;

    // ---- per-chain aggregates (Sec. II-C) -----------------------------------
    uint32_t tm2 = 0, mg = 0, lg = 0, Dv = 0, Ev = 0, Sv = 0, Emx = 0, Mv = 0, Amn = 0, dlv = 0, seg0 = 0;
    int32_t pr = INT32_MIN, ep = INT32_MIN, ex = -1 - j, co = -1 - j;
    bool sp = false;
    unsigned fit = 1, rank_ok = 1;
    Mask rbit = 0;
    uint32_t rsx = 0, rco = 0; // same-executor and same-core chains, from the records
    const bool val = j < n;
    if (val) {
        const int64_t g = c0 + j;
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[j];
            rank_ok = (r >= 0 && r < n) ? 1u : 0u;
            rbit = rank_ok ? 1u << r : 0u;
            pr = n - 1 - r;
        } else {
            pr = b.prio[g];
        }
        if constexpr (REC) {
            const uint4 *r = p.chain_recs + g * 4;
            const uint4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3];
            tm2 = r0.x, mg = r0.y, lg = r0.z, Dv = r0.w;
            Ev = r1.x, Sv = r1.y, Emx = r1.z, Mv = r1.w;
            Amn = r2.x, dlv = r2.y, seg0 = r2.z, fit = r2.w & 1u, sp = (r2.w >> 1) & 1u;
            ex = (int32_t)r3.x, co = (int32_t)r3.y;
            rsx = r3.z, rco = r3.w;
            if (xprio) ep = xprio[x0 + ex];
        } else {
            ex = b.exec[g];
            co = b.exec_core[x0 + ex];
            if (xprio) ep = xprio[x0 + ex];
            sp = b.spin[g] != 0;
            ChainAgg a;
            chain_aggregates(b, g, kappa2, eps, a);
            fit = a.fit;
            tm2 = a.tm2, mg = a.mg, lg = a.lg;
            Dv = a.D;
            Ev = a.E;
            Sv = a.S;
            Emx = a.Emax;
            Mv = a.M;
            Amn = a.Amin;
            dlv = a.dl;
            seg0 = (uint32_t)(a.q0 - seg_base);
        }
    }
    if (lane == 0) {
        s.c0 = c0;
        s.sys = sys;
        s.seg_base = seg_base;
        s.cand = cand;
    }
    const unsigned sh = LG == 32 ? 0u : (threadIdx.x & 16u); // the group's first lane in the warp
    const Mask users = __ballot_sync(gm, val && dlv != 0) >> sh;
    const Mask spins = __ballot_sync(gm, sp) >> sh;
    const Mask all = (n >= 32) ? ~0u : ((1u << n) - 1u);
    if (rank_row) { // a candidate must be a permutation of 0..n-1
        rank_ok = __reduce_and_sync(gm, rank_ok);
        rbit = __reduce_or_sync(gm, rbit);
        if (!rank_ok || rbit != all) {
            if (lane == 0) {
                atomicExch(p.err, PAAM_E_INVAL);
                if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = 0;
            }
            return;
        }
    }
    if (!__reduce_and_sync(gm, fit)) { // outside the 32-bit bound
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    const uint32_t dmax = __reduce_max_sync(gm, Dv);
    if (dmax >= kNarrow - LG) { // inside it but not narrow: the 64-chain kernel (first pass) or the int64 kernel
        if (lane == 0) {
            if (LG == 16) big_list[atomicAdd(big_count, 1)] = (int32_t)item;
            else wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        }
        return;
    }
    uint32_t nseg = 0; // the system's segments (safe reading)
    if constexpr (SAFE) {
        nseg = __reduce_add_sync(gm, val ? dlv : 0u);
        if (nseg > (uint32_t)kSafeSegs) {
            if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
            return;
        }
    }
    // The system's iteration bound: a recurrence of Eq. 3 or Eq. 6 rises strictly until
    // it converges or passes its deadline, and after its first step only when some
    // arrival count ceil(t / T_h) + 1 (Lemma 1) has grown, at most ceil(Dmax / T_h) times
    // per chain h while t <= Dmax; so none takes more than L = sum_h ceil(Dmax / T_h) + 2
    // evaluations.  With L within kIterCap (always, for a validated batch) the loops run
    // without counters; otherwise every loop stops at kIterCap (PAAM_ST_ITERCAP).
    const uint32_t L = __reduce_add_sync(gm, val ? umin(rarrivals(dmax, tm2, mg, lg) - 1u, kIterCap + 1u) : 0u) + 2u;
    const bool counted = L > kIterCap;

    // ---- relations (Lemma 4, Theorem 1, Eq. 3), analysis order ---------------
    // lanes of the same executor (unique keys past n) and of the same core: from the
    // chain records (every lane of the group takes the same path), or matched here
    unsigned xm;
    Mask corem;
    if constexpr (REC) {
        xm = (val ? rsx : jbit) << sh;
        corem = val ? rco : jbit;
    } else {
        xm = __match_any_sync(gm, ex);
        corem = __match_any_sync(gm, co) >> sh;
    }
    const Mask samex = xm >> sh;
    if (!xprio) ep = __reduce_max_sync(xm, pr); // criticality-as-priority: highest chain priority on the executor
    const bool one_bucket = p.n_buckets == 1;
    const Mask eqx = __match_any_sync(gm, ep) >> sh; // equal executor priority
    // higher chain priority and higher executor priority
    Mask higher = 0, ehigher = 0;
    if (__reduce_and_sync(gm, (!val || ((uint32_t)pr < (uint32_t)LG && (uint32_t)ep < (uint32_t)LG)) ? 1u : 0u)) {
        // priorities below LG (a permutation of 0..n-1, and executor priorities taken
        // from them): the chains of each priority value go to slot value, and the set
        // above a value is the OR of the slots past it, a suffix scan over the group
        s.inv[j] = 0u;
        s.exm[j] = 0u;
        __syncwarp(gm);
        if (val) {
            s.inv[pr] = jbit; // distinct priorities: one chain per slot
            s.exm[ep] = eqx;  // every chain of this executor priority writes the same mask
        }
        __syncwarp(gm);
        uint32_t a = s.inv[j], e = s.exm[j];
#pragma unroll
        for (int d = 1; d < LG; d <<= 1) {
            const uint32_t aw = __shfl_down_sync(gm, a, d, LG), ew = __shfl_down_sync(gm, e, d, LG);
            if (j + d < LG) {
                a |= aw;
                e |= ew;
            }
        }
        a = __shfl_down_sync(gm, a, 1, LG); // slots past this one
        e = __shfl_down_sync(gm, e, 1, LG);
        if (j + 1 >= LG) a = e = 0u;
        higher = __shfl_sync(gm, a, val ? pr : 0, LG);
        ehigher = __shfl_sync(gm, e, val ? ep : 0, LG);
        if (!val) higher = ehigher = all;
    } else { // one comparison each per chain
#pragma unroll
        for (int t = 0; t < LG; ++t) {
            const int32_t pt = __shfl_sync(gm, pr, t, LG), et = __shfl_sync(gm, ep, t, LG);
            higher |= (t < n && pt > pr) ? 1u << t : 0u;
            ehigher |= (t < n && et > ep) ? 1u << t : 0u;
        }
    }
    // position in the analysis order: executor priority, then chain priority
    const int pos = __popc(ehigher) + __popc(eqx & higher & all);
    const Mask hp = samex & higher;                 // hp(c), Lemma 4
    const Mask hpp = corem & ~samex & ehigher;      // hpp(c), Theorem 1
    const Mask hps = users & higher;                // hps(c), Eq. 3
    const bool user = (users >> j) & 1;
    s.emax[j] = Emx;
    if (!one_bucket) s.m[j] = Mv;
    const int prank = __popc(higher); // rank by chain priority, 0 = highest
    if (val) {
        s.ssort[prank] = user ? umin(Sv, kNarrow - 1) : 0u;
        if (one_bucket) s.msort[prank] = user ? Mv : 0u;
    }
    uint32_t Bv = 0, blk = 0;
    __syncwarp(gm);
    // sum_h S*_h over hps(c), the users of higher priority: a prefix sum in priority
    // order, saturating at 2^27 (a larger sum only ever meets bounds below it)
    uint32_t sums = j < n ? s.ssort[j] : 0u;
#pragma unroll
    for (int d = 1; d < LG; d <<= 1) {
        const uint32_t w = __shfl_up_sync(gm, sums, d, LG);
        if (j >= d) sums = umin(sums + w, kNarrow);
    }
    sums = __shfl_up_sync(gm, sums, 1, LG);
    if (j == 0) sums = 0u;
    sums = __shfl_sync(gm, sums, prank < LG ? prank : 0, LG);
    if constexpr (!SAFE)
        for (Mask lo = samex & ~higher & ~jbit & all; lo; lo &= lo - 1) // Lemma 4: one LP callback on the executor
            Bv = umax(Bv, s.emax[__ffs(lo) - 1]);
    if (one_bucket) { // every user shares the bucket: the longest lower-priority request (R2-R3)
        // the largest M* over the users of rank > r: a suffix maximum in priority order
        uint32_t v = j < n ? s.msort[j] : 0u;
#pragma unroll
        for (int d = 1; d < LG; d <<= 1) {
            const uint32_t w = __shfl_down_sync(gm, v, d, LG);
            if (j + d < LG) v = umax(v, w);
        }
        uint32_t below = __shfl_down_sync(gm, v, 1, LG);
        if (j + 1 >= LG) below = 0u;
        below = __shfl_sync(gm, below, prank < LG ? prank : 0, LG);
        if (user) blk = below;
    }
    if (!one_bucket) { // bucket = floor(rank * n_buckets / |U|), rank among the users (R2)
        const int32_t bk = user ? (int32_t)((uint32_t)__popc(hps) * (uint32_t)p.n_buckets / (uint32_t)__popc(users))
                                : -1;
        s.bucket[j] = bk;
        __syncwarp(gm);
        if (user)
            for (Mask lo = users & ~higher & ~jbit; lo; lo &= lo - 1) {
                const int l = __ffs(lo) - 1;
                if (s.bucket[l] == bk) blk = umax(blk, s.m[l]);
            }
    }

    uint32_t hsum = 0; // safe reading: Eq. 3's exact sum over the chain's segments (kInfR none, kCapR cut short)
    if constexpr (SAFE) {
        // every segment's fixed point h = A* + blk + sum over hps(c) of (ceil(h / T_t)
        // + 1) S*_t (Lemma 2), one segment per lane, each lane summing the terms of
        // its chain's higher-priority users itself
        if (val) {
            sx->dv[j] = make_uint4(tm2, mg, lg, Sv);
            sx->ch[j] = make_uint4(hps, Dv, blk, 0u);
            for (uint32_t i = 0; i < dlv; ++i) sx->segc[seg0 + i] = (uint8_t)j;
        }
        __syncwarp(gm);
        for (uint32_t k = j; k < nseg; k += LG) {
            const int c = sx->segc[k];
            const uint4 ch = sx->ch[c];
            const uint64_t base = (uint64_t)b.A[seg_base + k] + kappa2 + ch.z;
            uint64_t h = base; // the recurrence starts with the first two terms
            uint32_t out, evs = 0;
            for (;;) {
                if (h > ch.y) {
                    out = kInfR;
                    break;
                }
                if (counted && evs++ == kIterCap) {
                    out = kCapR;
                    break;
                }
                uint64_t sum = 0;
                for (Mask m = ch.x; m; m &= m - 1) {
                    const uint4 dv = sx->dv[__ffs(m) - 1];
                    const uint64_t term = (uint64_t)rarrivals((uint32_t)h, dv.x, dv.y, dv.z) * dv.w;
                    sum += term < kSafeTermCap ? term : kSafeTermCap;
                }
                const uint64_t nh = base + sum;
                if (nh == h) { // strictly increasing until here, bounded by D
                    out = (uint32_t)h;
                    break;
                }
                h = nh;
            }
            sx->hq[k] = out;
        }
        __syncwarp(gm);
        // this lane's chain: its callbacks' holds E_i + sum over the callback's segments
        // of (bound + eps), and Eq. 3's sum over all its segments; a chain without
        // segments holds its executor for its longest callback
        uint32_t hold = Emx;
        if (val && dlv) {
            const int64_t g = c0 + j;
            const int64_t cb1 = b.chain_cb_off[g + 1];
            uint64_t Hsum = 0, hl = 0;
            bool seg_inf = false, hold_inf = false, capped = false;
            for (int64_t cb = b.chain_cb_off[g]; cb < cb1; ++cb) {
                uint64_t t = (uint64_t)b.E[cb];
                bool t_inf = false;
                const uint32_t k1 = (uint32_t)(b.cb_seg_off[cb + 1] - seg_base);
                for (uint32_t k = (uint32_t)(b.cb_seg_off[cb] - seg_base); k < k1; ++k) {
                    const uint32_t h = sx->hq[k];
                    if (h >= kCapR) { // no bound
                        seg_inf = t_inf = true;
                        capped |= h == kCapR;
                    } else {
                        Hsum += h;
                        t += h + eps;
                    }
                }
                if (t_inf) hold_inf = true;
                else if (t > hl) hl = t;
            }
            const uint64_t cap = (uint64_t)Dv + 1;
            hsum = capped ? kCapR : seg_inf ? kInfR : (uint32_t)(Hsum < cap ? Hsum : cap);
            hold = hold_inf || hl >= kHoldInf ? kHoldInf : (uint32_t)hl;
        }
        s.emax[j] = hold;
        __syncwarp(gm);
        for (Mask lo = samex & ~higher & ~jbit & all; lo; lo &= lo - 1) // safe Lemma 4: the longest LP hold
            Bv = umax(Bv, s.emax[__ffs(lo) - 1]);
    }

    // ---- own recurrence terms ------------------------------------------------
    if (val) {
        const uint64_t own = (uint64_t)Sv + (uint64_t)dlv * blk;
        const uint64_t cap = (uint64_t)Dv + 1; // values above D act the same as D + 1
        const Mask needs = hp | (hpp & spins);
        s.rel[pos] = make_uint4(hp, hpp, hps, needs);
        s.seg0[pos] = seg0;
        s.needs[j] = needs;
        s.rec[pos] = make_uint4(Dv, Bv + Ev, (uint32_t)(own < cap ? own : cap), (uint32_t)((uint64_t)dlv * eps));
        // Lemma 2's sum is at least own + lb, lb = f delta sum_h S*_h (every segment's fixed
        // point is at least x + f sum_h S*_h with x = A* + blk, f = 2 if x >= 1, as mu >= 2
        // for t >= 1), kept capped at 2^27 like the interference sums it is compared with
        const uint64_t lb = (((uint64_t)Amn + blk) >= 1 ? 2 : 1) * (uint64_t)dlv * sums;
        s.seg[pos] = make_uint4((uint32_t)j, SAFE ? hsum : (lb < kNarrow ? (uint32_t)lb : kNarrow), blk, dlv);
    }
    __syncwarp(gm);

    // ---- Theorem 1 (Eq. 6), chain by chain -----------------------------------
    uint32_t Ehp = Ev, Ehpp = Ev + (sp ? 0u : (uint32_t)((uint64_t)dlv * eps)), Rv = 0;
    Mask sched = 0;
    const uint32_t k2 = (uint32_t)kappa2;
    auto chains = [&](auto counted_tag) {
    constexpr bool CNT = decltype(counted_tag)::value;
    // target mode: up to the target chain's step
    const int nsteps = TGT ? __shfl_sync(gm, pos, tgt, LG) + 1 : n;
    for (int step = 0; step < nsteps; ++step) {
        const uint4 rl = s.rel[step];
        if (rl.w & ~sched) { // a needed H*_h is not available (the chain is DEP)
            if (rank_row && !TGT) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        const uint4 rc = s.rec[step], sg = s.seg[step];
        const int c = (int)sg.x;
        const Mask cbit = 1u << c;
        const uint32_t D32 = rc.x, base = rc.y, own = rc.z, deps = rc.w;
        const uint32_t ccoef = ((rl.x >> j) & 1) ? Ehp : (((rl.y >> j) & 1) ? Ehpp : 0u);
        const uint32_t acoef = ((rl.z >> j) & 1) ? Sv : 0u;
        const uint32_t dl = sg.w;
        if (SAFE && dl && sg.y == kCapR) { // a segment recurrence was cut short: no bound (PAAM_ST_ITERCAP)
            if (j == c) Rv = kCapR;
            if (rank_row && !TGT) break;
            continue;
        }
        // start: B + E + H* with the interference part of Eq. 4 empty; Lemma 2's sum is
        // never below own = S* + delta blk (each segment's fixed point is at least its
        // A* + blk), so H* starts at own + delta eps either way
        uint32_t R = base + (dl ? own + deps : 0u);
        uint32_t hs = 0, ev = 0;
        bool ok = false, capped = false;
        if (R <= D32) {
            // Lemma 2's sum is at least own + lb: while Eq. 4's interference part is at
            // most lb, the minimum of Eq. 3 and Eq. 4 is Eq. 4; the exact per-segment fixed
            // points are taken at the first evaluation where it is larger, if any
            // (safe reading: the exact sum is known from the start, and lb is not used)
            uint32_t lb = (dl && !SAFE) ? sg.y : kInfR; // kInfR once they are taken
            uint32_t Hs = (SAFE && dl) ? sg.y : kInfR;  // Lemma 2's per-segment sum: unbounded, or not needed yet
            // every deadline is below 2^27 - 16: in the loop base <= R <= D, each group
            // sum is capped at 2^27 where it is added (a capped term already exceeds D)
            for (;;) { // twice at most: before and after the fixed points are taken
                bool need = false;
                for (;;) {
                    if (CNT && ev++ == kIterCap) break;
                    const uint32_t cs = __reduce_add_sync(gm, capped_term(R, tm2, mg, lg, ccoef));
                    const uint32_t as = umin(__reduce_add_sync(gm, capped_term(R, tm2, mg, lg, acoef)), kNarrow);
                    hs = 0;
                    if (dl) {
                        if (as > lb) { // this evaluation is taken again once Lemma 2's sum is known
                            need = true;
                            if (CNT) --ev;
                            break;
                        }
                        hs = umin(Hs, own + as) + deps; // Eq. 1 with min(Eq. 3, Eq. 4)
                    }
                    const uint32_t Rn = base + umin(hs, kNarrow) + umin(cs, kNarrow);
                    if (Rn == R) {
                        ok = true;
                        break;
                    }
                    R = Rn;
                    if (R > D32) break;
                }
                if (!need) break;
                lb = kInfR;
                // the sum matters only below Eq. 4 at R = D (and below D + 1)
                const uint32_t hchd = umin(__reduce_add_sync(gm, capped_term(D32, tm2, mg, lg, acoef)), kNarrow);
                const uint32_t lim = umin(own + hchd, D32 + 1);
                const uint32_t blkc = s.seg[step].z;
                const int64_t qb = s.seg_base + s.seg0[step];
                uint32_t H32 = 0;
                bool inf = false;
                for (uint32_t q = 0; q < dl && !inf; ++q) {
                    const uint32_t hb = (uint32_t)b.A[qb + q] + k2 + blkc;
                    uint32_t h = hb; // the recurrence starts with the first two terms
                    uint32_t evs = 0;
                    for (;;) {
                        if (h > D32 || H32 + h >= lim) {
                            inf = true;
                            break;
                        }
                        if (CNT && evs++ == kIterCap) {
                            inf = capped = true;
                            break;
                        }
                        const uint32_t nh =
                            hb + umin(__reduce_add_sync(gm, capped_term(h, tm2, mg, lg, acoef)), kNarrow);
                        if (nh == h) break; // strictly increasing until here, bounded by D
                        h = nh;
                    }
                    H32 += h;
                }
                if (capped) break; // a segment recurrence was cut short
                if (!inf) Hs = H32;
            }
        }
        if (capped) { // no bound (PAAM_ST_ITERCAP)
            if (j == c) Rv = kCapR;
            if (rank_row && !TGT) break;
            continue;
        }
        if (ok) {
            sched |= cbit;
            if (j == c) {
                Rv = R;
                Ehp = Ev + hs;
                if (sp) Ehpp = Ev + hs;
            }
        } else {
            if (ev > kIterCap && j == c) Rv = kCapR; // the recurrence was cut short (PAAM_ST_ITERCAP)
            if (rank_row && !TGT) break;
        }
    }
    };
    if (counted)
        chains(std::true_type{});
    else
        chains(std::false_type{});

    // ---- outputs -------------------------------------------------------------
    {
    const int64_t c0 = s.c0, sys = s.sys;
    const int32_t cand = s.cand;
    if (TGT) { // the target chain's verdict; first_ok is not touched
        if (lane == 0) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = ((sched >> tgt) & 1) ? 1 : 0;
        __syncwarp(gm);
        return;
    }
    if (rank_row) {
        if (lane == 0) {
            const bool ok = sched == all;
            if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = ok ? 1 : 0;
            if (ok) atomicMin(p.first_ok + sys, cand);
        }
        __syncwarp(gm);
        return;
    }
    if (val) {
        const bool ok = (sched >> j) & 1;
        R_out[c0 + j] = ok ? (int64_t)Rv : -1;
        // DEP: skipped at its step, i.e. some chain of its DEP-rule set (all earlier in
        // the analysis order) is not schedulable
        st_out[c0 + j] = ok ? PAAM_ST_SCHED
                            : (Rv == kCapR ? PAAM_ST_ITERCAP : ((s.needs[j] & ~sched) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
    }
    if (lane == 0 && verdict) verdict[sys] = sched == all ? 1 : 0;
    }
    __syncwarp(gm);
}

// BLOCKS resident blocks of 256 threads per SM: the register budget per thread.
// Items are all of the launch (list == nullptr) or list[0 .. *count).
template <int LG, int BLOCKS, bool REC, bool TGT = false, bool SAFE = false>
__global__ void __launch_bounds__(256, BLOCKS) analyze_lazy_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                                   uint8_t *st, uint8_t *verdict, const int32_t *list,
                                                                   const int32_t *count, int32_t *big_list,
                                                                   int32_t *big_count, int32_t *wide_list,
                                                                   int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / LG;
    const int grp = threadIdx.x / LG;
    const int lane = threadIdx.x % LG;
    using SM = typename std::conditional<SAFE, LazySafeSmem<LG>, LazySmem<LG>>::type;
    SM &s = reinterpret_cast<SM *>(smem_raw)[grp];
    LazySafeExt<LG> *sx = nullptr;
    if constexpr (SAFE) sx = &s.x;
    const unsigned gm = rgroup_mask<LG>();
    const int64_t n_items = list ? (int64_t)*count : (p.K > 0 ? b.n_sys * p.K : b.n_sys);
    for_each_item<LG>(p, n_items, grp, groups, lane, gm, [&](int64_t i) {
        // first pass over a batch's systems, handed out in increasing order (within
        // windows of the size binning): the group that starts each slice of
        // kPrefetchSlice items prefetches the same slice of the next window's systems,
        // so the prefetches of a window are spread over many SMs
        if (!list && p.K == 0 && lane == 0 && i % kPrefetchSlice == 0)
            prefetch_systems(b, p.sys_order, i + kBinWindow, kPrefetchSlice);
        const int64_t item = list ? (int64_t)list[i] : i;
        lazy_system<LG, REC, TGT, SAFE>(b, p, item, s, sx, lane, gm, R, st, verdict, big_list, big_count, wide_list,
                                        wide_count);
    });
}

// one warp per system, one lane per chain: the records of chain_recs
__global__ void __launch_bounds__(256) chain_records_kernel(BatchDev b, uint64_t kappa2, uint64_t eps, uint4 *recs)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t sys = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); sys < b.n_sys; sys += nw) {
        const int64_t c0 = b.sys_chain_off[sys];
        const int n = (int)(b.sys_chain_off[sys + 1] - c0);
        if (n <= 0) continue;
        const int64_t seg_base = b.cb_seg_off[b.chain_cb_off[c0]];
        const int64_t x0 = b.sys_exec_off[sys];
        for (int j = lane; j < n; j += 32) {
            const int64_t g = c0 + j;
            ChainAgg a;
            chain_aggregates(b, g, kappa2, eps, a);
            const int32_t ex = b.exec[g];
            const int32_t co = b.exec_core[x0 + ex];
            const unsigned sp = b.spin[g] != 0 ? 1u : 0u;
            // the chains of the same executor and of the same core (systems of up to 32
            // chains, the ones the lazy kernels read records for)
            uint32_t sx = 0, sc = 0;
            if (n <= 32) {
                const unsigned act = n == 32 ? 0xffffffffu : (1u << n) - 1u; // lanes j < n
                sx = __match_any_sync(act, ex);
                sc = __match_any_sync(act, co);
            }
            uint4 *r = recs + g * 4;
            r[0] = make_uint4(a.tm2, a.mg, a.lg, a.D);
            r[1] = make_uint4(a.E, a.S, a.Emax, a.M);
            r[2] = make_uint4(a.Amin, a.dl, (uint32_t)(a.q0 - seg_base), a.fit | (sp << 1));
            r[3] = make_uint4((uint32_t)ex, (uint32_t)co, sx, sc);
        }
    }
}

} // namespace

int paam_launch_chain_records(const paam_batch *bt, const AnalysisParams &p, uint4 *recs, cudaStream_t stream)
{
    if (bt->n_sys <= 0) return PAAM_OK;
    int64_t blocks = (bt->n_sys + 7) / 8;
    if (blocks > 16 * (int64_t)bt->ctx->n_sm) blocks = 16 * (int64_t)bt->ctx->n_sm;
    chain_records_kernel<<<(unsigned)blocks, 256, 0, stream>>>(batch_dev(bt), 2 * (uint64_t)p.kappa,
                                                               (uint64_t)p.eps, recs);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}

template <int LG, int BLOCKS>
int launch_lazy_pass(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                     const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream)
{
    if (threads % 32 != 0 || threads > 256) return PAAM_E_INVAL;
    const int groups = threads / LG;
    const size_t smem = sizeof(LazySmem<LG>) * groups;
    auto kern = p.chain_recs ? analyze_lazy_kernel<LG, BLOCKS, true> : analyze_lazy_kernel<LG, BLOCKS, false>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, list, count, bt->list_big,
                                                      bt->counts, bt->list_wide, bt->counts + 1);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

int paam_launch_lazy_safe(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                          int64_t max_items, cudaStream_t stream)
{
    constexpr int LG = 16, threads = 256;
    const int groups = threads / LG;
    const size_t smem = sizeof(LazySafeSmem<LG>) * groups;
    auto kern = analyze_lazy_kernel<LG, 5, false, false, true>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // every deferred system (over 16 chains or kSafeSegs segments, not narrow,
    // outside the 32-bit bound) to the int64 kernel's list
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, nullptr, nullptr,
                                                      bt->list_wide, bt->counts + 1, bt->list_wide, bt->counts + 1);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

int paam_launch_lazy_target(const paam_batch *bt, const AnalysisParams &p, int32_t *list, int32_t *count,
                            int64_t max_items, cudaStream_t stream)
{
    constexpr int LG = 16, threads = 256;
    const int groups = threads / LG;
    const size_t smem = sizeof(LazySmem<LG>) * groups;
    auto kern = p.chain_recs ? analyze_lazy_kernel<LG, 5, true, true> : analyze_lazy_kernel<LG, 5, false, true>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // every deferred trial (over 16 chains, not narrow, outside the 32-bit bound) to list
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                      list, count, list, count);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

template <int BLOCKS>
int launch_lazy(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream)
{
    if (list || count) return PAAM_E_INVAL; // first pass only: every item of the launch
    return launch_lazy_pass<16, BLOCKS>(bt, p, R, st, verdict, nullptr, nullptr, max_items, threads, stream);
}

template <int BLOCKS>
int launch_lazy32(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream)
{
    if (!list || !count) return PAAM_E_INVAL; // the pass over the deferral list
    return launch_lazy_pass<32, BLOCKS>(bt, p, R, st, verdict, list, count, max_items, threads, stream);
}

template int launch_lazy<4>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                            const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_lazy<5>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                            const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_lazy<6>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                            const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_lazy32<6>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                              const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
