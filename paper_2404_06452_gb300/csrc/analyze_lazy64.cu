// analyze_lazy64.cu -- the lazy register-table analysis for systems of 33 to
// 64 chains: one warp per system, two chains per lane (chain j = lane + 32 k,
// slot k), 64-bit chain masks.
//
// The mathematics and the order of work are those of analyze_lazy.cu (see
// there): Theorem 1 (Eq. 6) with Eqs. 1-5 chain by chain in the analysis
// order, Lemma 1's arrival counts by multiply-shift division, the 32-bit
// narrow sums (every deadline below 2^27 - 64; each lane adds its two capped
// terms and caps the pair at 2^27 - 1, so 32 lanes' sum fits 32 bits and a
// capped sum still exceeds every deadline), the relations from priority slots
// and suffix scans (or one comparison per chain pair for priorities of 64 and
// more), the same-bucket blocking and Lemma 2's lower bound from scans in
// priority order, Lemma 2's exact per-segment fixed points taken only at the
// first evaluation that needs them, and the DEP rule read back after the
// steps.  It takes the deferral list after the 32-lane pass (systems below
// AnalysisParams::min_chains were taken there); systems that are not narrow
// go to the int64 kernel's list.  One accelerator, Lemma 4 as printed,
// analysis and candidate mode.
#include "reg_common.cuh"

namespace {
using namespace paam_reg;

constexpr int kW = 32;       // lanes per system
constexpr int kN = 64;       // chain slots per system
using Mask = uint64_t;

struct Rel64 {
    Mask hp, hpp, hps, needs; // needs = hp and the spinning hpp: all must be schedulable (DEP rule)
};

struct Lazy64Smem {
    Rel64 rel[kN];       // by analysis position
    uint4 rec[kN];       // {D, base = B + E, own = S* + delta blk (capped at D + 1), deps = delta eps}
    uint4 seg[kN];       // {chain index, lb (Lemma 2's lower bound), blk, delta}
    uint32_t seg0[kN];   // by analysis position: first segment relative to the system's first
    Mask needs[kN];      // by chain: its DEP-rule set, read again for the status
    uint32_t emax[kN];   // by chain: longest callback (Lemma 4)
    uint32_t m[kN];      // by chain: M* (same-bucket blocking with several buckets)
    int32_t bucket[kN];  // by chain
    uint32_t msort[kN];  // by priority rank: M* of the users (0 for the others)
    uint32_t ssort[kN];  // by priority rank: S* of the users (capped at 2^27 - 1)
    Mask xms[kN];        // by executor index: its chains
    Mask cms[kN];        // by core index: the chains of its executors
    Mask exm[kN];        // by executor priority value: the chains of that executor priority
    Mask inv[kN];        // by chain priority value: the chain of that priority
    int32_t xep[kN];     // by executor index: its highest chain priority (criticality-as-priority)
    int64_t c0, sys, seg_base;
    int32_t cand;
};

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src)
{
    const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src), hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl64_down(uint64_t v, int d)
{
    const uint32_t lo = __shfl_down_sync(kFull, (uint32_t)v, d), hi = __shfl_down_sync(kFull, (uint32_t)(v >> 32), d);
    return ((uint64_t)hi << 32) | lo;
}

// value of slot v (0..63) of a pair {slot lane, slot lane + 32} held by every lane
template <typename V>
__device__ __forceinline__ V slot_value(V a0, V a1, int v)
{
    V x0, x1;
    if constexpr (sizeof(V) == 8) {
        x0 = shfl64(a0, v & 31);
        x1 = shfl64(a1, v & 31);
    } else {
        x0 = __shfl_sync(kFull, a0, v & 31);
        x1 = __shfl_sync(kFull, a1, v & 31);
    }
    return v < 32 ? x0 : x1;
}

// exclusive suffix OR over the 64 slots: out(v) = OR of slots v + 1 .. 63
__device__ __forceinline__ void suffix_or_excl(uint64_t &a0, uint64_t &a1, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t w0 = shfl64_down(a0, d), w1 = shfl64_down(a1, d);
        if (lane + d < 32) {
            a0 |= w0;
            a1 |= w1;
        }
    }
    const uint64_t upper = shfl64(a1, 0); // slots 32..63
    a0 |= upper;
    const uint64_t n0 = shfl64_down(a0, 1), n1 = shfl64_down(a1, 1);
    a0 = lane < 31 ? n0 : upper;
    a1 = lane < 31 ? n1 : 0ull;
}

// exclusive suffix maximum over the 64 slots
__device__ __forceinline__ void suffix_max_excl(uint32_t &a0, uint32_t &a1, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t w0 = __shfl_down_sync(kFull, a0, d), w1 = __shfl_down_sync(kFull, a1, d);
        if (lane + d < 32) {
            a0 = umax(a0, w0);
            a1 = umax(a1, w1);
        }
    }
    const uint32_t upper = __shfl_sync(kFull, a1, 0);
    a0 = umax(a0, upper);
    const uint32_t n0 = __shfl_down_sync(kFull, a0, 1), n1 = __shfl_down_sync(kFull, a1, 1);
    a0 = lane < 31 ? n0 : upper;
    a1 = lane < 31 ? n1 : 0u;
}

// exclusive prefix sum over the 64 slots, saturating at 2^27
__device__ __forceinline__ void prefix_sum_excl(uint32_t &a0, uint32_t &a1, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t w0 = __shfl_up_sync(kFull, a0, d), w1 = __shfl_up_sync(kFull, a1, d);
        if (lane >= d) {
            a0 = umin(a0 + w0, kNarrow);
            a1 = umin(a1 + w1, kNarrow);
        }
    }
    const uint32_t lower = __shfl_sync(kFull, a0, 31); // slots 0..31
    a1 = umin(a1 + lower, kNarrow);
    const uint32_t p0 = __shfl_up_sync(kFull, a0, 1), p1 = __shfl_up_sync(kFull, a1, 1);
    a0 = lane > 0 ? p0 : 0u;
    a1 = lane > 0 ? p1 : lower;
}

// ceil(t / T) + 1 (Lemma 1) times c, capped at 2^27 - 1
__device__ __forceinline__ uint32_t capped_term(uint32_t t, uint32_t tm2, uint32_t mg, uint32_t lg, uint32_t c)
{
    const uint64_t v = (uint64_t)rarrivals(t, tm2, mg, lg) * c;
    return v < kNarrow - 1 ? (uint32_t)v : kNarrow - 1;
}

// the group sum over both slots of every lane
__device__ __forceinline__ uint32_t pair_sum(uint32_t t, const uint32_t (&tm2)[2], const uint32_t (&mg)[2],
                                             const uint32_t (&lg)[2], uint32_t c0, uint32_t c1)
{
    const uint32_t v = umin(capped_term(t, tm2[0], mg[0], lg[0], c0) + capped_term(t, tm2[1], mg[1], lg[1], c1),
                            kNarrow - 1);
    return __reduce_add_sync(kFull, v);
}

__device__ void lazy64_system(const BatchDev &b, const AnalysisParams &p, int64_t item, Lazy64Smem &s, int lane,
                              int64_t *__restrict__ R_out, uint8_t *__restrict__ st_out,
                              uint8_t *__restrict__ verdict, int32_t *wide_list, int32_t *wide_count)
{
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int pruned = __shfl_sync(kFull, cand_pruned(p, sys, cand) ? 1 : 0, 0);
        if (pruned) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    if (n < p.min_chains) return; // an earlier pass over the same list took it
    if (n > kN) {                 // not a validated batch's; the int64 kernel reports it
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;

    // ---- per-chain aggregates (Sec. II-C), two slots per lane ----------------
    uint32_t tm2[2], mg[2], lg[2], Dv[2], Ev[2], Sv[2], Emx[2], Mv[2], Amn[2], dlv[2], seg0[2];
    int32_t pr[2], ep[2], ex[2], co[2];
    bool sp[2], val[2];
    unsigned fit = 1, rank_ok = 1;
    Mask rbit = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int j = lane + kW * k;
        val[k] = j < n;
        tm2[k] = mg[k] = lg[k] = Dv[k] = Ev[k] = Sv[k] = Emx[k] = Mv[k] = Amn[k] = dlv[k] = seg0[k] = 0;
        pr[k] = ep[k] = INT32_MIN;
        ex[k] = co[k] = -1 - j;
        sp[k] = false;
        if (!val[k]) continue;
        const int64_t g = c0 + j;
        const int64_t T = b.T[g], D = b.D[g];
        ex[k] = b.exec[g];
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[j];
            const bool ok = r >= 0 && r < n;
            rank_ok &= ok ? 1u : 0u;
            rbit |= ok ? (Mask)1 << r : 0;
            pr[k] = n - 1 - r;
        } else {
            pr[k] = b.prio[g];
        }
        co[k] = b.exec_core[x0 + ex[k]];
        if (xprio) ep[k] = xprio[x0 + ex[k]];
        sp[k] = b.spin[g] != 0;
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        // sums and extremes in 32 bits over values capped at 2^30 (a capped value
        // takes its chain's sum to the 32-bit bound, and the system to the int64 kernel)
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
            const uint32_t a = ((uint64_t)Ap[i] < kFitR ? (uint32_t)Ap[i] : (uint32_t)kFitR) + k2c; // A* = A + 2 kappa
            S = umin(S + a, (uint32_t)kFitR);
            M = umax(M, a);
            Amin = umin(Amin, a);
        }
        const uint64_t dl = (uint64_t)nq;
        const bool f = (uint64_t)T < kFitR && (uint64_t)D < kFitR && E < kFitR && S < kFitR && dl < kFitR &&
                       (eps == 0 || dl <= (kFitR - 1) / eps);
        fit &= f ? 1u : 0u;
        if (f) rdivisor((uint32_t)T, tm2[k], mg[k], lg[k]);
        Dv[k] = (uint32_t)D;
        Ev[k] = E;
        Sv[k] = S;
        Emx[k] = Emax;
        Mv[k] = M;
        Amn[k] = dl ? (Amin < kFitR ? Amin : 0u) : 0u;
        dlv[k] = (uint32_t)dl;
        seg0[k] = (uint32_t)(q0 - seg_base);
    }
    if (lane == 0) {
        s.c0 = c0;
        s.sys = sys;
        s.seg_base = seg_base;
        s.cand = cand;
    }
    const Mask users = (Mask)__ballot_sync(kFull, val[0] && dlv[0] != 0) |
                       ((Mask)__ballot_sync(kFull, val[1] && dlv[1] != 0) << 32);
    const Mask spins = (Mask)__ballot_sync(kFull, sp[0]) | ((Mask)__ballot_sync(kFull, sp[1]) << 32);
    const Mask all = n >= 64 ? ~(Mask)0 : (((Mask)1 << n) - 1);
    if (rank_row) { // a candidate must be a permutation of 0..n-1
        rank_ok = __reduce_and_sync(kFull, rank_ok);
        const Mask rb = (Mask)__reduce_or_sync(kFull, (uint32_t)rbit) |
                        ((Mask)__reduce_or_sync(kFull, (uint32_t)(rbit >> 32)) << 32);
        if (!rank_ok || rb != all) {
            if (lane == 0) {
                atomicExch(p.err, PAAM_E_INVAL);
                if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = 0;
            }
            return;
        }
    }
    if (!__reduce_and_sync(kFull, fit)) { // outside the 32-bit bound
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    const uint32_t dmax = __reduce_max_sync(kFull, umax(Dv[0], Dv[1]));
    if (dmax >= kNarrow - kN) { // inside it but not narrow: the int64 kernel
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    // The system's iteration bound (as in analyze_lazy.cu): no recurrence of Eq. 3 or
    // Eq. 6 takes more than L = sum_h ceil(Dmax / T_h) + 2 evaluations; with L within
    // kIterCap the loops run without counters, otherwise every loop stops at kIterCap.
    uint32_t lpart = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (val[k]) lpart += umin(rarrivals(dmax, tm2[k], mg[k], lg[k]) - 1u, kIterCap + 1u);
    const uint32_t L = __reduce_add_sync(kFull, lpart) + 2u;
    const bool counted = L > kIterCap;

    // ---- relations (Lemma 4, Theorem 1, Eq. 3), analysis order ---------------
    Mask samex[2], corem[2], eqx[2], higher[2], ehigher[2];
    const bool small = __reduce_and_sync(
        kFull, ((!val[0] || ((uint32_t)ex[0] < kN && (uint32_t)co[0] < kN && (uint32_t)pr[0] < kN &&
                              (!xprio || (uint32_t)ep[0] < kN))) &&
                (!val[1] || ((uint32_t)ex[1] < kN && (uint32_t)co[1] < kN && (uint32_t)pr[1] < kN &&
                              (!xprio || (uint32_t)ep[1] < kN))))
            ? 1u
            : 0u);
    if (small) {
        // keys below 64 (executor and core indices, a permutation of 0..n-1 as chain
        // priorities, executor priorities taken from them) index slots of shared
        // memory into which each chain ORs its bit; the set above a priority value is
        // the OR of the slots past it, a suffix scan over the 64 slots
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int v = lane + kW * k;
            s.xms[v] = s.cms[v] = s.exm[v] = s.inv[v] = 0;
            s.xep[v] = INT32_MIN;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (val[k]) {
                const Mask bit = (Mask)1 << (lane + kW * k);
                atomicOr((unsigned long long *)&s.xms[ex[k]], (unsigned long long)bit);
                atomicOr((unsigned long long *)&s.cms[co[k]], (unsigned long long)bit);
                if (!xprio) atomicMax(&s.xep[ex[k]], pr[k]);
            }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const Mask bit = (Mask)1 << (lane + kW * k);
            samex[k] = val[k] ? s.xms[ex[k]] : bit;
            corem[k] = val[k] ? s.cms[co[k]] : bit;
            if (!xprio && val[k]) ep[k] = s.xep[ex[k]]; // criticality-as-priority
            if (val[k]) {
                s.inv[pr[k]] = bit; // distinct priorities: one chain per slot
                atomicOr((unsigned long long *)&s.exm[ep[k]], (unsigned long long)bit);
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) eqx[k] = val[k] ? s.exm[ep[k]] : (Mask)1 << (lane + kW * k);
        uint64_t a0 = s.inv[lane], a1 = s.inv[lane + kW], e0 = s.exm[lane], e1 = s.exm[lane + kW];
        suffix_or_excl(a0, a1, lane);
        suffix_or_excl(e0, e1, lane);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            higher[k] = slot_value(a0, a1, val[k] ? pr[k] : 0);
            ehigher[k] = slot_value(e0, e1, val[k] ? ep[k] : 0);
            if (!val[k]) higher[k] = ehigher[k] = all;
        }
    } else { // one comparison each per chain pair
        if (!xprio) { // criticality-as-priority: the highest chain priority on the executor
            int32_t best[2] = {INT32_MIN, INT32_MIN};
            for (int t = 0; t < n; ++t) {
                const int32_t pt = slot_value(pr[0], pr[1], t), xt = slot_value(ex[0], ex[1], t);
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (xt == ex[k] && pt > best[k]) best[k] = pt;
            }
            ep[0] = best[0];
            ep[1] = best[1];
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) samex[k] = corem[k] = eqx[k] = higher[k] = ehigher[k] = 0;
        for (int t = 0; t < n; ++t) {
            const int32_t pt = slot_value(pr[0], pr[1], t), et = slot_value(ep[0], ep[1], t);
            const int32_t xt = slot_value(ex[0], ex[1], t), kt = slot_value(co[0], co[1], t);
            const Mask bit = (Mask)1 << t;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                samex[k] |= xt == ex[k] ? bit : 0;
                corem[k] |= kt == co[k] ? bit : 0;
                eqx[k] |= et == ep[k] ? bit : 0;
                higher[k] |= pt > pr[k] ? bit : 0;
                ehigher[k] |= et > ep[k] ? bit : 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (!val[k]) { // past n: only itself on its executor and core
                const Mask bit = (Mask)1 << (lane + kW * k);
                samex[k] = corem[k] = eqx[k] = bit;
                higher[k] = ehigher[k] = all;
            }
    }
    const bool one_bucket = p.n_buckets == 1;
    int pos[2], prank[2];
    Mask hp[2], hpp[2], hps[2];
    bool user[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int j = lane + kW * k;
        // position in the analysis order: executor priority, then chain priority
        pos[k] = __popcll(ehigher[k]) + __popcll(eqx[k] & higher[k] & all);
        hp[k] = samex[k] & higher[k];            // hp(c), Lemma 4
        hpp[k] = corem[k] & ~samex[k] & ehigher[k]; // hpp(c), Theorem 1
        hps[k] = users & higher[k];              // hps(c), Eq. 3
        user[k] = (users >> j) & 1;
        prank[k] = __popcll(higher[k]); // rank by chain priority, 0 = highest
        s.emax[j] = Emx[k];
        s.m[j] = Mv[k];
        if (val[k]) {
            s.ssort[prank[k]] = user[k] ? umin(Sv[k], kNarrow - 1) : 0u;
            s.msort[prank[k]] = user[k] ? Mv[k] : 0u;
        }
    }
    __syncwarp();
    // sum_h S*_h over hps(c): a prefix sum in priority order, saturating at 2^27
    uint32_t sums[2];
    {
        uint32_t a0 = lane < n ? s.ssort[lane] : 0u, a1 = lane + kW < n ? s.ssort[lane + kW] : 0u;
        prefix_sum_excl(a0, a1, lane);
#pragma unroll
        for (int k = 0; k < 2; ++k) sums[k] = slot_value(a0, a1, prank[k] < kN ? prank[k] : 0);
    }
    uint32_t Bv[2] = {0u, 0u}, blk[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const Mask jb = (Mask)1 << (lane + kW * k);
        for (Mask lo = samex[k] & ~higher[k] & ~jb & all; lo; lo &= lo - 1) // Lemma 4: one LP callback
            Bv[k] = umax(Bv[k], s.emax[__ffsll((long long)lo) - 1]);
    }
    if (one_bucket) { // every user shares the bucket: the longest lower-priority request (R2-R3)
        uint32_t a0 = lane < n ? s.msort[lane] : 0u, a1 = lane + kW < n ? s.msort[lane + kW] : 0u;
        suffix_max_excl(a0, a1, lane);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t below = slot_value(a0, a1, prank[k] < kN ? prank[k] : 0);
            if (user[k]) blk[k] = below;
        }
    } else { // bucket = floor(rank * n_buckets / |U|), rank among the users (R2)
        const uint32_t nu = (uint32_t)__popcll(users);
        int32_t bk[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            bk[k] = user[k] ? (int32_t)((uint32_t)__popcll(hps[k]) * (uint32_t)p.n_buckets / nu) : -1;
            s.bucket[lane + kW * k] = bk[k];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const Mask jb = (Mask)1 << (lane + kW * k);
            if (user[k])
                for (Mask lo = users & ~higher[k] & ~jb; lo; lo &= lo - 1) {
                    const int l = __ffsll((long long)lo) - 1;
                    if (s.bucket[l] == bk[k]) blk[k] = umax(blk[k], s.m[l]);
                }
        }
    }

    // ---- own recurrence terms ------------------------------------------------
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (!val[k]) continue;
        const int j = lane + kW * k;
        const uint64_t own = (uint64_t)Sv[k] + (uint64_t)dlv[k] * blk[k];
        const uint64_t cap = (uint64_t)Dv[k] + 1; // values above D act the same as D + 1
        const Mask needs = hp[k] | (hpp[k] & spins);
        s.rel[pos[k]] = Rel64{hp[k], hpp[k], hps[k], needs};
        s.seg0[pos[k]] = seg0[k];
        s.needs[j] = needs;
        s.rec[pos[k]] = make_uint4(Dv[k], Bv[k] + Ev[k], (uint32_t)(own < cap ? own : cap),
                                   (uint32_t)((uint64_t)dlv[k] * eps));
        // Lemma 2's sum is at least own + lb, lb = f delta sum_h S*_h (f = 2 if A* + blk >= 1)
        const uint64_t lb = (((uint64_t)Amn[k] + blk[k]) >= 1 ? 2 : 1) * (uint64_t)dlv[k] * sums[k];
        s.seg[pos[k]] = make_uint4((uint32_t)j, lb < kNarrow ? (uint32_t)lb : kNarrow, blk[k], dlv[k]);
    }
    __syncwarp();

    // ---- Theorem 1 (Eq. 6), chain by chain -----------------------------------
    uint32_t Ehp[2], Ehpp[2], Rv[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        Ehp[k] = Ev[k];
        Ehpp[k] = Ev[k] + (sp[k] ? 0u : (uint32_t)((uint64_t)dlv[k] * eps));
    }
    Mask sched = 0;
    const uint32_t k2 = (uint32_t)kappa2;
    auto chains = [&](auto counted_tag) {
    constexpr bool CNT = decltype(counted_tag)::value;
    for (int step = 0; step < n; ++step) {
        const Rel64 rl = s.rel[step];
        if (rl.needs & ~sched) { // a needed H*_h is not available (the chain is DEP)
            if (rank_row) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        const uint4 rc = s.rec[step], sg = s.seg[step];
        const int c = (int)sg.x;
        const uint32_t D32 = rc.x, base = rc.y, own = rc.z, deps = rc.w;
        uint32_t cc[2], ac[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int j = lane + kW * k;
            cc[k] = ((rl.hp >> j) & 1) ? Ehp[k] : (((rl.hpp >> j) & 1) ? Ehpp[k] : 0u);
            ac[k] = ((rl.hps >> j) & 1) ? Sv[k] : 0u;
        }
        const uint32_t dl = sg.w;
        // start: B + E + H* with the interference part of Eq. 4 empty; Lemma 2's sum is
        // never below own, so H* starts at own + delta eps either way
        uint32_t R = base + (dl ? own + deps : 0u);
        uint32_t hs = 0, ev = 0;
        bool ok = false, capped = false;
        if (R <= D32) {
            uint32_t lb = dl ? sg.y : kInfR; // kInfR once the fixed points are taken
            uint32_t Hs = kInfR;             // Lemma 2's per-segment sum: unbounded, or not needed yet
            for (;;) { // twice at most: before and after the fixed points are taken
                bool need = false;
                for (;;) {
                    if (CNT && ev++ == kIterCap) break;
                    const uint32_t cs = pair_sum(R, tm2, mg, lg, cc[0], cc[1]);
                    const uint32_t as = umin(pair_sum(R, tm2, mg, lg, ac[0], ac[1]), kNarrow);
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
                const uint32_t hchd = umin(pair_sum(D32, tm2, mg, lg, ac[0], ac[1]), kNarrow);
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
                        const uint32_t nh = hb + umin(pair_sum(h, tm2, mg, lg, ac[0], ac[1]), kNarrow);
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
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (lane + kW * k == c) Rv[k] = kCapR;
            if (rank_row) break;
            continue;
        }
        if (ok) {
            sched |= (Mask)1 << c;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (lane + kW * k == c) {
                    Rv[k] = R;
                    Ehp[k] = Ev[k] + hs;
                    if (sp[k]) Ehpp[k] = Ev[k] + hs;
                }
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (ev > kIterCap && lane + kW * k == c) Rv[k] = kCapR; // cut short (PAAM_ST_ITERCAP)
            if (rank_row) break;
        }
    }
    };
    if (counted)
        chains(std::true_type{});
    else
        chains(std::false_type{});

    // ---- outputs -------------------------------------------------------------
    {
        const int64_t c0s = s.c0, syss = s.sys;
        const int32_t cands = s.cand;
        if (rank_row) {
            if (lane == 0) {
                const bool ok = sched == all;
                if (p.cand_ok) p.cand_ok[syss * p.Kc + cand_of(p, syss, cands)] = ok ? 1 : 0;
                if (ok) atomicMin(p.first_ok + syss, cands);
            }
            __syncwarp();
            return;
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!val[k]) continue;
            const int j = lane + kW * k;
            const bool ok = (sched >> j) & 1;
            R_out[c0s + j] = ok ? (int64_t)Rv[k] : -1;
            // DEP: skipped at its step, i.e. some chain of its DEP-rule set (all earlier in
            // the analysis order) is not schedulable
            st_out[c0s + j] = ok ? PAAM_ST_SCHED
                                 : (Rv[k] == kCapR ? PAAM_ST_ITERCAP
                                                   : ((s.needs[j] & ~sched) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
        }
        if (lane == 0 && verdict) verdict[syss] = sched == all ? 1 : 0;
    }
    __syncwarp();
}

// BLOCKS resident blocks of 256 threads per SM (three: 80 registers, which beat two
// blocks without spills by 3.5% on the 4M-system workload); items list[0 .. *count)
template <int BLOCKS>
__global__ void __launch_bounds__(256, BLOCKS) analyze_lazy64_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                                     uint8_t *st, uint8_t *verdict,
                                                                     const int32_t *list, const int32_t *count,
                                                                     int32_t *wide_list, int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / kW;
    const int grp = threadIdx.x / kW;
    const int lane = threadIdx.x % kW;
    Lazy64Smem &s = reinterpret_cast<Lazy64Smem *>(smem_raw)[grp];
    const int64_t n_items = (int64_t)*count;
    for_each_item<kW>(p, n_items, grp, groups, lane, kFull, [&](int64_t i) {
        lazy64_system(b, p, (int64_t)list[i], s, lane, R, st, verdict, wide_list, wide_count);
    });
}

} // namespace

int launch_lazy64(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                  const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream)
{
    if (!list || !count || threads % 32 != 0 || threads > 256) return PAAM_E_INVAL;
    const int groups = threads / kW;
    const size_t smem = sizeof(Lazy64Smem) * groups;
    auto kern = analyze_lazy64_kernel<3>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, list, count, bt->list_wide,
                                                      bt->counts + 1);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}
