// analyze_lazy_acc.cu -- the lazy register-table analysis of systems whose
// segments use several accelerators (rule R1: one server per accelerator,
// analysed on its own; reading R10).
//
// The work order of analyze_lazy.cu (relations from priority slots and scans,
// Lemma 2's per-segment fixed points only at the first evaluation of a chain's
// own recurrence that needs them, the DEP rule read back after the steps)
// with an accelerator dimension on every server-side quantity: per
// accelerator u its users U_u, their buckets (rank
// among U_u, Sec. IV-C), the same-bucket blocking blk_u (R2-R3), the
// higher-priority users hps_u (Eq. 3, Eq. 4), Lemma 2's fixed points over the
// chain's segments on u (Eq. 3) and Eq. 4's per-chain bound own_u + sum over
// hps_u of mu(t) S*_{h,u}.  A chain's handling time is the sum over the
// accelerators it uses of min(Eq. 3 sum, Eq. 4), plus delta eps over all its
// segments (Eq. 1); the chain recurrence of Theorem 1 (Eq. 6) is otherwise
// that of one accelerator.  One system per group of 16 lanes, one chain per
// lane, the 32-bit narrow sums (every deadline below 2^27 - 16); systems with
// more chains, outside the 32-bit bound or not narrow go to the int64
// kernel's list.  Lemma 4 as printed, analysis and candidate mode.
#include "reg_common.cuh"

namespace {
using namespace paam_reg;

constexpr int kG = 16;
using Mask = uint32_t;

template <int NACC>
struct LazyAccSmem {
    uint4 rel[kG];          // by analysis position: {hp, hpp, needs (DEP rule), first segment}
    uint4 rec[kG];          // {D, base = B + E, deps = delta eps (all segments), delta (all segments)}
    uint4 acc[kG][NACC];    // per accelerator: {own = S*_u + delta_u blk_u (capped at D + 1), lb_u, blk_u, delta_u}
    uint32_t hps[kG][NACC]; // per accelerator: hps_u
    uint32_t chain[kG];     // by analysis position: the chain
    uint32_t needs[kG];     // by chain: its DEP-rule set, read again for the status
    uint32_t emax[kG];      // by chain: longest callback (Lemma 4)
    uint32_t m[kG][NACC];   // by chain: M*_u (same-bucket blocking with several buckets)
    int32_t bucket[kG][NACC];
    uint32_t msort[NACC][kG]; // by priority rank: M*_u of the users of u (0 for the others)
    uint32_t ssort[NACC][kG]; // by priority rank: S*_u of the users of u (capped at 2^27 - 1)
    uint32_t inv[kG];       // by chain priority value: the chain of that priority
    uint32_t exm[kG];       // by executor priority value: the chains of that executor priority
    int64_t c0, sys, seg_base;
    int32_t cand;
};

// accelerator of segment q (validated: 0 .. PAAM_MAX_ACC - 1; the launch covers the largest)
template <int NACC>
__device__ __forceinline__ int acc_of(const BatchDev &b, int64_t q)
{
    const int u = b.acc[q];
    return u < NACC ? u : NACC - 1;
}

// ceil(t / T) + 1 (Lemma 1) times c, capped at 2^27 - 1 so that 16 lanes' sum fits 32 bits
__device__ __forceinline__ uint32_t cterm(uint32_t mu, uint32_t c)
{
    const uint64_t v = (uint64_t)mu * c;
    return v < kNarrow - 1 ? (uint32_t)v : kNarrow - 1;
}

template <int NACC>
__device__ void lazy_acc_system(const BatchDev &b, const AnalysisParams &p, int64_t item, LazyAccSmem<NACC> &s,
                                int lane, unsigned gm, int64_t *__restrict__ R_out, uint8_t *__restrict__ st_out,
                                uint8_t *__restrict__ verdict, int32_t *wide_list, int32_t *wide_count)
{
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int pruned = __shfl_sync(gm, cand_pruned(p, sys, cand) ? 1 : 0, 0, kG);
        if (pruned) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    if (n > kG) {
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;
    const int j = lane;
    const Mask jbit = 1u << j;

    // ---- per-chain aggregates (Sec. II-C), per accelerator ------------------
    uint32_t tm2 = 0, mg = 0, lg = 0, Dv = 0, Ev = 0, Emx = 0, dlt = 0, seg0 = 0;
    uint32_t Sa[NACC], Ma[NACC], Amn[NACC], dla[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) Sa[u] = Ma[u] = Amn[u] = dla[u] = 0;
    int32_t pr = INT32_MIN, ep = INT32_MIN, ex = -1 - j, co = -1 - j;
    bool sp = false;
    unsigned fit = 1, rank_ok = 1;
    Mask rbit = 0;
    const bool val = j < n;
    if (val) {
        const int64_t g = c0 + j;
        const int64_t T = b.T[g], D = b.D[g];
        ex = b.exec[g];
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[j];
            rank_ok = (r >= 0 && r < n) ? 1u : 0u;
            rbit = rank_ok ? 1u << r : 0u;
            pr = n - 1 - r;
        } else {
            pr = b.prio[g];
        }
        co = b.exec_core[x0 + ex];
        if (xprio) ep = xprio[x0 + ex];
        sp = b.spin[g] != 0;
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        // sums and extremes in 32 bits over values capped at 2^30 (a capped value
        // takes its chain's sum to the 32-bit bound, and the system to the int64 kernel)
        const int64_t *Ep = b.E + cb0;
        const int ncb = (int)(cb1 - cb0);
        uint32_t E = 0, Emax = 0;
#pragma unroll 4
        for (int i = 0; i < ncb; ++i) {
            const uint32_t e = (uint64_t)Ep[i] < kFitR ? (uint32_t)Ep[i] : (uint32_t)kFitR;
            E = umin(E + e, (uint32_t)kFitR);
            Emax = umax(Emax, e);
        }
        const int nq = (int)(q1 - q0);
        const uint32_t k2c = kappa2 < kFitR ? (uint32_t)kappa2 : (uint32_t)kFitR;
        uint32_t Amin[NACC];
#pragma unroll
        for (int u = 0; u < NACC; ++u) Amin[u] = 0xFFFFFFFFu;
        for (int i = 0; i < nq; ++i) {
            const int64_t q = q0 + i;
            const uint32_t a = ((uint64_t)b.A[q] < kFitR ? (uint32_t)b.A[q] : (uint32_t)kFitR) + k2c; // A* = A + 2 kappa
            const int uq = acc_of<NACC>(b, q);
#pragma unroll
            for (int u = 0; u < NACC; ++u)
                if (u == uq) {
                    Sa[u] = umin(Sa[u] + a, (uint32_t)kFitR);
                    Ma[u] = umax(Ma[u], a);
                    Amin[u] = umin(Amin[u], a);
                    dla[u] += 1;
                }
        }
        uint32_t Stot = 0;
#pragma unroll
        for (int u = 0; u < NACC; ++u) Stot = umin(Stot + Sa[u], (uint32_t)kFitR);
        const uint64_t dl = (uint64_t)nq;
        fit = ((uint64_t)T < kFitR && (uint64_t)D < kFitR && E < kFitR && Stot < kFitR && dl < kFitR &&
               (eps == 0 || dl <= (kFitR - 1) / eps))
                  ? 1u
                  : 0u;
        if (fit) rdivisor((uint32_t)T, tm2, mg, lg);
        Dv = (uint32_t)D;
        Ev = E;
        Emx = Emax;
        dlt = (uint32_t)dl;
        seg0 = (uint32_t)(q0 - seg_base);
#pragma unroll
        for (int u = 0; u < NACC; ++u) Amn[u] = dla[u] ? (Amin[u] < kFitR ? Amin[u] : 0u) : 0u;
    }
    if (lane == 0) {
        s.c0 = c0;
        s.sys = sys;
        s.seg_base = seg_base;
        s.cand = cand;
    }
    const unsigned sh = threadIdx.x & 16u; // the group's first lane in the warp
    Mask users[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) users[u] = __ballot_sync(gm, val && dla[u] != 0) >> sh;
    const Mask spins = __ballot_sync(gm, sp) >> sh;
    const Mask all = (1u << n) - 1u; // n <= 16
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
    if (dmax >= kNarrow - kG) { // inside it but not narrow: the int64 kernel
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    // The system's iteration bound (as in analyze_lazy.cu): no recurrence of Eq. 3 or
    // Eq. 6 takes more than L = sum_h ceil(Dmax / T_h) + 2 evaluations; with L within
    // kIterCap the loops run without counters, otherwise every loop stops at kIterCap.
    const uint32_t L = __reduce_add_sync(gm, val ? umin(rarrivals(dmax, tm2, mg, lg) - 1u, kIterCap + 1u) : 0u) + 2u;
    const bool counted = L > kIterCap;

    // ---- relations (Lemma 4, Theorem 1, Eq. 3), analysis order ---------------
    const unsigned xm = __match_any_sync(gm, ex); // lanes of the same executor (unique keys past n)
    const Mask samex = xm >> sh;
    const Mask corem = __match_any_sync(gm, co) >> sh;
    if (!xprio) ep = __reduce_max_sync(xm, pr); // criticality-as-priority: highest chain priority on the executor
    const bool one_bucket = p.n_buckets == 1;
    const Mask eqx = __match_any_sync(gm, ep) >> sh; // equal executor priority
    Mask higher = 0, ehigher = 0;
    if (__reduce_and_sync(gm, (!val || ((uint32_t)pr < (uint32_t)kG && (uint32_t)ep < (uint32_t)kG)) ? 1u : 0u)) {
        // priorities below 16: each chain's bit in the slot of its priority value, the
        // set above a value the OR of the slots past it (a suffix scan)
        s.inv[j] = 0u;
        s.exm[j] = 0u;
        __syncwarp(gm);
        if (val) {
            s.inv[pr] = jbit;
            s.exm[ep] = eqx;
        }
        __syncwarp(gm);
        uint32_t a = s.inv[j], e = s.exm[j];
#pragma unroll
        for (int d = 1; d < kG; d <<= 1) {
            const uint32_t aw = __shfl_down_sync(gm, a, d, kG), ew = __shfl_down_sync(gm, e, d, kG);
            if (j + d < kG) {
                a |= aw;
                e |= ew;
            }
        }
        a = __shfl_down_sync(gm, a, 1, kG);
        e = __shfl_down_sync(gm, e, 1, kG);
        if (j + 1 >= kG) a = e = 0u;
        higher = __shfl_sync(gm, a, val ? pr : 0, kG);
        ehigher = __shfl_sync(gm, e, val ? ep : 0, kG);
        if (!val) higher = ehigher = all;
    } else { // one comparison each per chain
#pragma unroll
        for (int t = 0; t < kG; ++t) {
            const int32_t pt = __shfl_sync(gm, pr, t, kG), et = __shfl_sync(gm, ep, t, kG);
            higher |= (t < n && pt > pr) ? 1u << t : 0u;
            ehigher |= (t < n && et > ep) ? 1u << t : 0u;
        }
    }
    // position in the analysis order: executor priority, then chain priority
    const int pos = __popc(ehigher) + __popc(eqx & higher & all);
    const Mask hp = samex & higher;            // hp(c), Lemma 4
    const Mask hpp = corem & ~samex & ehigher; // hpp(c), Theorem 1
    s.emax[j] = Emx;
    const int prank = __popc(higher); // rank by chain priority, 0 = highest
#pragma unroll
    for (int u = 0; u < NACC; ++u) {
        const bool user = (users[u] >> j) & 1;
        s.m[j][u] = Ma[u];
        if (val) {
            s.ssort[u][prank] = user ? umin(Sa[u], kNarrow - 1) : 0u;
            s.msort[u][prank] = user ? Ma[u] : 0u;
        }
    }
    uint32_t Bv = 0;
    uint32_t blk[NACC], sums[NACC];
    __syncwarp(gm);
    for (Mask lo = samex & ~higher & ~jbit & all; lo; lo &= lo - 1) // Lemma 4: one LP callback on the executor
        Bv = umax(Bv, s.emax[__ffs(lo) - 1]);
#pragma unroll
    for (int u = 0; u < NACC; ++u) {
        const bool user = (users[u] >> j) & 1;
        // sum_h S*_{h,u} over hps_u(c): a prefix sum in priority order, saturating at 2^27
        uint32_t v = j < n ? s.ssort[u][j] : 0u;
#pragma unroll
        for (int d = 1; d < kG; d <<= 1) {
            const uint32_t w = __shfl_up_sync(gm, v, d, kG);
            if (j >= d) v = umin(v + w, kNarrow);
        }
        v = __shfl_up_sync(gm, v, 1, kG);
        if (j == 0) v = 0u;
        sums[u] = __shfl_sync(gm, v, prank < kG ? prank : 0, kG);
        blk[u] = 0;
        if (one_bucket) { // every user of u shares its bucket: the longest lower-priority request
            uint32_t x = j < n ? s.msort[u][j] : 0u;
#pragma unroll
            for (int d = 1; d < kG; d <<= 1) {
                const uint32_t w = __shfl_down_sync(gm, x, d, kG);
                if (j + d < kG) x = umax(x, w);
            }
            uint32_t below = __shfl_down_sync(gm, x, 1, kG);
            if (j + 1 >= kG) below = 0u;
            below = __shfl_sync(gm, below, prank < kG ? prank : 0, kG);
            if (user) blk[u] = below;
        }
    }
    if (!one_bucket) { // bucket = floor(rank * n_buckets / |U_u|), rank among the users of u (R2)
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const bool user = (users[u] >> j) & 1;
            s.bucket[j][u] = user ? (int32_t)((uint32_t)__popc(users[u] & higher) * (uint32_t)p.n_buckets /
                                              (uint32_t)__popc(users[u]))
                                  : -1;
        }
        __syncwarp(gm);
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const bool user = (users[u] >> j) & 1;
            const int32_t bk = s.bucket[j][u];
            if (user)
                for (Mask lo = users[u] & ~higher & ~jbit; lo; lo &= lo - 1) {
                    const int l = __ffs(lo) - 1;
                    if (s.bucket[l][u] == bk) blk[u] = umax(blk[u], s.m[l][u]);
                }
        }
    }

    // ---- own recurrence terms ------------------------------------------------
    if (val) {
        const uint64_t cap = (uint64_t)Dv + 1; // values above D act the same as D + 1
        const Mask needs = hp | (hpp & spins);
        s.rel[pos] = make_uint4(hp, hpp, needs, seg0);
        s.chain[pos] = (uint32_t)j;
        s.needs[j] = needs;
        s.rec[pos] = make_uint4(Dv, Bv + Ev, (uint32_t)((uint64_t)dlt * eps), dlt);
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const uint64_t own = (uint64_t)Sa[u] + (uint64_t)dla[u] * blk[u];
            // Lemma 2's sum over the segments on u is at least own_u + lb_u, lb_u =
            // f delta_u sum_h S*_{h,u} (f = 2 if A*_u + blk_u >= 1)
            const uint64_t lb = (((uint64_t)Amn[u] + blk[u]) >= 1 ? 2 : 1) * (uint64_t)dla[u] * sums[u];
            s.acc[pos][u] = make_uint4((uint32_t)(own < cap ? own : cap), lb < kNarrow ? (uint32_t)lb : kNarrow,
                                       blk[u], dla[u]);
            s.hps[pos][u] = users[u] & higher;
        }
    }
    __syncwarp(gm);

    // ---- Theorem 1 (Eq. 6), chain by chain -----------------------------------
    uint32_t Ehp = Ev, Ehpp = Ev + (sp ? 0u : (uint32_t)((uint64_t)dlt * eps)), Rv = 0;
    Mask sched = 0;
    const uint32_t k2 = (uint32_t)kappa2;
    auto chains = [&](auto counted_tag) {
    constexpr bool CNT = decltype(counted_tag)::value;
    for (int step = 0; step < n; ++step) {
        const uint4 rl = s.rel[step];
        if (rl.z & ~sched) { // a needed H*_h is not available (the chain is DEP)
            if (rank_row) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        const uint4 rc = s.rec[step];
        const int ch = (int)s.chain[step];
        const uint32_t D32 = rc.x, base = rc.y, deps = rc.z, dl = rc.w;
        const uint32_t ccoef = ((rl.x >> j) & 1) ? Ehp : (((rl.y >> j) & 1) ? Ehpp : 0u);
        uint32_t acoef[NACC], own[NACC], lb[NACC], Hs[NACC];
        uint32_t h0 = 0, uses = 0; // uses: the accelerators of the chain's segments
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const uint4 ar = s.acc[step][u];
            own[u] = ar.x;
            lb[u] = ar.w ? ar.y : kInfR; // kInfR: u unused by the chain, or its fixed points taken
            acoef[u] = ((s.hps[step][u] >> j) & 1) ? Sa[u] : 0u;
            Hs[u] = kInfR;
            uses |= ar.w ? 1u << u : 0u;
            if (ar.w) h0 += own[u]; // Lemma 2's sum on u is never below own_u
        }
        // start: B + E + H* with the interference parts of Eq. 4 empty
        uint32_t R = base + (dl ? umin(h0, kNarrow) + deps : 0u);
        uint32_t hs = 0, ev = 0;
        bool ok = false, capped = false;
        if (R <= D32) {
            for (;;) { // until no accelerator's fixed points are newly needed
                int need = -1;
                for (;;) {
                    if (CNT && ev++ == kIterCap) break;
                    const uint32_t mu = rarrivals(R, tm2, mg, lg);
                    const uint32_t cs = __reduce_add_sync(gm, cterm(mu, ccoef));
                    hs = 0;
#pragma unroll
                    for (int u = 0; u < NACC; ++u) {
                        if (!((uses >> u) & 1)) continue; // the same in every lane of the group
                        const uint32_t as = umin(__reduce_add_sync(gm, cterm(mu, acoef[u])), kNarrow);
                        if (as > lb[u] && need < 0) need = u;
                        hs += umin(Hs[u], own[u] + as); // min(Eq. 3, Eq. 4) on u, summed (R1)
                    }
                    if (need >= 0) { // this evaluation is taken again once that sum is known
                        if (CNT) --ev;
                        break;
                    }
                    if (dl) hs = umin(hs, kNarrow) + deps; // Eq. 1
                    const uint32_t Rn = base + umin(hs, kNarrow) + umin(cs, kNarrow);
                    if (Rn == R) {
                        ok = true;
                        break;
                    }
                    R = Rn;
                    if (R > D32) break;
                }
                if (need < 0) break;
                // Lemma 2 over the chain's segments on accelerator `need`: the sum matters
                // only below Eq. 4 at R = D on it (and below D + 1)
#pragma unroll
                for (int u = 0; u < NACC; ++u) {
                    if (u != need) continue;
                    lb[u] = kInfR;
                    const uint32_t mud = rarrivals(D32, tm2, mg, lg);
                    const uint32_t hchd = umin(__reduce_add_sync(gm, cterm(mud, acoef[u])), kNarrow);
                    const uint32_t lim = umin(own[u] + hchd, D32 + 1);
                    const uint32_t blkc = s.acc[step][u].z;
                    const int64_t qb = s.seg_base + s.rel[step].w;
                    uint32_t H32 = 0;
                    bool inf = false;
                    for (uint32_t q = 0; q < dl && !inf; ++q) {
                        if (acc_of<NACC>(b, qb + q) != u) continue; // the chain's segments on u
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
                            const uint32_t muh = rarrivals(h, tm2, mg, lg);
                            const uint32_t nh = hb + umin(__reduce_add_sync(gm, cterm(muh, acoef[u])), kNarrow);
                            if (nh == h) break; // strictly increasing until here, bounded by D
                            h = nh;
                        }
                        H32 += h;
                    }
                    if (!inf) Hs[u] = H32;
                }
                if (capped) break; // a segment recurrence was cut short
            }
        }
        if (capped) { // no bound (PAAM_ST_ITERCAP)
            if (j == ch) Rv = kCapR;
            if (rank_row) break;
            continue;
        }
        if (ok) {
            sched |= 1u << ch;
            if (j == ch) {
                Rv = R;
                Ehp = Ev + hs;
                if (sp) Ehpp = Ev + hs;
            }
        } else {
            if (ev > kIterCap && j == ch) Rv = kCapR; // the recurrence was cut short (PAAM_ST_ITERCAP)
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
                const bool okc = sched == all;
                if (p.cand_ok) p.cand_ok[syss * p.Kc + cand_of(p, syss, cands)] = okc ? 1 : 0;
                if (okc) atomicMin(p.first_ok + syss, cands);
            }
            __syncwarp(gm);
            return;
        }
        if (val) {
            const bool okc = (sched >> j) & 1;
            R_out[c0s + j] = okc ? (int64_t)Rv : -1;
            // DEP: skipped at its step, i.e. some chain of its DEP-rule set (all earlier in
            // the analysis order) is not schedulable
            st_out[c0s + j] = okc ? PAAM_ST_SCHED
                                  : (Rv == kCapR ? PAAM_ST_ITERCAP
                                                 : ((s.needs[j] & ~sched) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
        }
        if (lane == 0 && verdict) verdict[syss] = sched == all ? 1 : 0;
    }
    __syncwarp(gm);
}

// four resident blocks of 256 per SM (64 registers, no spills) for up to three
// accelerators, two for four
template <int NACC>
__global__ void __launch_bounds__(256, NACC <= 3 ? 4 : 2) analyze_lazy_acc_kernel(BatchDev b, AnalysisParams p,
                                                                                int64_t *R, uint8_t *st,
                                                                                uint8_t *verdict, int32_t *wide_list,
                                                                                int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / kG;
    const int grp = threadIdx.x / kG;
    const int lane = threadIdx.x % kG;
    LazyAccSmem<NACC> &s = reinterpret_cast<LazyAccSmem<NACC> *>(smem_raw)[grp];
    const unsigned gm = rgroup_mask<kG>();
    const int64_t n_items = p.K > 0 ? b.n_sys * p.K : b.n_sys;
    for_each_item<kG>(p, n_items, grp, groups, lane, gm, [&](int64_t i) {
        lazy_acc_system<NACC>(b, p, i, s, lane, gm, R, st, verdict, wide_list, wide_count);
    });
}

template <int NACC>
int launch_lazy_acc_n(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                      int64_t max_items, cudaStream_t stream)
{
    constexpr int threads = 256;
    const int groups = threads / kG;
    const size_t smem = sizeof(LazyAccSmem<NACC>) * groups;
    auto kern = analyze_lazy_acc_kernel<NACC>;
    PAAM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PAAM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (max_items + groups - 1) / groups;
    const int64_t cap = (int64_t)per_sm * bt->ctx->n_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(batch_dev(bt), p, R, st, verdict, bt->list_wide, bt->counts + 1);
    PAAM_CUDA_TRY(cudaGetLastError());
    return PAAM_OK;
}

} // namespace

int paam_launch_lazy_acc(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                         int64_t max_items, cudaStream_t stream)
{
    const unsigned long long used = bt->stats[ST_ACCMAX] + 1;
    static_assert(PAAM_MAX_ACC == 4, "instantiations below cover 2..4 accelerators");
    if (used >= 4) return launch_lazy_acc_n<4>(bt, p, R, st, verdict, max_items, stream);
    if (used == 3) return launch_lazy_acc_n<3>(bt, p, R, st, verdict, max_items, stream);
    return launch_lazy_acc_n<2>(bt, p, R, st, verdict, max_items, stream);
}
