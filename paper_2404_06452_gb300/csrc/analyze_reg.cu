// analyze_reg.cu -- register-resident variant of the fast analysis path.
//
// Same mathematics and the same 32-bit bound as analyze_fast.cu (see there):
// arrival counts ceil(t / T) + 1 of Lemma 1 by exact multiply-shift division,
// interferer sets as bitmasks, the exact skip of Lemma 2's per-segment sum
// when it cannot beat Eq. 4 at R = D, and the chain recurrences of Theorem 1
// in an order where every needed H*_h is final.
//
// Layout: a group of G lanes owns one system and each lane owns CPL of its
// chains (chain j lives in lane j % G, slot j / G), held in registers.  Chain
// relations (hp, hpp, hps, lower-priority same-executor, bucket rank, order)
// come from O(n) broadcasts of each chain's keys.  Fixed points iterate with
// every lane adding the terms of its own chains for the chain under analysis;
// the group combines them with shuffles.  Shared memory only holds each
// chain's own recurrence terms, read by the whole group as broadcasts.
#include "reg_common.cuh"

namespace {
using namespace paam_reg;

template <int NMAX>
struct OwnSmem {
    using Mask = typename RegMask<NMAX>::type;
    // each chain's keys, read by the whole group as broadcasts in the relations pass
    int4 key[NMAX];   // {chain priority, executor, core, executor priority}
    uint4 dv[NMAX];   // {Emax, 2 (T - 1), magic, l}: the divisor T (rdivisor)
    uint2 sm[NMAX];   // {S*, M*}
    Mask hp[NMAX], hpp[NMAX], hps[NMAX];
    uint4 rec[NMAX];  // {D, base = B + E, own = S* + delta blk (capped at D + 1), deps = delta eps}
    uint4 seg[NMAX];  // {Hseg, limit, blk, delta}
    uint32_t seg0[NMAX];
    uint8_t order[NMAX];
};


template <int G, int CPL>
__device__ void reg_system(const BatchDev &b, const AnalysisParams &p, int64_t item, OwnSmem<G * CPL> &s, int lane, unsigned gm, int64_t *__restrict__ R_out,
                           uint8_t *__restrict__ st_out,
                           uint8_t *__restrict__ verdict, int32_t *big_list, int32_t *big_count,
                           int32_t *wide_list, int32_t *wide_count)
{
    constexpr int NMAX = G * CPL;
    using Mask = typename RegMask<NMAX>::type;
    int64_t sys;
    int32_t cand;
    item_of(p, item, sys, cand);
    if (p.K > 0 && p.early) { // candidate above the best schedulable one found so far
        const int pruned = __shfl_sync(gm, cand_pruned(p, sys, cand) ? 1 : 0, 0, G);
        if (pruned) return;
    }
    const int64_t c0 = b.sys_chain_off[sys];
    const int n = (int)(b.sys_chain_off[sys + 1] - c0);
    if (n < p.min_chains) return; // an earlier pass over the same list took it
    if (n > NMAX) {
        if (lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;

    // ---- per-chain aggregates (Sec. II-C), one chain per slot ---------------
    uint32_t tm2[CPL], mg[CPL], lg[CPL], Dv[CPL], Ev[CPL], Sv[CPL], Emx[CPL], Mv[CPL], Amn[CPL], dlv[CPL];
    uint32_t seg0[CPL];
    int32_t pr[CPL], ep[CPL], ex[CPL], co[CPL];
    bool sp[CPL], val[CPL];
    Mask users = 0, spins = 0, rbits = 0;
    unsigned fits = 1, rank_ok = 1;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int j = lane + G * k;
        val[k] = j < n;
        tm2[k] = mg[k] = lg[k] = Dv[k] = Ev[k] = Sv[k] = Emx[k] = Mv[k] = Amn[k] = dlv[k] = seg0[k] = 0;
        pr[k] = ep[k] = INT32_MIN;
        ex[k] = co[k] = -1 - j;
        sp[k] = false;
        if (!val[k]) continue;
        const int64_t g = c0 + j;
        const int64_t T = b.T[g], D = b.D[g];
        const int x = b.exec[g];
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[j];
            rank_ok &= (r >= 0 && r < n) ? 1u : 0u;
            rbits |= (r >= 0 && r < n) ? (Mask)1 << r : 0;
            pr[k] = n - 1 - r;
        } else {
            pr[k] = b.prio[g];
        }
        ex[k] = x;
        co[k] = b.exec_core[x0 + x];
        ep[k] = xprio ? xprio[x0 + x] : INT32_MIN;
        sp[k] = b.spin[g] != 0;
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        uint64_t E = 0, Emax = 0, S = 0, M = 0, Amin = ~0ull;
#pragma unroll 4
        for (int64_t cb = cb0; cb < cb1; ++cb) {
            const uint64_t e = (uint64_t)b.E[cb];
            E += e;
            Emax = e > Emax ? e : Emax;
        }
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
#pragma unroll 4
        for (int64_t q = q0; q < q1; ++q) {
            const uint64_t a = (uint64_t)b.A[q] + kappa2; // A* = A + 2 kappa
            S += a;
            M = a > M ? a : M;
            Amin = a < Amin ? a : Amin;
        }
        const uint64_t dl = (uint64_t)(q1 - q0);
        const bool fit = (uint64_t)T < kFitR && (uint64_t)D < kFitR && E < kFitR && S < kFitR && dl < kFitR &&
                         (eps == 0 || dl <= (kFitR - 1) / eps);
        fits &= fit ? 1u : 0u;
        if (fit) rdivisor((uint32_t)T, tm2[k], mg[k], lg[k]);
        Dv[k] = (uint32_t)D;
        Ev[k] = (uint32_t)E;
        Sv[k] = (uint32_t)S;
        Emx[k] = (uint32_t)Emax;
        Mv[k] = (uint32_t)M;
        Amn[k] = dl ? (uint32_t)(Amin < kFitR ? Amin : 0) : 0;
        dlv[k] = (uint32_t)dl;
        seg0[k] = (uint32_t)(q0 - seg_base);
        users |= dl ? (Mask)1 << j : 0;
        spins |= sp[k] ? (Mask)1 << j : 0;
    }
    fits = rand_<G>(fits, gm);
    users = ror<G>(users, gm);
    spins = ror<G>(spins, gm);
    const Mask all = n >= (int)(8 * sizeof(Mask)) ? ~(Mask)0 : (((Mask)1 << n) - 1);
    if (rank_row) { // a candidate must be a permutation of 0..n-1
        rank_ok = rand_<G>(rank_ok, gm);
        rbits = ror<G>(rbits, gm);
        if (!rank_ok || rbits != all) {
            if (lane == 0) {
                atomicExch(p.err, PAAM_E_INVAL);
                if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = 0;
            }
            return;
        }
    }
    uint32_t dmax = 0;
#pragma unroll
    for (int k = 0; k < CPL; ++k) dmax = Dv[k] > dmax ? Dv[k] : dmax;
    const uint32_t dsys = rmax<G>(dmax, gm);
    const bool narrow = dsys < kNarrow - G * CPL;
    if (!fits) {
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    // The system's iteration bound (see the header of paam_rta_load_systems): no
    // recurrence of Eq. 3 or Eq. 6 takes more than L = sum_h ceil(Dmax / T_h) + 2
    // evaluations.  With L within kIterCap (always, for a validated batch) the loops
    // run without counters; otherwise every loop stops at kIterCap (PAAM_ST_ITERCAP).
    uint32_t lpart = 0;
#pragma unroll
    for (int k = 0; k < CPL; ++k)
        if (val[k]) lpart += rarrivals(dsys, tm2[k], mg[k], lg[k]) - 1u;
    const bool counted = __reduce_add_sync(gm, umin(lpart, kIterCap + 1u)) + 2u > kIterCap;
    if (!xprio) { // criticality-as-priority: highest chain priority on the executor
        int32_t best[CPL];
#pragma unroll
        for (int k = 0; k < CPL; ++k) best[k] = INT32_MIN;
        for (int t = 0; t < n; ++t) {
            const int32_t pt = bcast<G, CPL>(pr, t, gm), xt = bcast<G, CPL>(ex, t, gm);
#pragma unroll
            for (int k = 0; k < CPL; ++k)
                if (xt == ex[k] && pt > best[k]) best[k] = pt;
        }
#pragma unroll
        for (int k = 0; k < CPL; ++k) ep[k] = best[k];
    }

    // ---- relations, analysis order, CPU blocking (Lemma 4), and the sums of
    // the Lemma 2 skip test over hps; with one bucket (every user shares it)
    // also the same-bucket blocking of R2-R3
    Mask higher[CPL], samex[CPL], hppm[CPL];
    int pos[CPL], rank[CPL];
    uint32_t Bv[CPL], blk[CPL];
    uint64_t hchd[CPL], sums[CPL];
    const bool one_bucket = p.n_buckets == 1;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        higher[k] = samex[k] = hppm[k] = 0;
        pos[k] = rank[k] = 0;
        Bv[k] = blk[k] = 0;
        hchd[k] = sums[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        if (!val[k]) continue;
        const int j = lane + G * k;
        s.key[j] = make_int4(pr[k], ex[k], co[k], ep[k]);
        s.dv[j] = make_uint4(Emx[k], tm2[k], mg[k], lg[k]);
        s.sm[j] = make_uint2(Sv[k], Mv[k]);
    }
    __syncwarp(gm);
    for (int t = 0; t < n; ++t) {
        const int4 kt4 = s.key[t];
        const uint4 dv4 = s.dv[t];
        const uint2 sm2 = s.sm[t];
        const int32_t pt = kt4.x, xt = kt4.y, kt = kt4.z, et = kt4.w;
        const uint32_t emt = dv4.x, tmt = dv4.y, mgt = dv4.z, lgt = dv4.w;
        const uint32_t st = sm2.x, mt = sm2.y;
        const bool ut = (users >> t) & 1;
        const Mask bit = (Mask)1 << t;
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const bool hi = pt > pr[k];
            const bool sx = xt == ex[k];
            higher[k] |= hi ? bit : 0;
            samex[k] |= sx ? bit : 0;
            hppm[k] |= (!sx && kt == co[k] && et > ep[k]) ? bit : 0; // hpp, Lemma 4
            pos[k] += (et > ep[k]) || (et == ep[k] && hi);           // executor, then chain priority
            if (sx && pt < pr[k] && emt > Bv[k]) Bv[k] = emt; // one LP callback on the executor
            const bool act = dlv[k] != 0 && ut;               // c and t both use the accelerator
            const uint32_t sv = (act && hi) ? st : 0u;
            hchd[k] += (uint64_t)rarrivals(Dv[k], tmt, mgt, lgt) * sv;
            sums[k] += sv;
            if (one_bucket && act && pt < pr[k] && mt > blk[k]) blk[k] = mt;
        }
    }
    const int n_users = rpopc(users);
#pragma unroll
    for (int k = 0; k < CPL; ++k) rank[k] = rpopc(higher[k] & users); // users of higher priority
    int32_t bucket[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) // bucket = floor(rank * n_buckets / |U|) (R2)
        bucket[k] = (val[k] && dlv[k]) ? (int32_t)((uint32_t)rank[k] * (uint32_t)p.n_buckets / (uint32_t)n_users)
                                       : -1;

    // ---- same-bucket blocking (R2-R3) with several buckets ------------------
    if (!one_bucket) {
        for (int t = 0; t < n; ++t) {
            const uint32_t mt = bcast<G, CPL>(Mv, t, gm);
            const int32_t bt = bcast<G, CPL>(bucket, t, gm);
            const bool ut = (users >> t) & 1;
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const bool act = bucket[k] >= 0 && ut;
                const bool hi = (higher[k] >> t) & 1;
                const bool same = act && !hi && t != lane + G * k && bt == bucket[k];
                blk[k] = (same && mt > blk[k]) ? mt : blk[k];
            }
        }
    }

    // ---- own recurrence terms to shared memory ------------------------------
    Mask need_exact = 0;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        if (!val[k]) continue;
        const int j = lane + G * k;
        const uint64_t dl = dlv[k];
        const uint64_t own = (uint64_t)Sv[k] + dl * blk[k];
        const uint64_t cap = (uint64_t)Dv[k] + 1; // values above D act the same as D + 1
        s.hp[j] = higher[k] & samex[k];
        s.hpp[j] = hppm[k];
        s.hps[j] = higher[k] & users;
        s.rec[j] = make_uint4(Dv[k], Bv[k] + Ev[k], (uint32_t)(own < cap ? own : cap), (uint32_t)(dl * eps));
        const uint64_t lim = own + hchd[k];
        s.seg[j] = make_uint4(kInfR, (uint32_t)(lim < cap ? lim : cap), blk[k], (uint32_t)dl);
        s.seg0[j] = seg0[k];
        s.order[pos[k]] = (uint8_t)j;
        // Lemma 2's sum is at least sum_j (x_j + f sum_h S_h), x_j = A*_j + blk, f = 2 if x_j >= 1;
        // Eq. 4 is at most own + sum_h mu_h(D) S_h for every R <= D.  Exact sum only if it can win.
        const uint64_t f = ((uint64_t)Amn[k] + blk[k]) >= 1 ? 2 : 1;
        if (dl && f * dl * sums[k] < hchd[k]) need_exact |= (Mask)1 << j;
    }
    need_exact = ror<G>(need_exact, gm);
    __syncwarp(gm);

    uint32_t Ehp[CPL], Ehpp[CPL], Rv[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        Ehp[k] = Ev[k];
        Ehpp[k] = Ev[k] + (sp[k] ? 0u : (uint32_t)((uint64_t)dlv[k] * eps));
        Rv[k] = 0;
    }
    Mask sched = 0, dep = 0;
    // the fixed points: counted loops only where the bound above exceeds kIterCap
    auto fixed_points = [&](auto counted_tag) {
    constexpr bool CNT = decltype(counted_tag)::value;

    // ---- exact per-segment fixed points (Lemma 2), chains one at a time ------
    for (Mask nm = need_exact; nm; nm &= nm - 1) {
        const int c = rlowest(nm);
        const Mask hps = s.hps[c];
        const uint4 sg = s.seg[c];
        const uint32_t Dc = s.rec[c].x, lim = sg.y, blkc = sg.z, dl = sg.w;
        uint32_t acoef[CPL];
#pragma unroll
        for (int k = 0; k < CPL; ++k) acoef[k] = ((hps >> (lane + G * k)) & 1) ? Sv[k] : 0u;
        uint64_t Hsum = 0;
        bool inf = false;
        uint32_t ev = 0; // evaluations of the current segment's recurrence
        if (narrow) {
            // 32 bits hold every value: base below 2^31, h <= D below 2^27, the
            // group sum capped at 2^27 (a capped sum exceeds D as the true one would)
            uint32_t H32 = 0;
            const uint32_t k2 = (uint32_t)kappa2;
            for (uint32_t q = 0; q < dl && !inf; ++q) {
                const uint32_t base = (uint32_t)b.A[seg_base + s.seg0[c] + q] + k2 + blkc;
                uint32_t h = base;
                ev = 0;
                for (;;) {
                    if (h > Dc || H32 + h >= lim) {
                        inf = true;
                        break;
                    }
                    if (CNT && ev++ == kIterCap) {
                        inf = true;
                        break;
                    }
                    uint64_t part = 0;
#pragma unroll
                    for (int k = 0; k < CPL; ++k) part += (uint64_t)rarrivals(h, tm2[k], mg[k], lg[k]) * acoef[k];
                    const uint32_t nh =
                        base + umin(__reduce_add_sync(gm, part < kNarrow - 1 ? (uint32_t)part : kNarrow - 1), kNarrow);
                    if (nh == h) break;
                    h = nh;
                }
                H32 += h;
            }
            Hsum = H32;
        } else {
            for (uint32_t q = 0; q < dl && !inf; ++q) {
                const uint64_t base = (uint64_t)b.A[seg_base + s.seg0[c] + q] + kappa2 + blkc;
                uint64_t h = base; // the recurrence starts with the first two terms
                ev = 0;
                for (;;) {
                    if (h > Dc || Hsum + h >= lim) {
                        inf = true;
                        break;
                    }
                    if (CNT && ev++ == kIterCap) {
                        inf = true;
                        break;
                    }
                    uint64_t part = 0;
#pragma unroll
                    for (int k = 0; k < CPL; ++k)
                        part += (uint64_t)rarrivals((uint32_t)h, tm2[k], mg[k], lg[k]) * acoef[k];
                    const uint64_t nh = base + gsum<G>(part, narrow, gm);
                    if (nh == h) break; // strictly increasing until here, bounded by D
                    h = nh;
                }
                Hsum += h;
            }
        }
        if (lane == 0 && (!inf || (CNT && ev > kIterCap))) s.seg[c].x = CNT && ev > kIterCap ? kCapR : (uint32_t)Hsum;
        __syncwarp(gm);
    }

    // ---- Theorem 1 (Eq. 6), chain by chain ----------------------------------
    for (int step = 0; step < n; ++step) {
        const int c = s.order[step];
        const Mask hp = s.hp[c], hpp = s.hpp[c], hps = s.hps[c];
        const Mask cbit = (Mask)1 << c;
        if ((hp | (hpp & spins)) & ~sched) { // a needed H*_h is not available
            dep |= cbit;
            if (rank_row) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        uint32_t ccoef[CPL], acoef[CPL];
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int j = lane + G * k;
            ccoef[k] = ((hp >> j) & 1) ? Ehp[k] : (((hpp >> j) & 1) ? Ehpp[k] : 0u);
            acoef[k] = ((hps >> j) & 1) ? Sv[k] : 0u;
        }
        const uint4 rc = s.rec[c], sg = s.seg[c];
        if (sg.x == kCapR) { // a segment recurrence was cut short: no bound (PAAM_ST_ITERCAP)
#pragma unroll
            for (int k = 0; k < CPL; ++k)
                if (lane + G * k == c) Rv[k] = kCapR;
            if (rank_row) break;
            continue;
        }
        const uint64_t Dc = rc.x, base = rc.y, own = rc.z, deps = rc.w, dl = sg.w;
        const uint64_t Hseg = sg.x == kInfR ? ~0ull : (uint64_t)sg.x;
        // start: B + E + H* with the interference part of Eq. 4 empty
        uint64_t R = base + (dl ? (Hseg < own ? Hseg : own) + deps : 0);
        uint64_t hs = 0;
        bool ok = false;
        uint32_t ev = 0; // evaluations of the recurrence
        if (narrow) {
            // the same iteration in 32 bits: every deadline is below 2^27 - 64, in
            // the loop base <= R <= D, the group sums are below 2^32, and each sum
            // is capped at 2^27 where it is added (a capped term already exceeds D)
            const uint32_t D32 = rc.x, base32 = rc.y, own32 = rc.z, deps32 = rc.w, Hs32 = sg.x;
            uint32_t R32 = (uint32_t)R, hs32 = 0;
            if (R <= Dc) {
                for (;;) {
                    if (CNT && ev++ == kIterCap) break;
                    uint64_t cpu = 0, acc = 0;
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        const uint64_t mu = rarrivals(R32, tm2[k], mg[k], lg[k]);
                        cpu += mu * ccoef[k];
                        acc += mu * acoef[k];
                    }
                    const uint32_t cs = __reduce_add_sync(gm, cpu < kNarrow - 1 ? (uint32_t)cpu : kNarrow - 1);
                    const uint32_t as = __reduce_add_sync(gm, acc < kNarrow - 1 ? (uint32_t)acc : kNarrow - 1);
                    hs32 = 0;
                    if (dl) {
                        const uint32_t hch = own32 + umin(as, kNarrow); // Eq. 4
                        hs32 = (Hs32 < hch ? Hs32 : hch) + deps32;      // Eq. 1 with min(Eq. 3, Eq. 4)
                    }
                    const uint32_t Rn = base32 + umin(hs32, kNarrow) + umin(cs, kNarrow);
                    if (Rn == R32) {
                        ok = true;
                        break;
                    }
                    R32 = Rn;
                    if (R32 > D32) break;
                }
            }
            R = R32;
            hs = hs32;
        } else {
            while (R <= Dc) {
                if (CNT && ev++ == kIterCap) break;
                uint64_t cpu = 0, acc = 0;
#pragma unroll
                for (int k = 0; k < CPL; ++k) {
                    const uint64_t mu = rarrivals((uint32_t)R, tm2[k], mg[k], lg[k]);
                    cpu += mu * ccoef[k];
                    acc += mu * acoef[k];
                }
                cpu = gsum<G>(cpu, narrow, gm);
                acc = gsum<G>(acc, narrow, gm);
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
                R = Rn;
            }
        }
        if (ok) {
            sched |= cbit;
#pragma unroll
            for (int k = 0; k < CPL; ++k)
                if (lane + G * k == c) {
                    Rv[k] = (uint32_t)R;
                    Ehp[k] = Ev[k] + (uint32_t)hs;
                    if (sp[k]) Ehpp[k] = Ev[k] + (uint32_t)hs;
                }
        } else {
            if (CNT && ev > kIterCap) // the recurrence was cut short (PAAM_ST_ITERCAP)
#pragma unroll
                for (int k = 0; k < CPL; ++k)
                    if (lane + G * k == c) Rv[k] = kCapR;
            if (rank_row) break;
        }
    }
    };
    if (counted)
        fixed_points(std::true_type{});
    else
        fixed_points(std::false_type{});

    // ---- outputs --------------------------------------------------------------
    if (rank_row) {
        if (lane == 0) {
            const bool ok = sched == all;
            if (p.cand_ok) p.cand_ok[sys * p.Kc + cand_of(p, sys, cand)] = ok ? 1 : 0;
            if (ok) atomicMin(p.first_ok + sys, cand);
        }
        __syncwarp(gm);
        return;
    }
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        if (!val[k]) continue;
        const int j = lane + G * k;
        const bool ok = (sched >> j) & 1;
        R_out[c0 + j] = ok ? (int64_t)Rv[k] : -1;
        st_out[c0 + j] = ok ? PAAM_ST_SCHED
                            : (Rv[k] == kCapR ? PAAM_ST_ITERCAP
                                              : (((dep >> j) & 1) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
    }
    if (lane == 0 && verdict) verdict[sys] = sched == all ? 1 : 0;
    __syncwarp(gm);
}

template <int G, int CPL>
__device__ __forceinline__ void reg_items(const BatchDev &b, const AnalysisParams &p, int64_t *R, uint8_t *st,
                                          uint8_t *verdict, const int32_t *list, const int32_t *count,
                                          int32_t *big_list, int32_t *big_count, int32_t *wide_list,
                                          int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    OwnSmem<G * CPL> &s = reinterpret_cast<OwnSmem<G * CPL> *>(smem_raw)[grp];
    const unsigned gm = rgroup_mask<G>();
    const int64_t n_items = list ? (int64_t)*count : (p.K > 0 ? b.n_sys * p.K : b.n_sys);
    for_each_item<G>(p, n_items, grp, groups, lane, gm, [&](int64_t i) {
        const int64_t item = list ? (int64_t)list[i] : i;
        reg_system<G, CPL>(b, p, item, s, lane, gm, R, st, verdict, big_list, big_count, wide_list, wide_count);
    });
}

template <int G, int CPL>
__global__ void __launch_bounds__(256) analyze_reg_kernel(BatchDev b, AnalysisParams p, int64_t *R, uint8_t *st,
                                                          uint8_t *verdict, const int32_t *list,
                                                          const int32_t *count, int32_t *big_list,
                                                          int32_t *big_count, int32_t *wide_list,
                                                          int32_t *wide_count)
{
    reg_items<G, CPL>(b, p, R, st, verdict, list, count, big_list, big_count, wide_list, wide_count);
}

// One chain per lane keeps few values per thread: 64 registers leave room for
// four resident blocks of 256 threads.
template <int G>
__global__ void __launch_bounds__(256, 4) analyze_reg1_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                              uint8_t *st, uint8_t *verdict, const int32_t *list,
                                                              const int32_t *count, int32_t *big_list,
                                                              int32_t *big_count, int32_t *wide_list,
                                                              int32_t *wide_count)
{
    reg_items<G, 1>(b, p, R, st, verdict, list, count, big_list, big_count, wide_list, wide_count);
}

} // namespace

template <int G, int CPL>
int launch_reg(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
               const int32_t *list, const int32_t *count, int64_t max_items, int threads, cudaStream_t stream)
{
    if (threads % 32 != 0 || threads > 256) return PAAM_E_INVAL;
    const int groups = threads / G;
    const size_t smem = sizeof(OwnSmem<G * CPL>) * groups;
    void (*kern)(BatchDev, AnalysisParams, int64_t *, uint8_t *, uint8_t *, const int32_t *, const int32_t *,
                 int32_t *, int32_t *, int32_t *, int32_t *);
    if constexpr (CPL == 1)
        kern = analyze_reg1_kernel<G>;
    else
        kern = analyze_reg_kernel<G, CPL>;
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

// instantiations used by the launch table (analyze_fast.cu)
template int launch_reg<8, 2>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                              const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_reg<16, 1>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                               const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_reg<4, 4>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                              const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_reg<16, 2>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                               const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_reg<32, 1>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                               const int32_t *, const int32_t *, int64_t, int, cudaStream_t);
template int launch_reg<32, 2>(const paam_batch *, const AnalysisParams &, int64_t *, uint8_t *, uint8_t *,
                               const int32_t *, const int32_t *, int64_t, int, cudaStream_t);

namespace {
__global__ void diag_divisor_kernel(const uint32_t *T, uint32_t *m, uint32_t *l, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t tm2, mi, li;
        rdivisor(T[i], tm2, mi, li);
        m[i] = mi;
        l[i] = li;
    }
}
} // namespace

extern "C" int paam_diag_divisor(const uint32_t *T, uint32_t *m, uint32_t *l, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!T || !m || !l))) return PAAM_E_INVAL;
    if (n == 0) return PAAM_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    diag_divisor_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(T, m, l, n);
    PAAM_CUDA_TRY(cudaGetLastError());
    paam_count_launch();
    return PAAM_OK;
}
