// analyze_reg_acc.cu -- register-table analysis of systems whose segments use
// several accelerators (rule R1: one server per accelerator, analysed on its
// own; reading R10): the mathematics of analyze_reg.cu with an accelerator
// dimension on every server-side quantity.
//
// Per accelerator a: its users, their buckets (rank among a's users, Sec.
// IV-C), same-bucket blocking blk_a (R2-R3), the higher-priority users hps_a
// (Eq. 3 and Eq. 4), Lemma 2's per-segment fixed points over the chain's
// segments on a (Eq. 3) and the per-chain bound own_a + sum over hps_a of
// mu(t) S*_{h,a} (Eq. 4).  A chain's handling time is the sum over the
// accelerators it uses of min(Eq. 3 sum, Eq. 4), plus delta eps (Eq. 1); the
// chain recurrence of Theorem 1 (Eq. 6) is otherwise that of one accelerator.
// The exact reformulations of analyze_reg.cu (multiply-shift division, the
// 32-bit bound with capped partial sums, the skip test of Lemma 2 and its abort
// limit) apply per accelerator.  A group of G = 16 lanes owns a system of at
// most 16 chains, one chain per lane; larger systems and systems outside the
// 32-bit bound go to the int64 kernel's list.
#include "reg_common.cuh"

namespace {
using namespace paam_reg;

template <int NMAX, int NACC>
struct AccSmem {
    using Mask = typename RegMask<NMAX>::type;
    int4 key[NMAX];           // {chain priority, executor, core, executor priority}
    uint4 dv[NMAX];           // {Emax, 2 (T - 1), magic, l}: the divisor T (rdivisor)
    uint2 sm[NMAX][NACC];     // {S*_a, M*_a}
    Mask hp[NMAX], hpp[NMAX];
    Mask hps[NMAX][NACC];
    uint4 rec[NMAX];          // {D, base = B + E, deps = delta eps, delta (all segments)}
    uint32_t own[NMAX][NACC]; // S*_a + delta_a blk_a, capped at D + 1
    uint4 seg[NMAX][NACC];    // {Hseg_a, limit_a, blk_a, delta_a}
    uint32_t seg0[NMAX];
    uint8_t order[NMAX];
};

// accelerator of segment q (validated: 0 .. PAAM_MAX_ACC - 1; the launch covers the largest)
template <int NACC>
__device__ __forceinline__ int acc_at(const BatchDev &b, int64_t q)
{
    const int u = b.acc[q];
    return u < NACC ? u : NACC - 1;
}

template <int G, int NACC>
__device__ void acc_system(const BatchDev &b, const AnalysisParams &p, int64_t item, AccSmem<G, NACC> &s, int lane,
                           unsigned gm, int64_t *__restrict__ R_out, uint8_t *__restrict__ st_out,
                           uint8_t *__restrict__ verdict, int32_t *wide_list, int32_t *wide_count)
{
    constexpr int NMAX = G;
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
    if (n > NMAX) {
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    const int16_t *rank_row = p.K > 0 ? p.ranks + (sys * p.Kc + cand_of(p, sys, cand)) * p.nmax : nullptr;
    const int32_t *xprio = p.K > 0 ? nullptr : b.exec_prio; // candidates: criticality-as-priority
    const int64_t x0 = b.sys_exec_off[sys];
    const uint64_t kappa2 = 2 * (uint64_t)p.kappa, eps = (uint64_t)p.eps;
    const int64_t seg_base = n > 0 ? b.cb_seg_off[b.chain_cb_off[c0]] : 0;

    // ---- per-chain aggregates (Sec. II-C), per accelerator ------------------
    const int j = lane;
    const bool val = j < n;
    uint32_t tm2 = 0, mg = 0, lg = 0, Dv = 0, Ev = 0, Emx = 0, seg0 = 0, dlt = 0;
    uint32_t Sa[NACC], Ma[NACC], Amn[NACC], dla[NACC];
    Mask users[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) Sa[u] = Ma[u] = Amn[u] = dla[u] = 0, users[u] = 0;
    int32_t pr = INT32_MIN, ep = INT32_MIN, ex = -1 - j, co = -1 - j;
    bool sp = false;
    Mask spins = 0, rbits = 0;
    unsigned fits = 1, rank_ok = 1;
    if (val) {
        const int64_t g = c0 + j;
        const int64_t T = b.T[g], D = b.D[g];
        const int x = b.exec[g];
        if (rank_row) { // candidate priority order: rank 0 is the highest priority
            const int r = rank_row[j];
            rank_ok &= (r >= 0 && r < n) ? 1u : 0u;
            rbits |= (r >= 0 && r < n) ? (Mask)1 << r : 0;
            pr = n - 1 - r;
        } else {
            pr = b.prio[g];
        }
        ex = x;
        co = b.exec_core[x0 + x];
        ep = xprio ? xprio[x0 + x] : INT32_MIN;
        sp = b.spin[g] != 0;
        const int64_t cb0 = b.chain_cb_off[g], cb1 = b.chain_cb_off[g + 1];
        uint64_t E = 0, Emax = 0;
        for (int64_t cb = cb0; cb < cb1; ++cb) {
            const uint64_t e = (uint64_t)b.E[cb];
            E += e;
            Emax = e > Emax ? e : Emax;
        }
        const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
        uint64_t S[NACC], M[NACC], Amin[NACC], dl[NACC];
#pragma unroll
        for (int u = 0; u < NACC; ++u) S[u] = M[u] = dl[u] = 0, Amin[u] = ~0ull;
        for (int64_t q = q0; q < q1; ++q) {
            const uint64_t a = (uint64_t)b.A[q] + kappa2; // A* = A + 2 kappa
            const int uq = acc_at<NACC>(b, q);
#pragma unroll
            for (int u = 0; u < NACC; ++u)
                if (u == uq) {
                    S[u] += a;
                    M[u] = a > M[u] ? a : M[u];
                    Amin[u] = a < Amin[u] ? a : Amin[u];
                    dl[u] += 1;
                }
        }
        const uint64_t dtot = (uint64_t)(q1 - q0);
        uint64_t Stot = 0;
#pragma unroll
        for (int u = 0; u < NACC; ++u) Stot += S[u];
        const bool fit = (uint64_t)T < kFitR && (uint64_t)D < kFitR && E < kFitR && Stot < kFitR && dtot < kFitR &&
                         (eps == 0 || dtot <= (kFitR - 1) / eps);
        fits = fit ? 1u : 0u;
        if (fit) rdivisor((uint32_t)T, tm2, mg, lg);
        Dv = (uint32_t)D;
        Ev = (uint32_t)E;
        Emx = (uint32_t)Emax;
        dlt = (uint32_t)dtot;
        seg0 = (uint32_t)(q0 - seg_base);
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            Sa[u] = (uint32_t)S[u];
            Ma[u] = (uint32_t)M[u];
            dla[u] = (uint32_t)dl[u];
            Amn[u] = dl[u] ? (uint32_t)(Amin[u] < kFitR ? Amin[u] : 0) : 0;
            users[u] = dl[u] ? (Mask)1 << j : 0;
        }
        spins = sp ? (Mask)1 << j : 0;
    }
    fits = rand_<G>(fits, gm);
#pragma unroll
    for (int u = 0; u < NACC; ++u) users[u] = ror<G>(users[u], gm);
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
    const uint32_t dsys = rmax<G>(Dv, gm);
    const bool narrow = dsys < kNarrow - G;
    if (!fits) {
        if (lane == 0) wide_list[atomicAdd(wide_count, 1)] = (int32_t)item;
        return;
    }
    // The system's iteration bound (see the header of paam_rta_load_systems): no
    // recurrence of Eq. 3 or Eq. 6 takes more than L = sum_h ceil(Dmax / T_h) + 2
    // evaluations.  With L within kIterCap (always, for a validated batch) the loops
    // run without counters; otherwise every loop stops at kIterCap (PAAM_ST_ITERCAP).
    const bool counted =
        __reduce_add_sync(gm, val ? umin(rarrivals(dsys, tm2, mg, lg) - 1u, kIterCap + 1u) : 0u) + 2u > kIterCap;
    if (!xprio) { // criticality-as-priority: highest chain priority on the executor
        int32_t best = INT32_MIN;
        for (int t = 0; t < n; ++t) {
            const int32_t pt = __shfl_sync(gm, pr, t, G), xt = __shfl_sync(gm, ex, t, G);
            if (xt == ex && pt > best) best = pt;
        }
        ep = best;
    }

    // ---- relations, analysis order, CPU blocking (Lemma 4), and per
    // accelerator the skip test's sums over hps_a and (one bucket) blk_a
    Mask higher = 0, samex = 0, hppm = 0;
    int pos = 0;
    uint32_t Bv = 0;
    int rank[NACC];
    uint32_t blk[NACC];
    uint64_t hchd[NACC], sums[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) rank[u] = 0, blk[u] = 0, hchd[u] = sums[u] = 0;
    const bool one_bucket = p.n_buckets == 1;
    if (val) {
        s.key[j] = make_int4(pr, ex, co, ep);
        s.dv[j] = make_uint4(Emx, tm2, mg, lg);
#pragma unroll
        for (int u = 0; u < NACC; ++u) s.sm[j][u] = make_uint2(Sa[u], Ma[u]);
    }
    __syncwarp(gm);
    for (int t = 0; t < n; ++t) {
        const int4 kt4 = s.key[t];
        const uint4 dv4 = s.dv[t];
        const int32_t pt = kt4.x, xt = kt4.y, kt = kt4.z, et = kt4.w;
        const bool hi = pt > pr;
        const bool sx = xt == ex;
        const Mask bit = (Mask)1 << t;
        higher |= hi ? bit : 0;
        samex |= sx ? bit : 0;
        hppm |= (!sx && kt == co && et > ep) ? bit : 0; // hpp, Lemma 4
        pos += (et > ep) || (et == ep && hi);           // executor, then chain priority
        if (sx && pt < pr && dv4.x > Bv) Bv = dv4.x;    // one LP callback on the executor
        const uint64_t mu_d = rarrivals(Dv, dv4.y, dv4.z, dv4.w);
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const uint2 sm2 = s.sm[t][u];
            const bool ut = (users[u] >> t) & 1;
            rank[u] += (ut && hi) ? 1 : 0;
            const bool act = dla[u] != 0 && ut; // c and t both use accelerator u
            const uint32_t sv = (act && hi) ? sm2.x : 0u;
            hchd[u] += mu_d * sv;
            sums[u] += sv;
            if (one_bucket && act && pt < pr && sm2.y > blk[u]) blk[u] = sm2.y;
        }
    }
    int32_t bucket[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) { // bucket = floor(rank * n_buckets / |U_a|) (R2), per accelerator
        const int nu = rpopc(users[u]);
        bucket[u] = (val && dla[u]) ? (int32_t)((uint32_t)rank[u] * (uint32_t)p.n_buckets / (uint32_t)nu) : -1;
    }
    if (!one_bucket) { // same-bucket blocking (R2-R3) with several buckets
        for (int t = 0; t < n; ++t) {
            const bool hi = (higher >> t) & 1;
#pragma unroll
            for (int u = 0; u < NACC; ++u) {
                const uint32_t mt = __shfl_sync(gm, Ma[u], t, G);
                const int32_t bt = __shfl_sync(gm, bucket[u], t, G);
                const bool ut = (users[u] >> t) & 1;
                const bool same = bucket[u] >= 0 && ut && !hi && t != j && bt == bucket[u];
                blk[u] = (same && mt > blk[u]) ? mt : blk[u];
            }
        }
    }

    // ---- own recurrence terms to shared memory ------------------------------
    Mask need_exact[NACC];
#pragma unroll
    for (int u = 0; u < NACC; ++u) need_exact[u] = 0;
    if (val) {
        const uint64_t cap = (uint64_t)Dv + 1; // values above D act the same as D + 1
        s.hp[j] = higher & samex;
        s.hpp[j] = hppm;
        s.rec[j] = make_uint4(Dv, Bv + Ev, (uint32_t)((uint64_t)dlt * eps), dlt);
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            s.hps[j][u] = higher & users[u];
            const uint64_t own = (uint64_t)Sa[u] + (uint64_t)dla[u] * blk[u];
            s.own[j][u] = (uint32_t)(own < cap ? own : cap);
            const uint64_t lim = own + hchd[u];
            s.seg[j][u] = make_uint4(kInfR, (uint32_t)(lim < cap ? lim : cap), blk[u], dla[u]);
            // exact Lemma 2 sum only where it can beat Eq. 4 below D (see analyze_reg.cu)
            const uint64_t f = ((uint64_t)Amn[u] + blk[u]) >= 1 ? 2 : 1;
            if (dla[u] && f * dla[u] * sums[u] < hchd[u]) need_exact[u] = (Mask)1 << j;
        }
        s.seg0[j] = seg0;
        s.order[pos] = (uint8_t)j;
    }
#pragma unroll
    for (int u = 0; u < NACC; ++u) need_exact[u] = ror<G>(need_exact[u], gm);
    __syncwarp(gm);

    Mask capm = 0; // chains whose recurrence reached kIterCap evaluations
    uint32_t Ehp = Ev, Ehpp = Ev + (sp ? 0u : (uint32_t)((uint64_t)dlt * eps)), Rv = 0;
    Mask sched = 0, dep = 0;
    // the fixed points: counted loops only where the bound above exceeds kIterCap
    auto fixed_points = [&](auto counted_tag) {
    constexpr bool CNT = decltype(counted_tag)::value;
    // ---- exact per-segment fixed points (Lemma 2), per accelerator ----------
#pragma unroll 1
    for (int u = 0; u < NACC; ++u) {
        for (Mask nm = need_exact[u]; nm; nm &= nm - 1) {
            const int c = rlowest(nm);
            const Mask hps = s.hps[c][u];
            const uint4 sg = s.seg[c][u];
            const uint32_t Dc = s.rec[c].x, dtc = s.rec[c].w, lim = sg.y, blkc = sg.z;
            const uint32_t acoef = ((hps >> j) & 1) ? Sa[u] : 0u;
            const int64_t qb = seg_base + s.seg0[c];
            uint64_t Hsum = 0;
            bool inf = false;
            for (uint32_t q = 0; q < dtc && !inf; ++q) {
                if (acc_at<NACC>(b, qb + q) != u) continue; // the chain's segments on accelerator u
                const uint64_t base = (uint64_t)b.A[qb + q] + kappa2 + blkc;
                uint64_t h = base; // the recurrence starts with the first two terms
                uint32_t ev = 0;
                for (;;) {
                    if (h > Dc || Hsum + h >= lim) {
                        inf = true;
                        break;
                    }
                    if (CNT && ev++ == kIterCap) {
                        inf = true;
                        capm |= (Mask)1 << c;
                        break;
                    }
                    const uint64_t part = (uint64_t)rarrivals((uint32_t)h, tm2, mg, lg) * acoef;
                    const uint64_t nh = base + gsum<G>(part, narrow, gm);
                    if (nh == h) break; // strictly increasing until here, bounded by D
                    h = nh;
                }
                Hsum += h;
            }
            if (lane == 0 && !inf) s.seg[c][u].x = (uint32_t)Hsum;
            __syncwarp(gm);
        }
    }

    // ---- Theorem 1 (Eq. 6), chain by chain ----------------------------------
    for (int step = 0; step < n; ++step) {
        const int c = s.order[step];
        const Mask hp = s.hp[c], hpp = s.hpp[c];
        const Mask cbit = (Mask)1 << c;
        if ((hp | (hpp & spins)) & ~sched) { // a needed H*_h is not available
            dep |= cbit;
            if (rank_row) break; // a candidate fails at its first unschedulable chain
            continue;
        }
        if (capm & cbit) { // a segment recurrence was cut short: no bound (PAAM_ST_ITERCAP)
            if (rank_row) break;
            continue;
        }
        const uint32_t ccoef = ((hp >> j) & 1) ? Ehp : (((hpp >> j) & 1) ? Ehpp : 0u);
        uint32_t acoef[NACC];
        bool uses[NACC]; // the same in every lane of the group
        uint64_t own[NACC], Hseg[NACC];
        const uint4 rc = s.rec[c];
        const uint64_t Dc = rc.x, base = rc.y, deps = rc.z, dl = rc.w;
        uint64_t h0 = 0;
#pragma unroll
        for (int u = 0; u < NACC; ++u) {
            const uint4 sg = s.seg[c][u];
            uses[u] = sg.w != 0;
            acoef[u] = ((s.hps[c][u] >> j) & 1) ? Sa[u] : 0u;
            own[u] = s.own[c][u];
            Hseg[u] = sg.x == kInfR ? ~0ull : (uint64_t)sg.x;
            if (uses[u]) h0 += Hseg[u] < own[u] ? Hseg[u] : own[u];
        }
        // start: B + E + H* with the interference parts of Eq. 4 empty
        uint64_t R = base + (dl ? h0 + deps : 0);
        uint64_t hs = 0;
        bool ok = false;
        uint32_t ev = 0;
        while (R <= Dc) {
            if (CNT && ev++ == kIterCap) {
                capm |= cbit;
                break;
            }
            const uint64_t mu = rarrivals((uint32_t)R, tm2, mg, lg);
            const uint64_t cpu = gsum<G>(mu * ccoef, narrow, gm);
            hs = 0;
#pragma unroll
            for (int u = 0; u < NACC; ++u) {
                if (!uses[u]) continue;
                const uint64_t hch = own[u] + gsum<G>(mu * acoef[u], narrow, gm); // Eq. 4 at accelerator u
                hs += Hseg[u] < hch ? Hseg[u] : hch; // min(Eq. 3, Eq. 4), summed over accelerators (R1)
            }
            if (dl) hs += deps; // Eq. 1
            const uint64_t Rn = base + hs + cpu;
            if (Rn == R) {
                ok = true;
                break;
            }
            R = Rn;
        }
        if (ok) {
            sched |= cbit;
            if (j == c) {
                Rv = (uint32_t)R;
                Ehp = Ev + (uint32_t)hs;
                if (sp) Ehpp = Ev + (uint32_t)hs;
            }
        } else if (rank_row) {
            break;
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
    if (val) {
        const bool ok = (sched >> j) & 1;
        R_out[c0 + j] = ok ? (int64_t)Rv : -1;
        st_out[c0 + j] = ok ? PAAM_ST_SCHED
                            : (((capm >> j) & 1) ? PAAM_ST_ITERCAP
                                                 : (((dep >> j) & 1) ? PAAM_ST_DEP : PAAM_ST_OVERRUN));
    }
    if (lane == 0 && verdict) verdict[sys] = sched == all ? 1 : 0;
    __syncwarp(gm);
}

// three resident blocks of 256 per SM for up to three accelerators (80
// registers, no spills); four accelerators need more registers: two blocks
template <int G, int NACC>
__global__ void __launch_bounds__(256, NACC <= 3 ? 3 : 2) analyze_reg_acc_kernel(BatchDev b, AnalysisParams p, int64_t *R,
                                                                 uint8_t *st, uint8_t *verdict, int32_t *wide_list,
                                                                 int32_t *wide_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int groups = blockDim.x / G;
    const int grp = threadIdx.x / G;
    const int lane = threadIdx.x % G;
    AccSmem<G, NACC> &s = reinterpret_cast<AccSmem<G, NACC> *>(smem_raw)[grp];
    const unsigned gm = rgroup_mask<G>();
    const int64_t n_items = p.K > 0 ? b.n_sys * p.K : b.n_sys;
    for_each_item<G>(p, n_items, grp, groups, lane, gm, [&](int64_t i) {
        acc_system<G, NACC>(b, p, i, s, lane, gm, R, st, verdict, wide_list, wide_count);
    });
}

template <int NACC>
int launch_acc_n(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                 int64_t max_items, cudaStream_t stream)
{
    constexpr int G = 16, threads = 256;
    const int groups = threads / G;
    const size_t smem = sizeof(AccSmem<G, NACC>) * groups;
    auto kern = analyze_reg_acc_kernel<G, NACC>;
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

int paam_launch_reg_acc(const paam_batch *bt, const AnalysisParams &p, int64_t *R, uint8_t *st, uint8_t *verdict,
                        int64_t max_items, cudaStream_t stream)
{
    const unsigned long long used = bt->stats[ST_ACCMAX] + 1;
    static_assert(PAAM_MAX_ACC == 4, "instantiations below cover 2..4 accelerators");
    if (used >= 4) return launch_acc_n<4>(bt, p, R, st, verdict, max_items, stream);
    if (used == 3) return launch_acc_n<3>(bt, p, R, st, verdict, max_items, stream);
    return launch_acc_n<2>(bt, p, R, st, verdict, max_items, stream);
}
