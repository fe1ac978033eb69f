// reg_common.cuh -- helpers of the register-table analysis kernels
// (analyze_reg.cu and the lazy kernels): group masks and reductions, the
// 32-bit bounds, broadcasts of per-lane slots, Lemma 1's arrival count by
// multiply-shift division.
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace paam_reg {

constexpr uint64_t kFitR = 1ull << 30;
constexpr uint32_t kInfR = 0xFFFFFFFFu;
// a per-segment sum, or a chain's R, whose recurrence was stopped at kIterCap
// evaluations (PAAM_ST_ITERCAP); above every 32-bit-bound value
constexpr uint32_t kCapR = 0xFFFFFFFEu;

template <int NMAX>
struct RegMask {
    using type = typename std::conditional<(NMAX <= 32), uint32_t, uint64_t>::type;
};



// Narrow systems (every deadline below 2^27 - 64) sum per-lane partials capped
// at 2^27 - 1 in 32 bits (at most 32 lanes: no wrap-around).  A capped partial
// already exceeds every deadline, so the capped sum decides each comparison
// with D, and each minimum with a per-segment sum <= D, as the true sum would.
constexpr uint32_t kNarrow = 1u << 27;

template <int G>
__device__ __forceinline__ unsigned rgroup_mask()
{
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

template <int G, typename V>
__device__ __forceinline__ V rsum(V v, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, G);
    return v;
}

// Group reductions.  32-bit ones are one redux.sync over the group's member
// mask (every lane of a group takes the same path; groups of one warp may
// reduce at the same time, each over its own mask); 64-bit ones use shuffles.
template <int G, typename V>
__device__ __forceinline__ V ror(V v, unsigned mask)
{
    if constexpr (sizeof(V) == 4) {
        return (V)__reduce_or_sync(mask, (unsigned)v);
    } else {
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(mask, v, off, G);
        return v;
    }
}

template <int G>
__device__ __forceinline__ unsigned rand_(unsigned v, unsigned mask)
{
    return __reduce_and_sync(mask, v);
}

template <int G>
__device__ __forceinline__ uint64_t gsum(uint64_t v, bool narrow, unsigned mask)
{
    if (narrow) {
        const uint32_t x = v < kNarrow - 1 ? (uint32_t)v : kNarrow - 1;
        return __reduce_add_sync(mask, x);
    }
    return rsum<G>(v, mask);
}

template <int G>
__device__ __forceinline__ uint32_t rmax(uint32_t v, unsigned mask)
{
    return __reduce_max_sync(mask, v);
}

// value of slot t / G held by lane t % G, broadcast to the group
template <int G, int CPL, typename V>
__device__ __forceinline__ V bcast(const V (&a)[CPL], int t, unsigned mask)
{
    const int k = t / G;
    V v = a[0];
#pragma unroll
    for (int i = 1; i < CPL; ++i)
        if (k == i) v = a[i];
    return __shfl_sync(mask, v, t % G, G);
}

template <typename Mask>
__device__ __forceinline__ int rpopc(Mask m)
{
    if constexpr (sizeof(Mask) == 8)
        return __popcll(m);
    else
        return __popc(m);
}

template <typename Mask>
__device__ __forceinline__ int rlowest(Mask m)
{
    if constexpr (sizeof(Mask) == 8)
        return __ffsll((long long)m) - 1;
    else
        return __ffs((int)m) - 1;
}

// Asks L2 to fetch elements [i0, i1) of an array of `elem`-byte elements, in
// 1 MB bulk requests; the range is shrunk to whole 16-byte units inside it
// (a bulk prefetch starts and ends on 16-byte boundaries), so nothing outside
// the elements is named.
__device__ __forceinline__ void prefetch_l2(const void *base, int elem, int64_t i0, int64_t i1)
{
    if (!base || i1 <= i0) return;
    uintptr_t a = (uintptr_t)base + (uintptr_t)(i0 * elem), e = (uintptr_t)base + (uintptr_t)(i1 * elem);
    a = (a + 15) & ~(uintptr_t)15;
    e &= ~(uintptr_t)15;
    while (a < e) {
        const uint32_t sz = e - a < (1u << 20) ? (uint32_t)(e - a) : (1u << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(sz) : "memory");
        a += sz;
    }
}

// The tables of systems [s0, s0 + count) (callbacks, segments, chains,
// executors), prefetched into L2 ahead of the groups that will read them.
__device__ __forceinline__ void prefetch_systems(const BatchDev &b, const int32_t *order, int64_t s0, int64_t count)
{
    if (s0 >= b.n_sys) return;
    const int64_t s1 = s0 + count < b.n_sys ? s0 + count : b.n_sys;
    const int64_t c0 = b.sys_chain_off[s0], c1 = b.sys_chain_off[s1];
    const int64_t x0 = b.sys_exec_off[s0], x1 = b.sys_exec_off[s1];
    const int64_t cb0 = b.chain_cb_off[c0], cb1 = b.chain_cb_off[c1];
    const int64_t q0 = b.cb_seg_off[cb0], q1 = b.cb_seg_off[cb1];
    prefetch_l2(order, 4, s0, s1);
    prefetch_l2(b.sys_chain_off, 8, s0, s1 + 1);
    prefetch_l2(b.sys_exec_off, 8, s0, s1 + 1);
    prefetch_l2(b.chain_cb_off, 8, c0, c1 + 1);
    prefetch_l2(b.T, 8, c0, c1);
    prefetch_l2(b.D, 8, c0, c1);
    prefetch_l2(b.prio, 4, c0, c1);
    prefetch_l2(b.exec, 4, c0, c1);
    prefetch_l2(b.spin, 1, c0, c1);
    prefetch_l2(b.exec_core, 4, x0, x1);
    prefetch_l2(b.exec_prio, 4, x0, x1);
    prefetch_l2(b.E, 8, cb0, cb1);
    prefetch_l2(b.cb_seg_off, 8, cb0, cb1 + 1);
    prefetch_l2(b.A, 8, q0, q1);
}

// Lemma 1 (Eq. 2): ceil(t / T) + 1 for t, T < 2^30.  With x = t + T - 1 < 2^31,
// l = ceil(log2 T) and m = ceil(2^(31 + l) / T), floor(x / T) = floor(x m /
// 2^(31 + l)) for every x < 2^31 (Granlund and Montgomery 1994, Theorem 4.2
// with N = 31).  Since 2x < 2^32 that is the high word of (2x) m shifted right
// by l: one multiply-high and one 32-bit shift.  The divisor is kept as
// {tm2 = 2 (T - 1), m, l}.
//
// m without a 64-bit division: for T = 2^l, m = 2^31.  Otherwise 3 <= T < 2^30,
// tn = T 2^(32 - l) lies in (2^31, 2^32) and 2^(31 + l) / T = 2^63 / tn, which is
// not an integer (T has an odd factor), so m = floor(2^63 / tn) + 1.  The
// quotient q = floor(2^63 / tn) < 2^32 comes from a single-precision reciprocal
// estimate r (relative error below 2^-21 with the conversion of tn): q0 = r 2^63
// is within 2^10 of q, the remainder 2^63 - q0 tn then has magnitude below 2^42,
// and q0 + trunc(r (2^63 - q0 tn)) is within 2 of q; two compare-and-step
// corrections each way on the exact remainder make it exact (Newton's step on
// the reciprocal followed by remainder correction, as in long division).
__device__ __forceinline__ float rcp_estimate(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t rmagic(uint32_t T, uint32_t l)
{
    if ((T & (T - 1u)) == 0u) return 1u << 31;
    const uint32_t tn = T << (32u - l);
    const float r = rcp_estimate((float)tn);
    int64_t q = (int64_t)__float2uint_rz(r * 0x1p63f);
    int64_t rem = (int64_t)((1ull << 63) - (uint64_t)q * tn);
    q += (int64_t)__float2int_rz((float)rem * r);
    rem = (int64_t)((1ull << 63) - (uint64_t)q * tn);
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (rem < 0) {
            --q;
            rem += tn;
        }
#pragma unroll
    for (int k = 0; k < 2; ++k)
        if (rem >= (int64_t)tn) {
            ++q;
            rem -= tn;
        }
    return (uint32_t)q + 1u;
}

__device__ __forceinline__ void rdivisor(uint32_t T, uint32_t &tm2, uint32_t &m, uint32_t &l)
{
    l = T > 1 ? 32u - (uint32_t)__clz(T - 1u) : 0u;
    m = rmagic(T, l);
    tm2 = 2u * (T - 1u);
}

__device__ __forceinline__ uint32_t rarrivals(uint32_t t, uint32_t tm2, uint32_t m, uint32_t l)
{
    return (__umulhi(2u * t + tm2, m) >> l) + 1u;
}

} // namespace paam_reg
