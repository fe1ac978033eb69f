"""Exactness of the division by multiply-shift that the 32-bit analysis
kernels use for Lemma 1's arrival count mu(t) = ceil(t / T) + 1 (Eq. 2),
checked on the CPU against plain integer division.

For T < 2^30, l = ceil(log2 T) and m = ceil(2^(31 + l) / T), every x < 2^31
has floor(x / T) = floor(x m / 2^(31 + l)) (Granlund and Montgomery 1994,
Theorem 4.2 with N = 31).  The register-table kernels take the same value as
the high 32-bit word of (2x) m shifted right by l (2x < 2^32); the others
shift the 64-bit product.  Edge cases (T = 1, powers of two and their
neighbours, the largest T, every x near a multiple of T and near 2^31) and
random pairs."""
import numpy as np


def _divisor(T):
    T = np.asarray(T, dtype=np.uint64)
    l = np.zeros_like(T)
    big = T > 1
    # ceil(log2 T) = bit length of T - 1
    l[big] = np.array([int(t - 1).bit_length() for t in T[big]], dtype=np.uint64)
    m = ((np.uint64(1) << (np.uint64(31) + l)) + T - np.uint64(1)) // T
    return l, m


def _check(x, T):
    x = np.asarray(x, dtype=np.uint64)
    T = np.asarray(T, dtype=np.uint64)
    l, m = _divisor(T)
    assert np.all(m < (1 << 32)) and np.all(x < (1 << 31))
    want = x // T
    shift_form = (x * m) >> (np.uint64(31) + l)
    high_form = (((np.uint64(2) * x) * m) >> np.uint64(32)) >> l
    assert np.array_equal(shift_form, want)
    assert np.array_equal(high_form, want)


def test_edge_divisors_and_dividends():
    Ts = set(range(1, 130))
    for k in range(1, 31):
        Ts.update({(1 << k) - 1, 1 << k, (1 << k) + 1})
    Ts = sorted(t for t in Ts if 1 <= t < (1 << 30))
    xs, ts = [], []
    for T in Ts:
        cand = {0, 1, T - 1, T, T + 1, 2 * T - 1, 2 * T, (1 << 31) - 1, (1 << 31) - 2}
        q = ((1 << 31) - 1) // T
        cand.update({q * T - 1, q * T, q * T + 1, (q - 1) * T + T - 1})
        for x in cand:
            if 0 <= x < (1 << 31):
                xs.append(x)
                ts.append(T)
    _check(xs, ts)


def test_random_pairs():
    rng = np.random.default_rng(20240406)
    n = 2_000_000
    T = rng.integers(1, 1 << 30, n, dtype=np.uint64)
    # log-uniform divisors as well, so that small and mid-range T are covered
    T[: n // 2] = np.exp(rng.uniform(0, np.log(2.0 ** 30 - 1), n // 2)).astype(np.uint64).clip(1, (1 << 30) - 1)
    x = rng.integers(0, 1 << 31, n, dtype=np.uint64)
    _check(x, T)


def test_arrival_count_form():
    # mu(t) = ceil(t / T) + 1 as the kernels take it: x = t + T - 1 with t, T < 2^30
    rng = np.random.default_rng(7)
    n = 500_000
    T = rng.integers(1, 1 << 30, n, dtype=np.uint64)
    t = rng.integers(0, 1 << 30, n, dtype=np.uint64)
    l, m = _divisor(T)
    tm2 = np.uint64(2) * (T - np.uint64(1))
    mu = ((((np.uint64(2) * t + tm2) * m) >> np.uint64(32)) >> l) + np.uint64(1)
    want = (t + T - np.uint64(1)) // T + np.uint64(1)
    assert np.array_equal(mu, want)
