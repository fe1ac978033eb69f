"""The multiply-shift divisor behind every arrival count ceil(t / T) of Lemma 1
(Eq. 2): the kernels build m = ceil(2^(31 + l) / T), l = ceil(log2 T) from a
single-precision reciprocal estimate and exact remainder corrections.  Checked
for every period T in [1, 2^30) against torch's int64 division."""
import pytest

pytestmark = pytest.mark.gpu

CHUNK = 1 << 26


def _exact(T):
    import torch

    t1 = T.to(torch.int64) - 1
    l = torch.zeros_like(t1)
    for k in range(31):
        l += ((t1 >> k) > 0).to(torch.int64)
    one = torch.ones_like(t1)
    m = (torch.bitwise_left_shift(one, 31 + l) + t1) // (t1 + 1)
    return m, l


def test_divisor_every_period_below_2_30():
    import torch

    import paper_2404_06452_gb300 as pkg

    n_bad = 0
    first_bad = None
    for lo in range(1, 1 << 30, CHUNK):
        hi = min(lo + CHUNK, 1 << 30)
        T = torch.arange(lo, hi, dtype=torch.int32, device="cuda")
        m = torch.empty_like(T)
        l = torch.empty_like(T)
        pkg.paam_diag_divisor(T, m, l)
        em, el = _exact(T)
        got_m = m.to(torch.int64) & 0xFFFFFFFF
        bad = (got_m != em) | (l.to(torch.int64) != el)
        nb = int(bad.sum().item())
        if nb and first_bad is None:
            i = int(torch.nonzero(bad)[0].item())
            first_bad = (lo + i, int(got_m[i].item()), int(em[i].item()), int(l[i].item()), int(el[i].item()))
        n_bad += nb
    assert n_bad == 0, (n_bad, first_bad)


def test_divisor_edge_periods_and_empty_call():
    """Powers of two, their neighbours and the largest period, against Python
    integers; n = 0 is a no-op."""
    import torch

    import paper_2404_06452_gb300 as pkg

    vals = sorted({v for k in range(31) for v in (1 << k, (1 << k) - 1, (1 << k) + 1) if 1 <= v < (1 << 30)})
    T = torch.tensor(vals, dtype=torch.int32, device="cuda")
    m = torch.empty_like(T)
    l = torch.empty_like(T)
    pkg.paam_diag_divisor(T, m, l)
    got = list(zip((m.to(torch.int64) & 0xFFFFFFFF).tolist(), l.tolist()))
    for t, (gm, gl) in zip(vals, got):
        el = (t - 1).bit_length()
        assert gl == el and gm == -(-(1 << (31 + el)) // t), (t, gm, gl)
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    pkg.paam_diag_divisor(e, e, e)
