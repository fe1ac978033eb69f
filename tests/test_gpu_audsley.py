"""The Audsley-style priority seed on the GPU (``paam_rta_audsley_order``)
against the oracle's greedy: identical rank rows, bit for bit, on the search
workloads, on uneven system sizes, with several accelerators and the safe
blocking reading, across internal system chunks, and on samples of the full
10,000-system search batch."""
import numpy as np
import pytest

import oracle
import paam_gen as g

from gpu_util import ctx

pytestmark = pytest.mark.gpu


def _seed(sy, nmax, **p):
    import torch

    import paper_2404_06452_gb300 as pkg

    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = pkg.audsley_order(ctx(), b, nmax, **p)
    torch.cuda.synchronize()
    b.free()
    return r.cpu().numpy()


@pytest.mark.parametrize("cfg,p", [("cfg1", {}), ("cfg4s", {}),
                                   ("cfg4s", dict(n_buckets=2, eps=391_000, kappa=129_180)),
                                   ("cfg4", dict(n_buckets=6, eps=1000))])
def test_seed_matches_oracle(cfg, p):
    sy = g.generate(cfg, n_sys=1500)
    nmax = int(np.diff(sy.sys_chain_off).max())
    got = _seed(sy, nmax, **p)
    ref = oracle.audsley(sy, nmax=nmax, threads=8, **p)
    np.testing.assert_array_equal(got, ref)


def test_seed_uneven_sizes():
    sy = g.generate("cfg3", n_sys=300)
    got = _seed(sy, 64, n_buckets=3, eps=500)
    ref = oracle.audsley(sy, nmax=64, threads=8, n_buckets=3, eps=500)
    np.testing.assert_array_equal(got, ref)
    counts = np.diff(sy.sys_chain_off)
    assert counts.max() > 30 and counts.min() <= 3  # large and tiny systems in one batch


def test_seed_deadlines_past_the_narrow_bound():
    # periods up to 300 ms: a third of the systems keep every deadline below 2^27 ns
    # (the lazy kernel's trials), the others reach past it (the int64 kernel's)
    sy = g.generate("cfg1", n_sys=1500, t_min=1e7, t_max=3e8, seed=5)
    dmax = np.maximum.reduceat(sy.D, sy.sys_chain_off[:-1])
    assert 0.2 < (dmax < 2**27 - 16).mean() < 0.8
    got = _seed(sy, 4, n_buckets=2, eps=391_000, kappa=129_180)
    ref = oracle.audsley(sy, nmax=4, threads=8, n_buckets=2, eps=391_000, kappa=129_180)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("blocking_mode", [0, 1])
def test_seed_several_accelerators_and_safe_blocking(blocking_mode):
    from paam_gen import tiny

    sy, _ = tiny.tiny_batch(17, 3000, n_max=6, cb_max=3, x_max=3, n_acc=3, seg_max=2)
    got = _seed(sy, 6, n_buckets=2, eps=1, kappa=1, blocking_mode=blocking_mode)
    ref = oracle.audsley(sy, nmax=6, threads=8, n_buckets=2, eps=1, kappa=1, blocking_mode=blocking_mode)
    np.testing.assert_array_equal(got, ref)


def test_seed_in_system_chunks():
    # long rows make the trial buffer exceed one chunk: 6,000 systems run in two
    sy = g.generate("cfg4s", n_sys=6000)
    got = _seed(sy, 4096)
    assert got.shape == (6000, 4096)
    assert (got[:, 16:] == -1).all()
    idx = np.r_[0:300, 3900:4300, 5700:6000]  # both sides of the chunk boundary
    ref = oracle.audsley(sy.subset(idx), nmax=16, threads=8)
    np.testing.assert_array_equal(got[idx, :16], ref)


def test_seed_full_search_batch_sampled():
    sy = g.generate("cfg4s")  # the 10,000-system, 16-chain search workload
    got = _seed(sy, 16)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(sy.n_sys, 600, replace=False))
    ref = oracle.audsley(sy.subset(idx), nmax=16, threads=8)
    np.testing.assert_array_equal(got[idx], ref)
    for row in got:
        assert sorted(row.tolist()) == list(range(16))


def test_seed_rejects_short_rows():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg4s", n_sys=10)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    with pytest.raises(pkg.PaamError):
        pkg.audsley_order(ctx(), b, 8)
    b.free()
