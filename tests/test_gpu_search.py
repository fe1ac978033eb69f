"""Exact priority-assignment search on the GPU against the oracle's search:
identical schedulable sets per candidate and identical first schedulable
candidate per system, in exhaustive and early-exit modes."""
import numpy as np
import pytest

import oracle
import paam_gen as g

from gpu_util import ctx

pytestmark = pytest.mark.gpu


def _run(sy, ranks, stop_at_first=False, cfg_index=None, **p):
    import torch

    import paper_2404_06452_gb300 as pkg

    b = pkg.paam_rta_load_systems(ctx(), sy)
    if cfg_index is not None:
        pkg.paam_rta_set_launch_config(b, cfg_index)
    r = torch.from_numpy(ranks).cuda()
    first, cand = pkg.search(ctx(), b, r, stop_at_first=stop_at_first, **p)
    torch.cuda.synchronize()
    b.free()
    return first.cpu().numpy(), cand.cpu().numpy()


@pytest.mark.parametrize("cfg", ["cfg4", "cfg4s"])
def test_search_exhaustive_matches_oracle(cfg):
    sy = g.generate(cfg, n_sys=600)
    ranks = g.candidate_ranks(sy, 64, 11)
    p = dict(n_buckets=2, eps=1000, kappa=500)
    first, cand = _run(sy, ranks, **p)
    ref = oracle.search(sy, ranks, threads=8, **p)
    assert np.array_equal(cand, ref["cand_ok"])
    assert np.array_equal(first, ref["first_ok"])


@pytest.mark.parametrize("stop_at_first", [False, True])
def test_search_deadlines_past_the_narrow_bound(stop_at_first):
    # periods up to 300 ms: about a third of the systems stay below 2^27 ns (the lazy
    # kernels, reading chain records), the others go to the int64 kernel
    sy = g.generate("cfg1", n_sys=1500, t_min=1e7, t_max=3e8, seed=5)
    ranks = g.candidate_ranks(sy, 24, 7)
    p = dict(n_buckets=2, eps=391_000, kappa=129_180)
    first, cand = _run(sy, ranks, stop_at_first=stop_at_first, **p)
    ref = oracle.search(sy, ranks, threads=8, **p)
    assert np.array_equal(first, ref["first_ok"])
    if stop_at_first:
        assert np.all(cand <= ref["cand_ok"])  # skipped candidates read 0
    else:
        assert np.array_equal(cand, ref["cand_ok"])


def test_search_early_exit_same_first_candidate():
    sy = g.generate("cfg4s", n_sys=2000)
    ranks = g.candidate_ranks(sy, 128, 5)
    first_x, cand_x = _run(sy, ranks)
    first_e, cand_e = _run(sy, ranks, stop_at_first=True)
    assert np.array_equal(first_e, first_x)
    assert np.all(cand_e <= cand_x)  # skipped candidates read 0
    assert (first_x >= 0).mean() > 0.2


def test_search_every_launch_config_and_mixed_sizes():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg3", n_sys=400)
    ranks = g.candidate_ranks(sy, 8, 3, nmax=64)
    ref = oracle.search(sy, ranks, threads=8, n_buckets=3)
    for i in range(pkg.paam_rta_num_launch_configs()):
        first, cand = _run(sy, ranks, cfg_index=i, n_buckets=3)
        assert np.array_equal(cand, ref["cand_ok"]), i
        assert np.array_equal(first, ref["first_ok"]), i


def test_search_rejects_non_permutation():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg4", n_sys=50)
    ranks = g.candidate_ranks(sy, 4, 1)
    ranks[7, 2, 3] = ranks[7, 2, 4]  # duplicate rank
    with pytest.raises(pkg.PaamError) as ei:
        _run(sy, ranks)
    assert ei.value.code == -1


def test_ordered_search_subset():
    """Visiting a permuted subset of candidates admits exactly those the full
    search admits among them; first_ok is the first admitted in visit order."""
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg4s", n_sys=800)
    Kc, K = 64, 20
    ranks = g.candidate_ranks(sy, Kc, 21)
    ref = oracle.search(sy, ranks, threads=8)
    rng = np.random.default_rng(3)
    order = np.stack([rng.permutation(Kc)[:K] for _ in range(sy.n_sys)]).astype(np.int32)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = torch.from_numpy(ranks).cuda()
    o = torch.from_numpy(order).cuda()
    for early in (False, True):
        first = torch.empty(sy.n_sys, dtype=torch.int32, device="cuda")
        cand = torch.empty((sy.n_sys, Kc), dtype=torch.uint8, device="cuda")
        pkg.paam_rta_search_ordered(ctx(), b, pkg.analysis_opts(), r, o, early, cand, first)
        torch.cuda.synchronize()
        first, cand = first.cpu().numpy(), cand.cpu().numpy()
        want_first = np.full(sy.n_sys, -1)
        for s in range(sy.n_sys):
            ok = [k for k in order[s] if ref["cand_ok"][s, k]]
            want_first[s] = ok[0] if ok else -1
        assert np.array_equal(first, want_first)
        visited = np.zeros_like(ref["cand_ok"])
        np.put_along_axis(visited, order.astype(np.int64), 1, axis=1)
        if not early:
            assert np.array_equal(cand, ref["cand_ok"] & visited)
        else:
            assert np.all(cand <= (ref["cand_ok"] & visited))
    bad = o.clone()
    bad[3, 2] = Kc
    with pytest.raises(pkg.PaamError):
        pkg.paam_rta_search_ordered(ctx(), b, pkg.analysis_opts(), r, bad, False, None,
                                    torch.empty(sy.n_sys, dtype=torch.int32, device="cuda"))
    b.free()


@pytest.mark.parametrize("cfg", ["cfg4", "cfg4s"])
def test_search_full_shape_matches_oracle(cfg):
    """The search workload at its specified shape, 10,000 systems of 16 chains
    x 256 candidate orders (slot 0 the Audsley-style seed, slot 1
    deadline-monotonic, the rest random permutations), in the launch
    configuration the search autotuner picks for each mode, against the
    oracle's exhaustive search on every system and candidate."""
    import os

    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate(cfg)
    assert sy.n_sys == 10000
    ranks = g.candidate_ranks(sy, 256, g.CONFIGS[cfg]["seed"] + 7)
    threads = os.cpu_count() or 8
    ranks[:, 0, :] = oracle.audsley(sy, nmax=ranks.shape[2], threads=threads)  # the seed, from the oracle
    ref = oracle.search(sy, ranks, threads=threads)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = torch.from_numpy(ranks).cuda()
    for stop in (False, True):
        pkg.paam_rta_autotune_search(ctx(), b, pkg.analysis_opts(), r, stop_at_first=stop)
        first, cand = pkg.search(ctx(), b, r, stop_at_first=stop)
        torch.cuda.synchronize()
        assert np.array_equal(first.cpu().numpy(), ref["first_ok"]), stop
        if not stop:
            assert np.array_equal(cand.cpu().numpy(), ref["cand_ok"])
        else:
            assert np.all(cand.cpu().numpy() <= ref["cand_ok"])
    b.free()
    if cfg == "cfg4s":
        assert 0.3 < (ref["first_ok"] >= 0).mean() < 0.95
