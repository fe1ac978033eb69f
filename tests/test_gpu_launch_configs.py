"""Every launch configuration, the int64 fallback and graph replay give the
oracle's bit-exact results."""
import random

import numpy as np
import pytest

import oracle
import paam_gen as g
from paam_gen import tiny

from gpu_util import analyze_poisoned, assert_same, ctx

pytestmark = pytest.mark.gpu


def _mixed_batch():
    """cfg3-shaped systems (2..64 chains) plus systems whose times exceed the
    32-bit fast path (periods up to ~34 s), interleaved."""
    a = g.generate("cfg3", n_sys=6000)
    rng = random.Random(17)
    big = [tiny.tiny_system(rng, n_min=2, n_max=40, cb_max=5, x_max=6, periods=tuple(range(2**30, 2**35, 2**27)),
                            e_max=2**27, a_max=2**26, p_seg=0.5, p_spin=0.5, seg_max=2) for _ in range(300)]
    b = tiny.to_systems(big)
    idx_a = np.arange(a.n_sys)
    parts = []
    # interleave: 20 fast systems, then 1 wide one
    out = []
    k = 0
    for i in range(b.n_sys):
        out.append(("a", idx_a[k:k + 20]))
        out.append(("b", np.array([i])))
        k += 20
    out.append(("a", idx_a[k:]))
    subs = [(a if w == "a" else b).subset(ix) for w, ix in out if len(ix)]
    return _concat(subs)


def _concat(subs):
    def cat_off(name, count_name):
        offs, base = [np.zeros(1, np.int64)], 0
        for s in subs:
            o = getattr(s, name)
            offs.append(o[1:] + base)
            base += o[-1]
        return np.concatenate(offs)

    cat = lambda f: np.concatenate([getattr(s, f) for s in subs])
    return g.Systems(cat_off("sys_chain_off", None), cat_off("chain_cb_off", None), cat_off("cb_seg_off", None),
                     cat("T"), cat("D"), cat("prio"), cat("exec"), cat("spin"), cat("E"), cat("A"), cat("acc"),
                     cat_off("sys_exec_off", None), cat("exec_core"), cat("exec_prio"))


def test_every_launch_config_bit_exact():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = _mixed_batch()
    ref = oracle.analyze(sy, threads=8, n_buckets=2, eps=1000, kappa=500)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    for i in range(pkg.paam_rta_num_launch_configs()):
        pkg.paam_rta_set_launch_config(b, i)
        assert_same(analyze_poisoned(ctx(), b, n_buckets=2, eps=1000, kappa=500), ref)
    b.free()


def _with_wide_deadlines(periods, n_min, n_max, implicit, seed):
    a = g.generate("cfg3", n_sys=3000)
    rng = random.Random(seed)
    mid = [tiny.tiny_system(rng, n_min=n_min, n_max=n_max, cb_max=5, x_max=6, periods=periods, e_max=2**21,
                            a_max=2**20, p_seg=0.5, p_spin=0.5, seg_max=2, implicit_deadline=implicit)
           for _ in range(200)]
    b = tiny.to_systems(mid)
    out, k = [], 0
    for i in range(b.n_sys):
        out.append(a.subset(np.arange(k, k + 15)))
        out.append(b.subset(np.array([i])))
        k += 15
    return _concat(out)


@pytest.mark.parametrize("case", ["deadlines 2^26..2^29", "deadline 2^27 - 40, 33-64 chains"])
def test_every_launch_config_between_the_narrow_and_32_bit_bounds(case):
    """Systems with deadlines at or above the narrow bounds of the 32-bit
    kernels (2^27 less 16, 32 or 64 by kernel) among ordinary ones: the batch
    takes the 32-bit path, but the narrow kernels defer those systems; every
    configuration must still analyse each of them (bit-exact)."""
    import paper_2404_06452_gb300 as pkg

    if case.startswith("deadlines"):
        sy = _with_wide_deadlines(tuple(range(2**27, 2**29, 2**22)), 2, 40, False, 23)
        assert sy.D.max() >= 2**27
    else:  # below the first pass's bound, above the 64-chain pass's
        sy = _with_wide_deadlines((2**27 - 40,), 33, 64, True, 29)
        assert sy.D.max() == 2**27 - 40
    assert sy.T.max() < 2**30
    ref = oracle.analyze(sy, threads=8)
    bt = pkg.paam_rta_load_systems(ctx(), sy)
    for i in range(pkg.paam_rta_num_launch_configs()):
        pkg.paam_rta_set_launch_config(bt, i)
        assert_same(analyze_poisoned(ctx(), bt), ref)
    bt.free()


def test_graph_replay_with_changing_outputs_and_options():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg3", n_sys=5000)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    dev = torch.device("cuda", 0)
    outs = [(torch.empty(b.n_chain, dtype=torch.int64, device=dev), torch.empty(b.n_chain, dtype=torch.uint8, device=dev),
             torch.empty(b.n_sys, dtype=torch.uint8, device=dev)) for _ in range(2)]
    plan = [(0, dict(n_buckets=1, eps=0, kappa=0)), (0, dict(n_buckets=1, eps=0, kappa=0)),
            (1, dict(n_buckets=1, eps=0, kappa=0)), (1, dict(n_buckets=3, eps=200_000, kappa=100_000)),
            (0, dict(n_buckets=3, eps=200_000, kappa=100_000)), (0, dict(n_buckets=1, eps=0, kappa=0))]
    refs = {}
    for which, p in plan:
        R, st, v = outs[which]
        R.fill_(123)
        st.fill_(9)
        pkg.paam_rta_analyze_batch(ctx(), b, pkg.analysis_opts(**p), R, st, v)
        torch.cuda.synchronize()
        key = tuple(sorted(p.items()))
        if key not in refs:
            refs[key] = oracle.analyze(sy, threads=8, **p)
        assert_same(dict(R=R.cpu().numpy(), status=st.cpu().numpy(), verdict=v.cpu().numpy()), refs[key])
    b.free()


def test_autotune_picks_a_valid_config_and_stays_exact():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg2", n_sys=50000)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    best, times = pkg.paam_rta_autotune(ctx(), b, pkg.analysis_opts())
    assert 0 <= best < pkg.paam_rta_num_launch_configs()
    assert all(t > 0 for t in times) and times[best] == min(times)
    assert pkg.paam_rta_get_launch_config(b) == best
    R, st, v = pkg.analyze(ctx(), b)
    torch.cuda.synchronize()
    assert_same(dict(R=R.cpu().numpy(), status=st.cpu().numpy(), verdict=v.cpu().numpy()),
                oracle.analyze(sy, threads=8))
    b.free()


def test_search_autotune_picks_a_valid_config_and_stays_exact():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg4s", n_sys=2000)
    ranks = g.candidate_ranks(sy, 32, 4)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    assert pkg.paam_rta_get_launch_config(b) == 28  # a new batch starts with the default configuration
    r = torch.from_numpy(ranks).cuda()
    best, times = pkg.paam_rta_autotune_search(ctx(), b, pkg.analysis_opts(), r)
    assert 0 <= best < pkg.paam_rta_num_launch_configs()
    assert all(t > 0 for t in times) and times[best] == min(times)
    assert pkg.paam_rta_get_launch_config(b) == best
    first, cand = pkg.search(ctx(), b, r)
    torch.cuda.synchronize()
    ref = oracle.search(sy, ranks, threads=8)
    assert np.array_equal(cand.cpu().numpy(), ref["cand_ok"])
    assert np.array_equal(first.cpu().numpy(), ref["first_ok"])
    b.free()


def test_safe_blocking_every_launch_config():
    """The safe reading of Lemma 4 (blocking_mode 1) in the register-table
    kernel, with the int64 kernel for systems over 16 chains or outside the
    32-bit bound, in every launch configuration, against the oracle."""
    import torch

    import paper_2404_06452_gb300 as pkg

    p = dict(n_buckets=2, eps=1_500, kappa=300)
    for sy in (g.generate("cfg2", n_sys=20_000, p_spin=0.5), g.generate("cfg3", n_sys=6_000, seed=8)):
        ref = oracle.analyze(sy, blocking_mode=1, threads=8, **p)
        b = pkg.paam_rta_load_systems(ctx(), sy)
        for i in range(pkg.paam_rta_num_launch_configs()):
            pkg.paam_rta_set_launch_config(b, i)
            assert_same(analyze_poisoned(ctx(), b, blocking_mode=1, **p), ref)
        b.free()
