"""Several accelerators per system (rule R1) on the GPU against the oracle:
bit-exact R, status and verdict, in both blocking readings and in the
priority search."""
import random

import numpy as np
import pytest

import oracle
import paam_gen as g
from paam_gen import tiny

from gpu_util import analyze_poisoned, assert_same, ctx, gpu_analyze

pytestmark = pytest.mark.gpu
PARAMS = [dict(n_buckets=1, eps=0, kappa=0), dict(n_buckets=2, eps=391_000, kappa=129_180)]


@pytest.mark.parametrize("p", PARAMS)
def test_wfd_units_match_oracle(p):
    for sy in (g.assign_accelerators(g.generate("cfg2", n_sys=100_000, p_spin=0.2), 3),
               g.assign_accelerators(g.generate("cfg3", n_sys=30_000, seed=41), 2)):
        assert sy.acc.max() > 0
        assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, threads=8, **p))


def test_three_accelerators_full_size():
    """The 1,000,000-system workload with its segments spread over three
    accelerator units by WFD (the benchmark's several-accelerator case), every
    chain compared bit-exactly."""
    import os

    sy = g.assign_accelerators(g.generate("cfg2"), 3)
    p = PARAMS[1]
    assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, threads=os.cpu_count() or 8, **p))


def test_tiny_systems_four_accelerators():
    rng = random.Random(42)
    dicts = [tiny.tiny_system(rng, n_max=6, cb_max=3, x_max=3, n_acc=4, seg_max=2, p_seg=0.6,
                              periods=tuple(range(20, 200)), e_max=20, a_max=20) for _ in range(3000)]
    sy = tiny.to_systems(dicts)
    for p in PARAMS + [dict(n_buckets=3, eps=2, kappa=1)]:
        assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, threads=8, **p))


def test_safe_mode_and_search_with_several_accelerators():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.assign_accelerators(g.generate("cfg2", n_sys=30_000, p_spin=0.3), 4)
    for p in PARAMS:
        assert_same(gpu_analyze(sy, blocking_mode=1, **p), oracle.analyze(sy, blocking_mode=1, threads=8, **p))
    s4 = g.assign_accelerators(g.generate("cfg4s", n_sys=200), 2)
    ranks = g.candidate_ranks(s4, 24, 3)
    b = pkg.paam_rta_load_systems(ctx(), s4)
    first, cand = pkg.search(ctx(), b, torch.from_numpy(ranks).cuda(), n_buckets=2)
    torch.cuda.synchronize()
    ref = oracle.search(s4, ranks, n_buckets=2, threads=8)
    assert np.array_equal(cand.cpu().numpy(), ref["cand_ok"]) and np.array_equal(first.cpu().numpy(), ref["first_ok"])
    b.free()


def test_one_accelerator_under_another_index_and_bad_index():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg2", n_sys=20_000, p_spin=0.3)
    base = gpu_analyze(sy, n_buckets=2, eps=1_000)
    moved = g.Systems(**{**sy.__dict__, "acc": np.full_like(sy.acc, 2)})  # tables for three accelerators
    assert_same(gpu_analyze(moved, n_buckets=2, eps=1_000), {k: base[k] for k in ("R", "status", "verdict")})
    bad = g.Systems(**{**sy.__dict__, "acc": np.where(np.arange(len(sy.acc)) == 5, 4, 0).astype(np.int32)})
    with pytest.raises(pkg.PaamError):
        pkg.paam_rta_load_systems(ctx(), bad)


def test_every_launch_config_with_several_accelerators():
    """The register-table kernel with per-accelerator tables (systems of up to
    16 chains inside the 32-bit bound) and the int64 kernel for the rest give
    the oracle's results in every launch configuration (static shares, work
    queue, size order), with several buckets."""
    import torch

    import paper_2404_06452_gb300 as pkg

    mixed = g.assign_accelerators(g.generate("cfg3", n_sys=20_000, seed=5), 3)  # 2-64 chains: both kernels
    sy2 = g.assign_accelerators(g.generate("cfg2", n_sys=20_000, p_spin=0.4), 2)
    for sy in (mixed, sy2):
        p = dict(n_buckets=3, eps=2_000, kappa=700)
        ref = oracle.analyze(sy, threads=8, **p)
        b = pkg.paam_rta_load_systems(ctx(), sy)
        for i in range(pkg.paam_rta_num_launch_configs()):
            pkg.paam_rta_set_launch_config(b, i)
            assert_same(analyze_poisoned(ctx(), b, **p), ref)
        b.free()

