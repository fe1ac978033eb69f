"""GPU vs CPU-oracle parity through the C ABI: bit-exact int64 R, status and
verdict on every workload shape and parameter set."""
import json
import os
import random

import numpy as np
import pytest

import oracle
import paam_gen as g
from paam_gen import tiny

from gpu_util import assert_same, ctx, gpu_analyze, oracle_on

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS = [dict(n_buckets=1, eps=0, kappa=0), dict(n_buckets=2, eps=391_000, kappa=129_180),
          dict(n_buckets=6, eps=198_000, kappa=0), dict(n_buckets=3, eps=0, kappa=41_210)]


def test_hand_cases():
    with open(os.path.join(HERE, "golden", "hand_cases.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        chains = [dict(T=c["T"], D=c["D"], prio=c["prio"], exec=c["exec"], spin=c["spin"],
                       cbs=[(e, list(a)) for e, a in c["cbs"]]) for c in case["system"]["chains"]]
        sy = tiny.to_systems([dict(chains=chains, execs=case["system"]["execs"])])
        out = gpu_analyze(sy, **case["params"])
        assert out["R"].tolist() == case["R"], case["name"]
        assert out["status"].tolist() == case["status"], case["name"]


@pytest.mark.parametrize("p", PARAMS)
def test_cfg1_full(p):
    sy = g.generate("cfg1")
    assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, **p))


@pytest.mark.parametrize("p", PARAMS)
def test_tiny_random_structures(p):
    rng = random.Random(99 + p["n_buckets"])
    dicts = [tiny.tiny_system(rng, n_max=8, cb_max=4, x_max=4, exec_per_core=rng.choice([1, 2, 3]),
                              periods=tuple(range(5, 200)), e_max=20, a_max=20, p_seg=0.5, p_spin=0.5,
                              seg_max=3) for _ in range(20000)]
    sy = tiny.to_systems(dicts)
    assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, **p))


def test_cfg1_shape_with_spin_and_random_executor_priorities():
    sy = g.generate("cfg2", n_sys=50000, p_spin=0.5, exec_prio_mode=1, x_min=2, x_max=8, exec_per_core=3)
    for p in PARAMS[:2]:
        assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, threads=8, **p))


def test_priorities_outside_zero_to_n():
    """Chain and executor priorities spread far beyond 0..n-1 (some negative) in
    every other system: only their order matters (Sec. II-A), so results equal
    those of the original permutations, and the oracle's, on both relation paths
    of the kernels (small priority values and general ones) within one launch."""
    import dataclasses

    sy = g.generate("cfg2", n_sys=20000, p_spin=0.3, exec_prio_mode=1, seed=41)
    far = np.repeat(np.arange(sy.n_sys) % 2 == 1, sy.chains_per_system())
    far_x = np.repeat(np.arange(sy.n_sys) % 2 == 1, np.diff(sy.sys_exec_off))
    prio = np.where(far, sy.prio.astype(np.int64) * 1_000_003 - 700_000_000, sy.prio).astype(np.int32)
    xprio = np.where(far_x, sy.exec_prio.astype(np.int64) * 999_983 - 5_000_000, sy.exec_prio).astype(np.int32)
    sy2 = dataclasses.replace(sy, prio=prio, exec_prio=xprio)
    for p in PARAMS[:2]:
        a, b = gpu_analyze(sy, **p), gpu_analyze(sy2, **p)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        assert_same(b, oracle.analyze(sy2, threads=8, **p))


def test_device_view_matches_host_view():
    sy = g.generate("cfg3", n_sys=20000)
    a = gpu_analyze(sy, n_buckets=2)
    b = gpu_analyze(sy, n_buckets=2, device_view=True)
    for k in a:
        assert np.array_equal(a[k], b[k])
    assert_same(a, oracle.analyze(sy, threads=8, n_buckets=2))


def test_cfg2_full_size():
    """The 1,000,000-system workload in the launch configuration the benchmark
    times (autotuned), compared bit-exactly on every chain."""
    sy = g.generate("cfg2")
    out = gpu_analyze(sy, autotune=True)
    assert_same(out, oracle.analyze(sy, threads=os.cpu_count() or 8))
    # every status value is legal and R is -1 exactly where not schedulable
    assert set(np.unique(out["status"]).tolist()) <= {0, 1, 2}
    assert np.all((out["R"] == -1) == (out["status"] != 0))
    # the analysis admits some chains but (with 8-16 chains per system) no whole system
    assert 0.05 < (out["status"] == 0).mean() < 0.95


def test_safe_blocking_full_size():
    """The 1,000,000-system workload under the safe reading of Lemma 4, with two
    buckets and both overheads: every segment bounded one per lane (no system
    has more than 128 segments), every chain compared bit-exactly."""
    sy = g.generate("cfg2")
    p = dict(n_buckets=2, eps=391_000, kappa=129_180)
    out = gpu_analyze(sy, blocking_mode=1, **p)
    assert_same(out, oracle.analyze(sy, blocking_mode=1, threads=os.cpu_count() or 8, **p))
    assert 0.005 < (out["status"] == 0).mean() < 0.5


def test_cfg3_full_size():
    """The 4,000,000-system uneven workload (2-64 chains), overheads on, every chain."""
    sy = g.generate("cfg3")
    p = dict(n_buckets=2, eps=198_000, kappa=41_210)
    out = gpu_analyze(sy, autotune=True, **p)
    assert_same(out, oracle.analyze(sy, threads=os.cpu_count() or 8, **p))
    n = sy.chains_per_system()
    assert n.max() == 64 and n.min() == 2


def test_edge_shapes():
    # empty systems, empty chains, 64 chains, a chain with 12 segments in one callback
    rng = random.Random(5)
    dicts = [dict(chains=[], execs=[dict(core=0, prio=0)])]
    dicts.append(dict(chains=[dict(T=10, D=10, prio=0, exec=0, spin=0, cbs=[])], execs=[dict(core=0, prio=0)]))
    dicts.append(tiny.tiny_system(rng, n_min=64, n_max=64, cb_max=3, x_max=8, periods=tuple(range(1000, 5000)),
                                  e_max=30, a_max=30, p_seg=0.5, seg_max=2))
    dicts.append(dict(chains=[dict(T=1, D=1, prio=5, exec=0, spin=1, cbs=[(0, [0] * 12)])],
                      execs=[dict(core=0, prio=0)]))
    dicts.append(tiny.tiny_system(rng, n_min=64, n_max=64, cb_max=12, x_max=8, periods=tuple(range(10**8, 10**9)),
                                  e_max=10**6, a_max=10**6, p_seg=0.5, seg_max=1))
    sy = tiny.to_systems(dicts)
    for p in PARAMS:
        assert_same(gpu_analyze(sy, **p), oracle.analyze(sy, **p))


def test_empty_batch():
    sy = tiny.to_systems([])
    out = gpu_analyze(sy)
    assert len(out["R"]) == 0 and len(out["verdict"]) == 0


def _expect_error(sy, code, **p):
    import paper_2404_06452_gb300 as pkg
    from gpu_util import ctx

    with pytest.raises(pkg.PaamError) as ei:
        b = pkg.paam_rta_load_systems(ctx(), sy)
        pkg.analyze(ctx(), b, **p)
    assert ei.value.code == code


def test_invalid_inputs_rejected():
    base = dict(chains=[dict(T=10, D=10, prio=1, exec=0, spin=0, cbs=[(2, [1])]),
                        dict(T=20, D=20, prio=0, exec=0, spin=0, cbs=[(3, [])])],
                execs=[dict(core=0, prio=1)])

    def mod(f):
        d = json.loads(json.dumps(base))
        f(d)
        for ch in d["chains"]:
            ch["cbs"] = [(e, a) for e, a in ch["cbs"]]
        return tiny.to_systems([d])

    _expect_error(mod(lambda d: d["chains"][0].update(D=11)), -1)      # D > T
    _expect_error(mod(lambda d: d["chains"][0].update(T=0, D=0)), -1)  # T <= 0
    _expect_error(mod(lambda d: d["chains"][1].update(prio=1)), -1)    # duplicate priority
    _expect_error(mod(lambda d: d["chains"][1].update(exec=3)), -1)    # executor out of range
    _expect_error(mod(lambda d: d["chains"][0].update(cbs=[(-1, [])])), -1)  # negative WCET
    sy = mod(lambda d: None)
    sy.acc = np.full_like(sy.acc, 4)
    _expect_error(sy, -1)                                              # accelerator index past PAAM_MAX_ACC
    big = mod(lambda d: d["chains"][0].update(T=2**40, D=2**40, cbs=[(2**40, [2**40] * 8)]))
    _expect_error(big, -2)                                             # int64 range
    _expect_error(mod(lambda d: None), -2, eps=2**33)                  # eps above the cap


@pytest.mark.parametrize("p", PARAMS[:2])
def test_safe_blocking_mode(p):
    """blocking_mode=1 (the safe reading of Lemma 4) on every shape: uneven
    sizes up to 64 chains, spinning chains, overheads, callbacks with two
    segments and systems of 40 to 192 segments (a quarter of them above 128,
    the most the register-table kernel bounds with one segment per lane; it
    takes those segment by segment); bit-exact with the oracle, and the search
    in the same mode."""
    import torch

    import paper_2404_06452_gb300 as pkg

    for sy in (g.generate("cfg1", p_spin=0.5), g.generate("cfg3", n_sys=3000, seed=31),
               g.generate("cfg2", n_sys=3000, p_spin=0.3, exec_prio_mode=1),
               g.generate("cfg2", n_sys=3000, seed=77, n_min=8, n_max=16, cb_min=3, cb_max=12, seg_per_cb=2,
                          p_acc=0.6, util_mode=0, util_lo=0.1, util_hi=0.5, a_min=10_000, a_max=200_000)):
        assert_same(gpu_analyze(sy, blocking_mode=1, **p), oracle.analyze(sy, blocking_mode=1, threads=8, **p))
    sy = g.generate("cfg4s", n_sys=200)
    ranks = g.candidate_ranks(sy, 24, 3)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    first, cand = pkg.search(ctx(), b, torch.from_numpy(ranks).cuda(), blocking_mode=1, **p)
    torch.cuda.synchronize()
    ref = oracle.search(sy, ranks, blocking_mode=1, threads=8, **p)
    assert np.array_equal(cand.cpu().numpy(), ref["cand_ok"])
    assert np.array_equal(first.cpu().numpy(), ref["first_ok"])
    b.free()
