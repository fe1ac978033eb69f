"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

- hand-derived worked examples (tests/golden/hand_cases.json);
- closed form of a lone chain (Eqs. 1, 3, 4, 6 with no interferer);
- an independent brute-force least-fixed-point scan (oracle/lfp_scan.py);
- monotonicity and relabelling invariance of the bound;
- a discrete-event simulation of the run-time rules R1-R4: the bound is never
  below an observed response where the paper's blocking term applies.
"""
import json
import os
import random

import numpy as np
import pytest

import oracle
import paam_gen as g
from oracle import des_sim, lfp_scan
from paam_gen import tiny

HERE = os.path.dirname(os.path.abspath(__file__))


def _hand_cases():
    with open(os.path.join(HERE, "golden", "hand_cases.json")) as f:
        return json.load(f)["cases"]


def _sys_from_case(case):
    chains = [dict(T=c["T"], D=c["D"], prio=c["prio"], exec=c["exec"], spin=c["spin"],
                   cbs=[(e, list(a)) for e, a in c["cbs"]]) for c in case["system"]["chains"]]
    return dict(chains=chains, execs=[dict(x) for x in case["system"]["execs"]])


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(case):
    d = _sys_from_case(case)
    p = case["params"]
    out = oracle.analyze(tiny.to_systems([d]), aux=True, **p)
    assert out["R"].tolist() == case["R"]
    assert out["status"].tolist() == case["status"]
    assert out["verdict"].tolist() == [int(all(s == 0 for s in case["status"]))]
    for k, v in case.get("aux", {}).items():
        col = oracle.AUX_FIELDS.index(k)
        assert out["aux"][:, col].tolist() == v, k
    # the independent scan agrees on every hand case too
    R, st = lfp_scan.scan_system(d, **p)
    assert R == case["R"] and st == case["status"]


def test_lone_chain_closed_form():
    sy = g.generate("cfg2", n_sys=3000, n_min=1, n_max=1, p_acc=0.6, seg_per_cb=2, util_mode=0,
                    util_lo=0.05, util_hi=1.2, d_lo=0.3, d_hi=1.0)
    for eps, kappa in [(0, 0), (391_000, 129_180), (7, 3)]:
        out = oracle.analyze(sy, eps=eps, kappa=kappa, n_buckets=3)
        E = np.add.reduceat(sy.E, sy.chain_cb_off[:-1]) if sy.n_cb else np.zeros(sy.n_chain)
        segs = sy.cb_seg_off[sy.chain_cb_off]
        delta = np.diff(segs)
        Asum = np.array([sy.A[segs[c]:segs[c + 1]].sum() for c in range(sy.n_chain)])
        bound = E + Asum + delta * (2 * kappa + eps)
        sched = bound <= sy.D
        assert np.array_equal(out["status"] == 0, sched)
        assert np.array_equal(out["R"][sched], bound[sched])
        assert np.all(out["R"][~sched] == -1) and np.all(out["status"][~sched] == 1)
        assert sched.any() and (~sched).any()


def test_no_accelerator_no_overhead_dependence():
    """With no accelerator segment, eps, kappa and the bucket count cannot matter (Eq. 6 -> Eq. 5)."""
    sy = g.generate("cfg2", n_sys=2000, p_acc=0.0, p_spin=0.5)
    a = oracle.analyze(sy)
    b = oracle.analyze(sy, eps=5_000_000, kappa=3_000_000, n_buckets=4)
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["status"], b["status"])


def test_bruteforce_scan_agrees():
    rng = random.Random(20240406)
    n_checked = 0
    for trial in range(3000):
        d = tiny.tiny_system(rng, n_max=5, cb_max=3, x_max=3, exec_per_core=rng.choice([1, 2, 3]),
                             periods=tuple(range(6, 61)), e_max=8, a_max=8, p_seg=0.6, p_spin=0.4,
                             seg_max=2)
        p = dict(n_buckets=rng.choice([1, 2, 3, 6]), eps=rng.choice([0, 1, 2]), kappa=rng.choice([0, 1]))
        R, st = lfp_scan.scan_system(d, **p)
        out = oracle.analyze(tiny.to_systems([d]), **p)
        assert out["R"].tolist() == R, (d, p)
        assert out["status"].tolist() == st, (d, p)
        n_checked += len(R)
    assert n_checked > 5000


def test_bruteforce_scan_agrees_safe_blocking():
    """The safe blocking reading (blocking_mode=1) evaluated twice: the C
    oracle against the brute-force scan, which takes each lower-priority
    callback's hold from its own per-segment least fixed points.  Systems have
    several callbacks per chain and several segments per callback, so the
    longest-callback maximum, eps per segment and unbounded segments all
    occur."""
    rng = random.Random(20240407)
    n_checked = n_differs = n_unbounded = 0
    for trial in range(3000):
        d = tiny.tiny_system(rng, n_max=5, n_min=2, cb_max=3, x_max=2, exec_per_core=rng.choice([1, 2]),
                             periods=tuple(range(6, 41)), e_max=6, a_max=6, p_seg=0.6, p_spin=0.4,
                             seg_max=rng.choice([2, 3]), n_acc=rng.choice([1, 1, 2]))
        p = dict(n_buckets=rng.choice([1, 2, 3]), eps=rng.choice([0, 1, 2]), kappa=rng.choice([0, 1]))
        R, st = lfp_scan.scan_system(d, blocking_mode=1, **p)
        out = oracle.analyze(tiny.to_systems([d]), blocking_mode=1, aux=True, **p)
        assert out["R"].tolist() == R, (d, p)
        assert out["status"].tolist() == st, (d, p)
        lit = oracle.analyze(tiny.to_systems([d]), aux=True, **p)
        col = oracle.AUX_FIELDS.index("B")
        n_differs += int(np.any(out["aux"][:, col] != lit["aux"][:, col]))
        n_unbounded += int(np.any(out["aux"][:, col] == np.iinfo(np.int64).max))
        n_checked += len(R)
    assert n_checked > 8000 and n_differs > 800 and n_unbounded > 50, (n_checked, n_differs, n_unbounded)


def test_monotone_in_wcets_and_overheads():
    sy = g.generate("cfg2", n_sys=3000, p_spin=0.5)
    base = oracle.analyze(sy, eps=10_000, kappa=5_000, n_buckets=2)
    variants = []
    up = dict(sy.__dict__)
    E2 = sy.E.copy(); E2[::7] += 400_000
    variants.append((g.Systems(**dict(up, E=E2)), dict(eps=10_000, kappa=5_000, n_buckets=2)))
    A2 = sy.A.copy(); A2[::5] += 300_000
    variants.append((g.Systems(**dict(up, A=A2)), dict(eps=10_000, kappa=5_000, n_buckets=2)))
    variants.append((sy, dict(eps=200_000, kappa=5_000, n_buckets=2)))
    variants.append((sy, dict(eps=10_000, kappa=90_000, n_buckets=2)))
    for sy2, p in variants:
        o = oracle.analyze(sy2, **p)
        both = (base["status"] == 0) & (o["status"] == 0)
        assert np.all(o["R"][both] >= base["R"][both])
        # never turns a non-schedulable chain schedulable
        assert not np.any((base["status"] != 0) & (o["status"] == 0))
        assert np.all(o["verdict"] <= base["verdict"])


def test_relabelling_invariance():
    sy = g.generate("cfg2", n_sys=500, p_spin=0.5)
    base = oracle.analyze(sy, eps=1000, kappa=100, n_buckets=3)
    rng = np.random.default_rng(7)
    # permute chains (with their callbacks) and executor indices inside every system
    perm_chain, new = [], dict(T=[], D=[], prio=[], exec=[], spin=[], E=[], A=[], acc=[], core=[], xprio=[])
    cb_counts, seg_counts, chain_counts, x_counts = [], [], [], []
    for s in range(sy.n_sys):
        c0, c1 = sy.sys_chain_off[s], sy.sys_chain_off[s + 1]
        x0, x1 = sy.sys_exec_off[s], sy.sys_exec_off[s + 1]
        pc = rng.permutation(c1 - c0)
        px = rng.permutation(x1 - x0)  # new executor j is old executor px[j]
        inv_px = np.argsort(px)
        for j in range(x1 - x0):
            new["core"].append(sy.exec_core[x0 + px[j]]); new["xprio"].append(sy.exec_prio[x0 + px[j]])
        x_counts.append(x1 - x0)
        for k in pc:
            c = c0 + k
            perm_chain.append(c)
            new["T"].append(sy.T[c]); new["D"].append(sy.D[c]); new["prio"].append(sy.prio[c])
            new["exec"].append(inv_px[sy.exec[c]]); new["spin"].append(sy.spin[c])
            b0, b1 = sy.chain_cb_off[c], sy.chain_cb_off[c + 1]
            cb_counts.append(b1 - b0)
            for b in range(b0, b1):
                new["E"].append(sy.E[b])
                q0, q1 = sy.cb_seg_off[b], sy.cb_seg_off[b + 1]
                seg_counts.append(q1 - q0)
                new["A"].extend(sy.A[q0:q1]); new["acc"].extend(sy.acc[q0:q1])
        chain_counts.append(c1 - c0)
    off = lambda v: np.concatenate([[0], np.cumsum(v)]).astype(np.int64)
    sy2 = g.Systems(off(chain_counts), off(cb_counts), off(seg_counts), np.array(new["T"], np.int64),
                    np.array(new["D"], np.int64), np.array(new["prio"], np.int32),
                    np.array(new["exec"], np.int32), np.array(new["spin"], np.uint8),
                    np.array(new["E"], np.int64), np.array(new["A"], np.int64), np.array(new["acc"], np.int32),
                    off(x_counts), np.array(new["core"], np.int32), np.array(new["xprio"], np.int32))
    o = oracle.analyze(sy2, eps=1000, kappa=100, n_buckets=3)
    pc = np.array(perm_chain)
    assert np.array_equal(o["R"], base["R"][pc])
    assert np.array_equal(o["status"], base["status"][pc])
    assert np.array_equal(o["verdict"], base["verdict"])


def test_derived_executor_priority_matches_capa_generator():
    sy = g.generate("cfg2", n_sys=1000)
    a = oracle.analyze(sy)
    b = oracle.analyze(sy, derive_exec_prio=True)
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["status"], b["status"])


def test_des_single_chain_equals_wcet_sum():
    rng = random.Random(3)
    n = 0
    while n < 40:
        d = tiny.tiny_system(rng, n_min=1, n_max=1, cb_max=3, x_max=1, seg_max=2)
        eps, kappa = rng.choice([0, 1]), rng.choice([0, 1])
        c = d["chains"][0]
        total = sum(e for e, _ in c["cbs"]) + sum(a + 2 * kappa + eps for _, ss in c["cbs"] for a in ss)
        if total > c["T"]:  # jobs would back up; the closed form is for one job at a time
            continue
        obs = des_sim.explore(d, eps=eps, kappa=kappa)
        assert obs == [total]
        n += 1


def _lp_same_exec_has_segments(d, c):
    ch = d["chains"]
    return any(ch[l]["exec"] == ch[c]["exec"] and ch[l]["prio"] < ch[c]["prio"] and
               any(ss for _, ss in ch[l]["cbs"]) for l in range(len(ch)))


def test_des_never_exceeds_bound():
    """Bound >= max observed response for every chain of a schedulable system,
    wherever the paper's blocking term (Lemma 4) covers the executor's LP work."""
    rng = random.Random(11)
    checked, literal_gaps = 0, 0
    for trial in range(1000):
        d = tiny.tiny_system(rng, n_max=3, cb_max=2, x_max=2, exec_per_core=2, periods=(4, 6, 8, 12),
                             e_max=2, a_max=2, p_seg=0.5, p_spin=0.5)
        p = dict(n_buckets=rng.choice([1, 2]), eps=rng.choice([0, 1]), kappa=rng.choice([0, 1]))
        out = oracle.analyze(tiny.to_systems([d]), **p)
        if not out["verdict"][0]:
            continue
        obs = des_sim.explore(d, **p)
        for c, (r, o) in enumerate(zip(out["R"].tolist(), obs)):
            if _lp_same_exec_has_segments(d, c):
                literal_gaps += int(o > r)
                continue
            assert o <= r, (d, p, c, r, o)
            checked += 1
    assert checked > 300


def test_des_never_exceeds_safe_bound():
    """The safe blocking reading (blocking_mode=1: a lower-priority callback
    holds the executor for its CPU work and for each of its accelerator
    requests, bounded by Lemma 2 plus eps) covers every observed response,
    including where Lemma 4 as printed does not."""
    rng = random.Random(12)
    checked, exposed = 0, 0
    for trial in range(3000):
        d = tiny.tiny_system(rng, n_max=3, cb_max=2, x_max=2, exec_per_core=2, periods=(4, 6, 8, 12),
                             e_max=2, a_max=2, p_seg=0.5, p_spin=0.5)
        p = dict(n_buckets=rng.choice([1, 2]), eps=rng.choice([0, 1]), kappa=rng.choice([0, 1]))
        out = oracle.analyze(tiny.to_systems([d]), blocking_mode=1, **p)
        if not out["verdict"][0]:
            continue
        obs = des_sim.explore(d, **p)
        for c, (r, o) in enumerate(zip(out["R"].tolist(), obs)):
            assert o <= r, (d, p, c, r, o)
            checked += 1
            exposed += int(_lp_same_exec_has_segments(d, c))
    assert checked > 1000 and exposed > 60, (checked, exposed)


def test_safe_blocking_relations():
    """Without accelerator segments the two readings coincide; with them the
    safe bound is never below the literal one, and admits no more systems."""
    sy = g.generate("cfg2", n_sys=3000, p_acc=0.0, p_spin=0.5)
    a, b = oracle.analyze(sy), oracle.analyze(sy, blocking_mode=1)
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["status"], b["status"])
    sy = g.generate("cfg1", n_sys=3000, p_spin=0.5, util_lo=0.2, util_hi=0.2)
    for p in (dict(), dict(eps=391_000, kappa=129_180, n_buckets=2)):
        a, b = oracle.analyze(sy, aux=True, **p), oracle.analyze(sy, blocking_mode=1, aux=True, **p)
        both = (a["status"] == 0) & (b["status"] == 0)
        assert np.all(b["R"][both] >= a["R"][both])
        assert np.all(a["verdict"] >= b["verdict"])
        B = oracle.AUX_FIELDS.index("B")
        assert np.all(b["aux"][:, B] >= a["aux"][:, B]) and np.any(b["aux"][:, B] > a["aux"][:, B])
        assert b["verdict"].mean() > 0.05


def test_des_witness_literal_blocking_gap():
    """A finding about Lemma 4 used inside Theorem 1: B_c counts only the CPU
    WCET of one lower-priority callback, but that callback keeps the
    single-threaded executor while its accelerator request is handled.  Here
    the low chain (E=2, one segment A=1, eps=1) holds the executor for up to
    4 units, so the high chain can respond after 4 > bound 3."""
    d = dict(chains=[dict(T=6, D=6, prio=1, exec=1, spin=0, cbs=[(1, [])]),
                     dict(T=6, D=6, prio=0, exec=1, spin=1, cbs=[(2, [1])])],
             execs=[dict(core=0, prio=-1), dict(core=0, prio=1)])
    p = dict(n_buckets=1, eps=1, kappa=0)
    out = oracle.analyze(tiny.to_systems([d]), **p)
    assert out["R"].tolist()[0] == 3 and out["verdict"][0] == 1
    assert des_sim.explore(d, **p)[0] == 4
    # the safe reading: B = E + (h + eps) = 2 + (1 + 1) = 4 for the low chain's
    # one callback (its segment's Lemma 2 bound is h = A* = 1), so R = 4 + 1 = 5
    safe = oracle.analyze(tiny.to_systems([d]), blocking_mode=1, aux=True, **p)
    assert safe["R"].tolist()[0] == 5 and safe["aux"][0, oracle.AUX_FIELDS.index("B")] == 4
