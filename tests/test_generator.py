"""The seeded generator: determinism, thread independence and workload shape."""
import numpy as np

import paam_gen as g

FIELDS = ["sys_chain_off", "chain_cb_off", "cb_seg_off", "T", "D", "prio", "exec", "spin", "E", "A",
          "acc", "sys_exec_off", "exec_core", "exec_prio"]


def test_thread_count_independent():
    a = g.generate("cfg3", n_sys=3000, threads=1)
    b = g.generate("cfg3", n_sys=3000, threads=7)
    for f in FIELDS:
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_prefix_is_stable():
    a = g.generate("cfg2", n_sys=500)
    b = g.generate("cfg2", n_sys=2000)
    assert np.array_equal(a.T, b.T[: a.n_chain])


def test_cfg_shapes():
    s = g.generate("cfg2", n_sys=5000)
    n = s.chains_per_system()
    assert n.min() >= 8 and n.max() <= 16
    ncb = np.diff(s.chain_cb_off)
    assert ncb.min() >= 3 and ncb.max() <= 8
    assert np.all(np.diff(s.sys_exec_off) == 4)
    assert np.all((s.T >= 10_000_000) & (s.T <= 100_000_000)) and np.array_equal(s.T, s.D)
    assert np.all((s.A >= 100_000) & (s.A <= 2_000_000))
    frac = s.n_seg / s.n_cb
    assert 0.47 < frac < 0.53
    for i in range(0, 5000, 997):  # priorities are a permutation per system
        c0, c1 = s.sys_chain_off[i], s.sys_chain_off[i + 1]
        assert sorted(s.prio[c0:c1].tolist()) == list(range(c1 - c0))
    s3 = g.generate("cfg3", n_sys=20000)
    n3 = s3.chains_per_system()
    assert n3.min() >= 2 and n3.max() <= 64 and 9.0 < n3.mean() < 11.0


def test_subset_roundtrip():
    s = g.generate("cfg3", n_sys=400)
    idx = np.array([5, 0, 399, 17])
    sub = s.subset(idx)
    assert sub.n_sys == 4
    for k, i in enumerate(idx):
        c0, c1 = s.sys_chain_off[i], s.sys_chain_off[i + 1]
        d0, d1 = sub.sys_chain_off[k], sub.sys_chain_off[k + 1]
        assert np.array_equal(s.T[c0:c1], sub.T[d0:d1])
        b0, b1 = s.chain_cb_off[c0], s.chain_cb_off[c1]
        e0, e1 = sub.chain_cb_off[d0], sub.chain_cb_off[d1]
        assert np.array_equal(s.E[b0:b1], sub.E[e0:e1])
        q0, q1 = s.cb_seg_off[b0], s.cb_seg_off[b1]
        r0, r1 = sub.cb_seg_off[e0], sub.cb_seg_off[e1]
        assert np.array_equal(s.A[q0:q1], sub.A[r0:r1])


def test_permutations():
    n = np.array([4, 16, 1], np.int32)
    p = g.permutations(123, n, K=5, nmax=16, first_slot=2)
    assert p.shape == (3, 5, 16)
    assert np.all(p[:, :2] == 0)
    for s in range(3):
        for k in range(2, 5):
            assert sorted(p[s, k, : n[s]].tolist()) == list(range(n[s]))
            assert np.all(p[s, k, n[s]:] == -1)


def test_candidate_ranks():
    import oracle

    sy = g.generate("cfg3", n_sys=300)
    r = g.candidate_ranks(sy, 6, 9, nmax=64)
    n = sy.chains_per_system()
    for s in range(0, 300, 37):
        c0 = sy.sys_chain_off[s]
        for k in range(6):
            assert sorted(r[s, k, : n[s]].tolist()) == list(range(n[s]))
            assert np.all(r[s, k, n[s]:] == -1)
        # slot 0 follows the given priorities, slot 1 the deadlines
        assert np.all(np.argsort(r[s, 0, : n[s]]) == np.argsort(-sy.prio[c0:c0 + n[s]], kind="stable"))
        assert np.all(np.diff(sy.D[c0:c0 + n[s]][np.argsort(r[s, 1, : n[s]])]) >= 0)
    # slot 0 is the plain analysis with criticality-as-priority executor priorities
    ref = oracle.search(sy, r[:, :1], threads=4)
    a = oracle.analyze(sy, derive_exec_prio=True, threads=4)
    assert np.array_equal(ref["cand_ok"][:, 0], a["verdict"])


def test_wfd_assignment_hand_case_and_balance():
    import numpy as np

    from paam_gen import tiny

    # one system: chain periods 10 and 20; segment utilisations 4/10, 1/10, 6/20, 5/20
    d = dict(chains=[dict(T=10, D=10, prio=1, exec=0, spin=0, cbs=[(1, [4, 1])]),
                     dict(T=20, D=20, prio=0, exec=0, spin=0, cbs=[(1, [6]), (1, [5])])],
             execs=[dict(core=0, prio=1)])
    out = g.assign_accelerators(tiny.to_systems([d]), 2)
    # decreasing: 0.4 (seg 0) -> unit 0; 0.3 (seg 2) -> unit 1; 0.25 (seg 3) -> unit 1 (0.3 < 0.4);
    # 0.1 (seg 1) -> unit 0 (0.4 < 0.55)
    assert out.acc.tolist() == [0, 0, 1, 1]
    sy = g.generate("cfg3", n_sys=300)
    for units in (2, 3, 5):
        acc = g.assign_accelerators(sy, units).acc
        for s in range(sy.n_sys):
            c0, c1 = sy.sys_chain_off[s], sy.sys_chain_off[s + 1]
            q0, q1 = sy.cb_seg_off[sy.chain_cb_off[c0]], sy.cb_seg_off[sy.chain_cb_off[c1]]
            if q1 == q0:
                continue
            chain_of = np.repeat(np.arange(c0, c1), np.diff(sy.cb_seg_off[sy.chain_cb_off[c0:c1 + 1]]))
            u = sy.A[q0:q1] / sy.T[chain_of]
            load = np.bincount(acc[q0:q1], weights=u, minlength=units)
            assert load.max() - load.min() <= u.max() + 1e-12
