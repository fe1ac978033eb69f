"""Pins of the end-to-end composition over sub-chains (Sec. IV-F) and of the
generator's split workload."""
import numpy as np

import oracle
import paam_gen as g
from oracle.end_to_end import DEP, OVERRUN, SCHED, end_to_end


def test_hand_cases():
    R = np.array([5, 7, -1, -1, 9], np.int64)
    st = np.array([SCHED, SCHED, OVERRUN, DEP, SCHED], np.uint8)
    off = np.array([0, 2, 4, 5, 5, 7], np.int64)       # {0,1}, {2,3}, {4}, {}, {0,4}
    chain = np.array([0, 1, 2, 3, 4, 0, 4], np.int64)
    D = np.array([14, 100, 9, 1, 15], np.int64)
    Rs, sts = end_to_end(R, st, off, chain, D, eps_prime=2)
    # 5 + 7 + one hand-over of 2 = 14 <= 14; DEP wins over OVERRUN; one sub-chain: R*
    # = R_c; an empty chain is 0; 5 + 9 + 2 = 16 > 15
    assert Rs.tolist() == [14, -1, 9, 0, -1]
    assert sts.tolist() == [SCHED, DEP, SCHED, SCHED, OVERRUN]
    Rs, sts = end_to_end(R, st, off, chain, D - 1, eps_prime=2)
    assert sts.tolist()[0] == OVERRUN and sts.tolist()[2] == OVERRUN


def test_split_workload_shape():
    sy = g.generate("cfg2", n_sys=2000)
    s2, off, chain, D = g.split_end_to_end(sy, 4)
    assert off[0] == 0 and off[-1] == s2.n_chain and np.all(np.diff(off) >= 1) and np.all(np.diff(off) <= 3)
    assert np.array_equal(chain, np.arange(s2.n_chain))
    sysid = np.repeat(np.arange(s2.n_sys), s2.chains_per_system())
    for e in range(0, len(D), 7):
        mem = chain[off[e]:off[e + 1]]
        assert len(set(sysid[mem])) == 1                 # within one system
        assert np.all(s2.T[mem] == D[e]) and np.all(s2.D[mem] == D[e])
        assert len(set(s2.exec[mem].tolist())) == len(mem)  # each sub-chain on its own executor
    assert np.any(np.diff(off) > 1)


def test_single_sub_chains_reduce_to_the_chain_bound():
    sy = g.generate("cfg2", n_sys=2000)
    s2, off, chain, D = g.split_end_to_end(sy, 4, max_sub=1)
    out = oracle.analyze(s2, threads=4)
    Rs, sts = end_to_end(out["R"], out["status"], off, chain, D, eps_prime=391_000)
    assert np.array_equal(Rs, out["R"]) and np.array_equal(sts, out["status"])
