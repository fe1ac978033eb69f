"""The iteration bound that ``paam_rta_load_systems`` enforces.

Every recurrence of Eqs. 3 and 6 starts at or below its least fixed point,
so it rises strictly until it converges or passes its deadline.  After its
first step it can rise again only when one of the arrival counts
ceil(t / T_h) + 1 of Lemma 1 has grown, and while t stays at or below the
system's largest deadline Dmax that happens at most ceil(Dmax / T_h) times per
chain h.  So no recurrence takes more than L = sum_h ceil(Dmax / T_h) + 2
evaluations.  These tests check the bound against the oracle's own counts,
with the bound computed here from its definition.
"""
import random

import numpy as np
import pytest

import oracle
import paam_gen as g
from paam_gen import tiny


def _bound(sy):
    n = np.diff(sy.sys_chain_off)
    sys_of = np.repeat(np.arange(sy.n_sys), n)
    dmax = np.zeros(sy.n_sys, np.int64)
    np.maximum.at(dmax, sys_of, sy.D)
    terms = -(-dmax[sys_of] // sy.T)  # ceil(Dmax / T_h) per chain h
    L = np.zeros(sy.n_sys, np.int64)
    np.add.at(L, sys_of, terms)
    return L + 2


@pytest.mark.parametrize("cfg,p", [("cfg2", dict()), ("cfg3", dict(n_buckets=2, eps=198_000, kappa=41_210)),
                                   ("cfg1", dict(eps=391_000, kappa=129_180))])
@pytest.mark.parametrize("blocking_mode", [0, 1])
def test_bound_covers_oracle_iterations(cfg, p, blocking_mode):
    sy = g.generate(cfg) if cfg == "cfg1" else g.generate(cfg, n_sys=20000)
    it = oracle.iterations(sy, blocking_mode=blocking_mode, threads=8, **p)
    L = _bound(sy)
    assert np.all(it["max_loop"] <= L), np.nonzero(it["max_loop"] > L)[0][:5]
    assert it["max_loop"].max() >= 4


def test_bound_covers_iteration_heavy_tiny_systems():
    """Short periods against long deadlines: many arrivals per window, so the
    recurrences take many steps, and the bound is approached."""
    rng = random.Random(31)
    dicts = []
    for _ in range(4000):
        d = tiny.tiny_system(rng, n_max=5, n_min=2, cb_max=3, x_max=2, exec_per_core=2,
                             periods=(1, 2, 3, 5, 40, 60, 90), e_max=2, a_max=2, p_seg=0.5, p_spin=0.5,
                             seg_max=2)
        for ch in d["chains"]:
            if ch["T"] <= 5:  # keep short-period chains light so long windows can converge
                ch["cbs"] = [(rng.randint(0, 1) if ch["T"] >= 3 else 0, [] if ch["T"] < 3 else s)
                             for _, s in ch["cbs"][:1]]
        dicts.append(d)
    sy = tiny.to_systems(dicts)
    L = _bound(sy)
    best = 0.0
    for mode in (0, 1):
        for p in (dict(), dict(eps=1, kappa=0, n_buckets=2)):
            it = oracle.iterations(sy, blocking_mode=mode, **p)
            assert np.all(it["max_loop"] <= L)
            best = max(best, float((it["max_loop"] / L).max()))
    assert it["max_loop"].max() >= 20
    assert best > 0.5, best  # the bound is not vacuous on these systems
