"""Tiny small-integer systems (time unit 1) for exhaustive checks.

Used by the brute-force fixed-point scan and the discrete-event simulation,
which need periods, deadlines and execution times of a few units.  Pure
Python, seeded with ``random.Random``; holds no analysis arithmetic.
"""
from __future__ import annotations

import random

import numpy as np


def seg_parts(seg):
    """(A, accelerator) of a segment entry: an int A (accelerator 0) or a pair."""
    return (seg, 0) if isinstance(seg, int) else (int(seg[0]), int(seg[1]))


def tiny_system(rng: random.Random, n_max: int = 3, cb_max: int = 2, x_max: int = 2,
                exec_per_core: int = 2, periods=(4, 6, 8, 12), e_max: int = 3, a_max: int = 3,
                p_seg: float = 0.5, p_spin: float = 0.5, implicit_deadline: bool = False,
                n_min: int = 1, seg_max: int = 1, n_acc: int = 1):
    """One system as a dict of Python lists (local indices).  With n_acc > 1
    each segment is an (A, accelerator) pair, the accelerator uniform."""
    n = rng.randint(n_min, n_max)
    nx = rng.randint(1, x_max)
    prios = list(range(n))
    rng.shuffle(prios)
    chains = []
    for c in range(n):
        T = rng.choice(periods)
        D = T if implicit_deadline else rng.randint(max(1, T // 2), T)
        ncb = rng.randint(1, cb_max)
        cbs = []
        for _ in range(ncb):
            E = rng.randint(0, e_max)
            segs = [rng.randint(0, a_max) for _ in range(seg_max) if rng.random() < p_seg]
            if n_acc > 1:
                segs = [(a, rng.randrange(n_acc)) for a in segs]
            cbs.append((E, segs))
        chains.append(dict(T=T, D=D, prio=prios[c], exec=rng.randrange(nx),
                           spin=1 if rng.random() < p_spin else 0, cbs=cbs))
    execs = [dict(core=x // exec_per_core) for x in range(nx)]
    # CAPA executor priorities: the highest chain priority on the executor
    for x in range(nx):
        ps = [ch["prio"] for ch in chains if ch["exec"] == x]
        execs[x]["prio"] = max(ps) if ps else -(x + 1)
    return dict(chains=chains, execs=execs)


def to_systems(dicts):
    """Pack a list of tiny-system dicts into a ``paam_gen.Systems`` batch."""
    from . import Systems

    sc, cbo, so, xo = [0], [0], [0], [0]
    T, D, prio, ex, spin, E, A, acc, core, xprio = [], [], [], [], [], [], [], [], [], []
    for d in dicts:
        for ch in d["chains"]:
            T.append(ch["T"]); D.append(ch["D"]); prio.append(ch["prio"])
            ex.append(ch["exec"]); spin.append(ch["spin"])
            for (e, segs) in ch["cbs"]:
                E.append(e)
                for sg in segs:
                    a, u = seg_parts(sg)
                    A.append(a); acc.append(u)
                so.append(len(A))
            cbo.append(len(E))
        sc.append(len(T))
        for x in d["execs"]:
            core.append(x["core"]); xprio.append(x["prio"])
        xo.append(len(core))
    i64 = lambda v: np.asarray(v, np.int64)
    i32 = lambda v: np.asarray(v, np.int32)
    return Systems(i64(sc), i64(cbo), i64(so), i64(T), i64(D), i32(prio), i32(ex),
                   np.asarray(spin, np.uint8), i64(E), i64(A), i32(acc), i64(xo), i32(core), i32(xprio),
                   meta={"cfg": "tiny"})


def tiny_batch(seed: int, count: int, **kw):
    """``count`` tiny systems packed into one batch, plus their dict form."""
    rng = random.Random(seed)
    dicts = [tiny_system(rng, **kw) for _ in range(count)]
    return to_systems(dicts), dicts
