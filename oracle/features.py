"""Surrogate input features in float64 -- TEST INFRASTRUCTURE ONLY.

Restates, for one (system, priority order), the 16 per-chain ratios the
surrogate network reads (the definitions are listed in the library header):
CPU and accelerator utilisation, deadline ratio, period spread, priority
rank, segment count, largest callback and request relative to the deadline,
the utilisation of each interferer class of Theorem 1 (hp, hpp) and of Eq. 3
(hps), the blocking terms of Lemma 4 and Eq. 3 relative to the deadline,
own demand, and one job of every CPU interferer.  Plain Python loops over
chains; shares no code with the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np

NCH, NF = 64, 16


def _system_tables(sy, s, kappa):
    c0, c1 = int(sy.sys_chain_off[s]), int(sy.sys_chain_off[s + 1])
    x0 = int(sy.sys_exec_off[s])
    ch = []
    for g in range(c0, c1):
        b0, b1 = int(sy.chain_cb_off[g]), int(sy.chain_cb_off[g + 1])
        Es = [float(e) for e in sy.E[b0:b1]]
        q0, q1 = int(sy.cb_seg_off[b0]), int(sy.cb_seg_off[b1])
        As = [float(a) + 2.0 * kappa for a in sy.A[q0:q1]]
        x = int(sy.exec[g])
        ch.append(dict(T=float(sy.T[g]), D=float(sy.D[g]), E=sum(Es), Emax=max(Es, default=0.0), S=sum(As),
                       M=max(As, default=0.0), dl=len(As), exec=x, core=int(sy.exec_core[x0 + x]),
                       given_eprio=None if sy.exec_prio is None else int(sy.exec_prio[x0 + x]),
                       given_prio=int(sy.prio[g])))
    return ch


def system_features(sy, s, rank_row=None, n_buckets=1, kappa=0):
    """[64 * 16] float64 features of system s under the priority order
    rank_row (0 = highest; None = the system's own priorities)."""
    ch = _system_tables(sy, s, kappa)
    n = len(ch)
    out = np.zeros(NCH * NF)
    if n == 0:
        return out
    if rank_row is None:
        prio = [c["given_prio"] for c in ch]
        derived = sy.exec_prio is None
    else:
        prio = [n - 1 - int(rank_row[c]) for c in range(n)]
        derived = True
    if derived:  # criticality-as-priority executor priorities
        eprio = [max(prio[k] for k in range(n) if ch[k]["exec"] == ch[c]["exec"]) for c in range(n)]
    else:
        eprio = [c["given_eprio"] for c in ch]
    users = [c for c in range(n) if ch[c]["dl"] > 0]
    bucket = {}
    for c in users:
        r = sum(1 for u in users if prio[u] > prio[c])
        bucket[c] = (r * n_buckets) // len(users)
    Tmin = min(c["T"] for c in ch)
    for c in range(n):
        a = ch[c]
        higher = [h for h in range(n) if h != c and prio[h] > prio[c]]
        hp = [h for h in higher if ch[h]["exec"] == a["exec"]]
        hpp = [h for h in range(n) if ch[h]["exec"] != a["exec"] and ch[h]["core"] == a["core"] and eprio[h] > eprio[c]]
        hps = [h for h in higher if ch[h]["dl"] > 0]
        lp_x = [l for l in range(n) if l != c and ch[l]["exec"] == a["exec"] and prio[l] < prio[c]]
        B = max([ch[l]["Emax"] for l in lp_x], default=0.0)
        blk = 0.0
        if c in bucket:
            blk = max([ch[l]["M"] for l in users if prio[l] < prio[c] and bucket[l] == bucket[c]], default=0.0)
        f = [a["E"] / a["T"], a["S"] / a["T"], a["D"] / a["T"], math.log2(a["T"] / Tmin) / 4.0,
             len(higher) / n, min(a["dl"], 16) / 16.0, a["Emax"] / a["D"], a["M"] / a["D"],
             sum((ch[h]["E"] + ch[h]["S"]) / ch[h]["T"] for h in hp),
             sum(ch[h]["E"] / ch[h]["T"] for h in hpp),
             sum(ch[h]["S"] / ch[h]["T"] for h in hps),
             B / a["D"], blk / a["D"], (a["E"] + a["S"]) / a["D"],
             sum(ch[h]["E"] + ch[h]["S"] for h in hp + hpp) / a["D"], 1.0]
        out[c * NF:(c + 1) * NF] = np.clip(f, 0.0, 8.0)
    return out


def features(sy, ranks=None, n_buckets=1, kappa=0, systems=None):
    """Rows system * K + candidate (K = 1 without ranks) for the given systems."""
    systems = range(sy.n_sys) if systems is None else systems
    rows = []
    for s in systems:
        if ranks is None:
            rows.append(system_features(sy, s, None, n_buckets, kappa))
        else:
            for k in range(ranks.shape[1]):
                rows.append(system_features(sy, s, ranks[s, k], n_buckets, kappa))
    return np.array(rows)
