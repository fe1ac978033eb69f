"""End-to-end bounds of chains spanning several executors -- TEST INFRASTRUCTURE ONLY.

Sec. IV-F: the end-to-end latency of a chain made of sub-chains, each run by
its own executor, is the sum of the sub-chains' response times plus the
communication cost between them; read as one cost eps' per hand-over:
R* = sum_c R_c + (m - 1) eps'.  The chain is schedulable when every sub-chain
is (status 0) and R* <= D*; otherwise R* = -1 and the status is 2 (DEP) if a
sub-chain is DEP, else 1 (OVERRUN).  Plain loops; shares no code with the
CUDA path.
"""
from __future__ import annotations

import numpy as np

SCHED, OVERRUN, DEP = 0, 1, 2


def end_to_end(R, status, e2e_off, e2e_chain, D_e2e, eps_prime: int):
    n = len(D_e2e)
    R_out = np.full(n, -1, np.int64)
    st_out = np.full(n, OVERRUN, np.uint8)
    for e in range(n):
        subs = [int(c) for c in e2e_chain[int(e2e_off[e]):int(e2e_off[e + 1])]]
        sts = [int(status[c]) for c in subs]
        if any(s == DEP for s in sts):
            st_out[e] = DEP
            continue
        if any(s != SCHED for s in sts):
            continue
        total = sum(int(R[c]) for c in subs) + max(len(subs) - 1, 0) * int(eps_prime)
        if total <= int(D_e2e[e]):
            R_out[e] = total
            st_out[e] = SCHED
    return R_out, st_out
