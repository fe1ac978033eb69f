"""Brute-force least-fixed-point scan of the PAAM bound -- TEST INFRASTRUCTURE.

An independent second evaluation of Sec. IV-F for tiny systems with small
integer times.  Every map in Eqs. 3, 4 and 6 is non-decreasing in its window
argument, so the value the paper's iteration converges to is the least t >= 0
with F(t) <= t.  Instead of iterating, this module scans t = 0, 1, 2, ... and
stops at the first such t (or reports "exceeds the deadline").  It works on
the dict form of ``paam_gen.tiny`` systems with plain Python ints and shares
no code with ``paam_oracle.c``.
"""
from __future__ import annotations

SCHED, OVERRUN, DEP = 0, 1, 2
INF = None


def _mu(t: int, T: int) -> int:
    # Lemma 1 (Eq. 2): ceil(t / T) + 1
    return -(-t // T) + 1


def _least_t(F, limit: int):
    """Least t in [0, limit] with F(t) <= t, else None."""
    for t in range(limit + 1):
        if F(t) <= t:
            return t
    return None


def scan_system(sysd: dict, n_buckets: int = 1, eps: int = 0, kappa: int = 0):
    """Returns (R list, status list) for one tiny system dict."""
    ch = sysd["chains"]
    ex = sysd["execs"]
    n = len(ch)
    prio = [c["prio"] for c in ch]
    T = [c["T"] for c in ch]
    D = [c["D"] for c in ch]
    xe = [c["exec"] for c in ch]
    core = [ex[c["exec"]]["core"] for c in ch]
    eprio = [ex[c["exec"]]["prio"] for c in ch]
    E = [sum(e for e, _ in c["cbs"]) for c in ch]
    Emax = [max([e for e, _ in c["cbs"]], default=0) for c in ch]
    segs = [[a + 2 * kappa for _, ss in c["cbs"] for a in ss] for c in ch]  # A* (Sec. IV-F)
    delta = [len(s) for s in segs]
    S = [sum(s) for s in segs]
    M = [max(s, default=0) for s in segs]

    users = sorted([c for c in range(n) if delta[c] > 0], key=lambda c: -prio[c])
    bucket = {c: (i * n_buckets) // len(users) for i, c in enumerate(users)}
    blk = [max([M[l] for l in users if prio[l] < prio[c] and bucket[l] == bucket.get(c)], default=0)
           for c in range(n)]
    B = [max([Emax[l] for l in range(n) if xe[l] == xe[c] and prio[l] < prio[c]], default=0)
         for c in range(n)]
    hps = [[h for h in users if prio[h] > prio[c]] for c in range(n)]
    hp = [[h for h in range(n) if xe[h] == xe[c] and prio[h] > prio[c]] for c in range(n)]
    hpp = [[h for h in range(n) if xe[h] != xe[c] and core[h] == core[c] and eprio[h] > eprio[c]]
           for c in range(n)]

    # Lemma 2 / Eq. 3 for every segment, summed; None if some segment exceeds D_c
    Hseg = []
    for c in range(n):
        tot = 0
        for a in segs[c]:
            h = _least_t(lambda t, a=a, c=c: a + blk[c] + sum(_mu(t, T[k]) * S[k] for k in hps[c]), D[c])
            if h is None:
                tot = None
                break
            tot += h
        Hseg.append(tot)

    def Hstar(c, t):
        if delta[c] == 0:
            return 0
        per_chain = S[c] + delta[c] * blk[c] + sum(_mu(t, T[k]) * S[k] for k in hps[c])  # Eq. 4
        h = per_chain if Hseg[c] is None else min(Hseg[c], per_chain)
        return h + delta[c] * eps  # Eq. 1

    R = [None] * n
    st = [None] * n
    Hfin = [None] * n
    # executor priority first, then chain priority: every needed H*_h is ready
    for c in sorted(range(n), key=lambda c: (-eprio[c], -prio[c])):
        need = hp[c] + [h for h in hpp[c] if ch[h]["spin"]]
        if any(st[h] != SCHED for h in need):
            st[c], R[c] = DEP, -1
            continue

        def F(t, c=c):
            v = B[c] + E[c] + Hstar(c, t)
            v += sum(_mu(t, T[h]) * (E[h] + Hfin[h]) for h in hp[c])
            v += sum(_mu(t, T[h]) * (E[h] + (Hfin[h] if ch[h]["spin"] else delta[h] * eps)) for h in hpp[c])
            return v  # Theorem 1, Eq. 6

        r = _least_t(F, D[c])
        if r is None:
            st[c], R[c] = OVERRUN, -1
        else:
            st[c], R[c], Hfin[c] = SCHED, r, Hstar(c, r)
    return R, st
