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


def _seg(seg):
    # a segment entry: A (accelerator 0) or an (A, accelerator) pair
    return (seg, 0) if isinstance(seg, int) else (int(seg[0]), int(seg[1]))


def _mu(t: int, T: int) -> int:
    # Lemma 1 (Eq. 2): ceil(t / T) + 1
    return -(-t // T) + 1


def _least_t(F, limit: int):
    """Least t in [0, limit] with F(t) <= t, else None."""
    for t in range(limit + 1):
        if F(t) <= t:
            return t
    return None


def scan_system(sysd: dict, n_buckets: int = 1, eps: int = 0, kappa: int = 0, blocking_mode: int = 0):
    """Returns (R list, status list) for one tiny system dict.

    ``blocking_mode`` 0 takes Lemma 4 as printed (the longest CPU WCET of a
    lower-priority callback on the executor); 1 takes the safe reading, in
    which such a callback keeps the single-threaded executor for its CPU work
    and for each of its accelerator requests, each request bounded by its own
    least fixed point of Eq. 3 plus the overhead eps, and an unbounded request
    makes the blocking, and so the chain, unbounded (OVERRUN after the DEP
    rule)."""
    if blocking_mode not in (0, 1):
        raise ValueError("blocking_mode: 0 or 1")
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
    # segments as (A*, accelerator); each accelerator has its own server (rule R1)
    segs = [[(a + 2 * kappa, u) for _, ss in c["cbs"] for a, u in map(_seg, ss)] for c in ch]  # A* (Sec. IV-F)
    delta = [len(s) for s in segs]
    accs = sorted({u for s in segs for _, u in s})
    S = {u: [sum(a for a, v in s if v == u) for s in segs] for u in accs}
    dl = {u: [sum(1 for _, v in s if v == u) for s in segs] for u in accs}
    M = {u: [max([a for a, v in s if v == u], default=0) for s in segs] for u in accs}
    blk, hps = {}, {}
    for u in accs:
        users = sorted([c for c in range(n) if dl[u][c] > 0], key=lambda c: -prio[c])
        bucket = {c: (i * n_buckets) // len(users) for i, c in enumerate(users)}
        blk[u] = [max([M[u][l] for l in users if prio[l] < prio[c] and bucket[l] == bucket.get(c)], default=0)
                  for c in range(n)]
        hps[u] = [[h for h in users if prio[h] > prio[c]] for c in range(n)]
    B = [max([Emax[l] for l in range(n) if xe[l] == xe[c] and prio[l] < prio[c]], default=0)
         for c in range(n)]
    hp = [[h for h in range(n) if xe[h] == xe[c] and prio[h] > prio[c]] for c in range(n)]
    hpp = [[h for h in range(n) if xe[h] != xe[c] and core[h] == core[c] and eprio[h] > eprio[c]]
           for c in range(n)]

    # Lemma 2 / Eq. 3: the least fixed point of every segment on its own
    # (None when it lies above D_c), kept per callback for the safe blocking
    # reading, and summed per accelerator (None if one of them is None)
    def seg_lfp(c, a, u):
        return _least_t(lambda t: a + blk[u][c] + sum(_mu(t, T[k]) * S[u][k] for k in hps[u][c]), D[c])

    cb_h = [[[(seg_lfp(c, a + 2 * kappa, u), u) for a, u in map(_seg, ss)] for _, ss in ch[c]["cbs"]]
            for c in range(n)]
    Hseg = {u: [] for u in accs}
    for u in accs:
        for c in range(n):
            hs = [h for cb in cb_h[c] for h, v in cb if v == u]
            Hseg[u].append(None if any(h is None for h in hs) else sum(hs))

    if blocking_mode == 1:
        # a lower-priority callback holds the executor for E plus, per request,
        # its Lemma 2 bound and eps; B_c is the longest hold on c's executor
        def cb_hold(l, i):
            hs = [h for h, _ in cb_h[l][i]]
            return None if any(h is None for h in hs) else ch[l]["cbs"][i][0] + sum(h + eps for h in hs)

        hold = []
        for l in range(n):
            hl = [cb_hold(l, i) for i in range(len(ch[l]["cbs"]))]
            hold.append(None if any(h is None for h in hl) else max(hl, default=0))
        for c in range(n):
            lp = [hold[l] for l in range(n) if xe[l] == xe[c] and prio[l] < prio[c]]
            B[c] = None if any(h is None for h in lp) else max(lp, default=0)

    def Hstar(c, t):
        if delta[c] == 0:
            return 0
        h = 0
        for u in accs:  # one term per accelerator the chain uses (R1)
            if dl[u][c] == 0:
                continue
            per_chain = S[u][c] + dl[u][c] * blk[u][c] + sum(_mu(t, T[k]) * S[u][k] for k in hps[u][c])  # Eq. 4
            h += per_chain if Hseg[u][c] is None else min(Hseg[u][c], per_chain)
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
        if B[c] is None:  # unbounded blocking (safe reading only)
            st[c], R[c] = OVERRUN, -1
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
