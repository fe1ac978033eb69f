"""Python entry to the discrete-event simulation (``des.c``) -- TEST INFRASTRUCTURE."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def _seg(seg):
    # a segment entry: A (accelerator 0) or an (A, accelerator) pair
    return (seg, 0) if isinstance(seg, int) else (int(seg[0]), int(seg[1]))


def explore(sysd: dict, n_buckets: int = 1, eps: int = 0, kappa: int = 0, all_variants: bool = True,
            t_limit_extra: int = 200) -> list:
    """Largest observed response per chain of one tiny system dict over every
    release-offset vector (and execution-time variant)."""
    ch, ex = sysd["chains"], sysd["execs"]
    n = len(ch)
    T = np.array([c["T"] for c in ch], np.int64)
    prio = np.array([c["prio"] for c in ch], np.int32)
    exe = np.array([c["exec"] for c in ch], np.int32)
    spin = np.array([c["spin"] for c in ch], np.uint8)
    cb_n = np.array([len(c["cbs"]) for c in ch], np.int32)
    E = np.array([e for c in ch for (e, _) in c["cbs"]], np.int64)
    nseg = np.array([len(ss) for c in ch for (_, ss) in c["cbs"]], np.int32)
    segs = [_seg(sg) for c in ch for (_, ss) in c["cbs"] for sg in ss]
    A = np.array([a for a, _ in segs] or [0], np.int64)
    acc = np.array([u for _, u in segs] or [0], np.int32)
    core = np.array([x["core"] for x in ex], np.int32)
    xprio = np.array([x["prio"] for x in ex], np.int32)
    out = np.zeros(n, np.int64)
    f = _lib("des").des_explore
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 9 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_void_p]
    p = lambda a: a.ctypes.data
    rc = f(n, p(T), p(prio), p(exe), p(spin), p(cb_n), p(E), p(nseg), p(A), p(acc), len(ex), p(core), p(xprio),
           n_buckets, eps, kappa, t_limit_extra, 1 if all_variants else 0, p(out))
    if rc != 0:
        raise RuntimeError(f"des_explore failed: {rc}")
    return out.tolist()
