"""CPU oracle for PAAM's response-time analysis -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library under ``paper_2404_06452_gb300/``; both read inputs from
``paam_gen``.

Contents
  paam_oracle.c   plain C evaluation of Eqs. 1-6 (Sec. IV-F), system by system
  lfp_scan.py     independent brute-force least-fixed-point scan (tiny systems)
  des.c           discrete-event simulation of the PAAM runtime rules (tiny)
  mlp.py          float64 numpy forward/backward of the surrogate network
  features.py     per-chain surrogate features, numpy
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_libs: dict = {}

ST_SCHED, ST_OVERRUN, ST_DEP, ST_ITERCAP = 0, 1, 2, 3


def _build_one(name: str) -> str:
    src = os.path.join(_HERE, f"{name}.c")
    out = os.path.join(_HERE, f"lib{name}.so")
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build() -> list:
    """Compile the C parts of the oracle (gcc, portable flags)."""
    return [_build_one(n) for n in ("paam_oracle", "des")]


def _lib(name: str):
    with _lock:
        if name in _libs:
            return _libs[name]
        src = os.path.join(_HERE, f"{name}.c")
        so = os.path.join(_HERE, f"lib{name}.so")
        if (not os.path.exists(so)) or os.path.getmtime(so) < os.path.getmtime(src):
            _build_one(name)
        lib = ctypes.CDLL(so)
        _libs[name] = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


MAX_ACC = 8  # accelerators per system the oracle handles (R1: one server each)


def _acc(sy):
    acc = getattr(sy, "acc", None)
    if acc is None or len(acc) == 0:
        return None
    acc = np.ascontiguousarray(acc, dtype=np.int32)
    if acc.min() < 0 or acc.max() >= MAX_ACC:
        raise ValueError(f"accelerator index outside 0..{MAX_ACC - 1}")
    return acc


def _arrays(sy):
    return dict(
        sys_chain_off=_c(sy.sys_chain_off, np.int64), chain_cb_off=_c(sy.chain_cb_off, np.int64),
        cb_seg_off=_c(sy.cb_seg_off, np.int64), T=_c(sy.T, np.int64), D=_c(sy.D, np.int64),
        prio=_c(sy.prio, np.int32), exec=_c(sy.exec, np.int32), spin=_c(sy.spin, np.uint8),
        E=_c(sy.E, np.int64), A=_c(sy.A, np.int64), acc=_acc(sy), sys_exec_off=_c(sy.sys_exec_off, np.int64),
        exec_core=_c(sy.exec_core, np.int32), exec_prio=_c(sy.exec_prio, np.int32),
    )


def _ranges(n, threads):
    threads = max(1, min(threads, n)) if n else 1
    b = np.linspace(0, n, threads + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(threads) if b[i] < b[i + 1]]


def analyze(sy, n_buckets: int = 1, eps: int = 0, kappa: int = 0, blocking_mode: int = 0,
            threads: int = 1, aux: bool = False, work: bool = False, derive_exec_prio: bool = False):
    """Run the oracle over every system of ``sy`` (a ``paam_gen.Systems``).

    Returns a dict with ``R`` (int64, -1 unless SCHED), ``status`` (uint8),
    ``verdict`` (uint8 per system) and optionally ``aux`` ([n_chain, 12]) and
    ``work`` (interference terms per system).
    """
    if blocking_mode not in (0, 1):
        raise ValueError("blocking_mode: 0 (Lemma 4 as printed) or 1 (safe reading)")
    lib = _lib("paam_oracle")
    a = _arrays(sy)
    if derive_exec_prio:
        a["exec_prio"] = None
    nc, ns = len(a["T"]), len(a["sys_chain_off"]) - 1
    R = np.zeros(nc, np.int64)
    st = np.zeros(nc, np.uint8)
    verdict = np.zeros(ns, np.uint8)
    ax = np.zeros((nc, 12), np.int64) if aux else None
    wk = np.zeros(ns, np.int64) if work else None
    f = lib.oracle_analyze
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 14 + [
        ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 5

    def run(r):
        f(r[0], r[1], _p(a["sys_chain_off"]), _p(a["chain_cb_off"]), _p(a["cb_seg_off"]), _p(a["T"]),
          _p(a["D"]), _p(a["prio"]), _p(a["exec"]), _p(a["spin"]), _p(a["E"]), _p(a["A"]), _p(a["acc"]),
          _p(a["sys_exec_off"]), _p(a["exec_core"]), _p(a["exec_prio"]), int(n_buckets), int(eps),
          int(kappa), int(blocking_mode), _p(R), _p(st), _p(verdict), _p(ax), _p(wk))

    rs = _ranges(ns, threads)
    if len(rs) <= 1:
        for r in rs:
            run(r)
    else:
        with ThreadPoolExecutor(len(rs)) as ex:
            list(ex.map(run, rs))
    out = dict(R=R, status=st, verdict=verdict)
    if aux:
        out["aux"] = ax
    if work:
        out["work"] = wk
    return out


def iterations(sy, n_buckets: int = 1, eps: int = 0, kappa: int = 0, blocking_mode: int = 0, threads: int = 1):
    """Evaluation counts of the fixed-point recurrences, per system: of the
    segment recurrences (Eq. 3), of the chain recurrences (Eq. 6), and the
    most evaluations any single recurrence took (``max_loop``)."""
    lib = _lib("paam_oracle")
    a = _arrays(sy)
    nc, ns = len(a["T"]), len(a["sys_chain_off"]) - 1
    out = {k: np.zeros(ns, np.int64) for k in ("seg", "chain", "max_loop")}
    f = lib.oracle_analyze_iters
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 14 + [
        ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 5

    def run(r):
        R = np.zeros(nc, np.int64)
        st = np.zeros(nc, np.uint8)
        f(r[0], r[1], _p(a["sys_chain_off"]), _p(a["chain_cb_off"]), _p(a["cb_seg_off"]), _p(a["T"]),
          _p(a["D"]), _p(a["prio"]), _p(a["exec"]), _p(a["spin"]), _p(a["E"]), _p(a["A"]), _p(a["acc"]),
          _p(a["sys_exec_off"]), _p(a["exec_core"]), _p(a["exec_prio"]), int(n_buckets), int(eps),
          int(kappa), int(blocking_mode), _p(R), _p(st), _p(out["seg"]), _p(out["chain"]), _p(out["max_loop"]))

    rs = _ranges(ns, threads)
    if len(rs) <= 1:
        for r in rs:
            run(r)
    else:
        with ThreadPoolExecutor(len(rs)) as ex:
            list(ex.map(run, rs))
    return out


AUX_FIELDS = ("E", "Emax", "delta", "S", "M", "bucket", "blk", "B", "Hseg", "Hstar", "eprio", "prio")


def search(sy, ranks: np.ndarray, n_buckets: int = 1, eps: int = 0, kappa: int = 0,
           stop_at_first: bool = False, threads: int = 1, blocking_mode: int = 0):
    """Exact priority-assignment search over candidate rank orders.

    ``ranks[s, k, c]`` is the rank (0 = highest priority) of chain c of system
    s in candidate k.  Returns ``cand_ok`` [S, K] (uint8) and ``first_ok`` [S].
    """
    lib = _lib("paam_oracle")
    a = _arrays(sy)
    S = len(a["sys_chain_off"]) - 1
    ranks = np.ascontiguousarray(ranks, dtype=np.int16)
    assert ranks.shape[0] == S
    K, nmax = ranks.shape[1], ranks.shape[2]
    cand_ok = np.zeros((S, K), np.uint8)
    first_ok = np.full(S, -1, np.int32)
    nc = len(a["T"])
    f = lib.oracle_search
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 13 + [
        ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
        ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4

    def run(r):
        Rs = np.zeros(nc, np.int64)
        sts = np.zeros(nc, np.uint8)
        f(r[0], r[1], _p(a["sys_chain_off"]), _p(a["chain_cb_off"]), _p(a["cb_seg_off"]), _p(a["T"]),
          _p(a["D"]), _p(a["prio"]), _p(a["exec"]), _p(a["spin"]), _p(a["E"]), _p(a["A"]), _p(a["acc"]),
          _p(a["sys_exec_off"]), _p(a["exec_core"]), int(n_buckets), int(eps), int(kappa), int(blocking_mode),
          _p(ranks),
          K, nmax, 1 if stop_at_first else 0, _p(cand_ok), _p(first_ok), _p(Rs), _p(sts))

    rs = _ranges(S, threads)
    if len(rs) <= 1:
        for r in rs:
            run(r)
    else:
        with ThreadPoolExecutor(len(rs)) as ex:
            list(ex.map(run, rs))
    return dict(cand_ok=cand_ok, first_ok=first_ok)


def audsley(sy, nmax: int | None = None, n_buckets: int = 1, eps: int = 0, kappa: int = 0,
            blocking_mode: int = 0, threads: int = 1):
    """Audsley-style greedy priority seed, lowest level first (see
    ``oracle_audsley`` in ``paam_oracle.c``).  Returns ranks [S, nmax] (int16,
    0 = highest priority, -1 beyond each system's chains)."""
    lib = _lib("paam_oracle")
    a = _arrays(sy)
    S = len(a["sys_chain_off"]) - 1
    counts = np.diff(a["sys_chain_off"])
    if nmax is None:
        nmax = int(counts.max()) if S else 1
    if S and nmax < int(counts.max()):
        raise ValueError("nmax below the largest chain count")
    ranks = np.full((S, nmax), -1, np.int16)
    nc = len(a["T"])
    f = lib.oracle_audsley
    f.restype = None
    f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 13 + [
        ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 3

    def run(r):
        Rs = np.zeros(nc, np.int64)
        sts = np.zeros(nc, np.uint8)
        f(r[0], r[1], _p(a["sys_chain_off"]), _p(a["chain_cb_off"]), _p(a["cb_seg_off"]), _p(a["T"]),
          _p(a["D"]), _p(a["prio"]), _p(a["exec"]), _p(a["spin"]), _p(a["E"]), _p(a["A"]), _p(a["acc"]),
          _p(a["sys_exec_off"]), _p(a["exec_core"]), int(n_buckets), int(eps), int(kappa), int(blocking_mode),
          int(nmax), _p(ranks), _p(Rs), _p(sts))

    rs = _ranges(S, threads)
    if len(rs) <= 1:
        for r in rs:
            run(r)
    else:
        with ThreadPoolExecutor(len(rs)) as ex:
            list(ex.map(run, rs))
    return ranks
