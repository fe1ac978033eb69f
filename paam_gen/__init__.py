"""Seeded synthetic workload generator for PAAM's chain model.

Produces structure-of-arrays, CSR-indexed systems in the layout the C ABI
takes (see ``include/paam_rta.h``): systems -> chains -> callbacks ->
accelerator segments, plus per-system executors.  The module holds no
response-time arithmetic; it only draws inputs.  Both the CPU oracle and the
CUDA library consume what it writes.

Workload presets mirror the analytical study of Sec. V-D (chains of
callbacks, one accelerator, random periods, chain utilisation split equally
over its callbacks) scaled up:

``cfg1``  1,000 systems, 4 chains of 2-4 callbacks, 2 executors on 1 core,
          U = 0.5, segment probability 0.3.
``cfg2``  1,000,000 systems, 8-16 chains of 3-8 callbacks, 4 executors on 2
          cores, U swept 0.3..0.9, segment probability 0.5.
``cfg3``  4,000,000 systems of uneven size: 2 + Geom(1/9) chains (<= 64),
          1-12 callbacks, 2-8 executors, U ~ Unif[0.2, 0.95].
``cfg4``  10,000 systems of 16 chains (cfg1 shape), U = 0.7 -- the
          priority-assignment search workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paam_gen.c")
_LIB = os.path.join(_HERE, "libpaam_gen.so")
_lock = threading.Lock()
_lib = None


class GenParams(ctypes.Structure):
    _fields_ = [
        ("n_sys", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("n_min", ctypes.c_int32),
        ("n_max", ctypes.c_int32),
        ("n_geom_p", ctypes.c_double),
        ("cb_min", ctypes.c_int32),
        ("cb_max", ctypes.c_int32),
        ("x_min", ctypes.c_int32),
        ("x_max", ctypes.c_int32),
        ("exec_per_core", ctypes.c_int32),
        ("util_mode", ctypes.c_int32),
        ("util_lo", ctypes.c_double),
        ("util_hi", ctypes.c_double),
        ("util_step", ctypes.c_double),
        ("util_n", ctypes.c_int32),
        ("seg_per_cb", ctypes.c_int32),
        ("p_acc", ctypes.c_double),
        ("a_min", ctypes.c_int64),
        ("a_max", ctypes.c_int64),
        ("t_min", ctypes.c_double),
        ("t_max", ctypes.c_double),
        ("d_lo", ctypes.c_double),
        ("d_hi", ctypes.c_double),
        ("p_spin", ctypes.c_double),
        ("exec_prio_mode", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
    ]


_BASE = dict(
    n_geom_p=0.0, exec_per_core=2, util_mode=0, util_step=0.0, util_n=1, seg_per_cb=1,
    a_min=100_000, a_max=2_000_000, t_min=1e7, t_max=1e8, d_lo=1.0, d_hi=1.0,
    p_spin=0.0, exec_prio_mode=0,
)

CONFIGS = {
    "cfg1": dict(_BASE, n_sys=1_000, seed=0x9AA40001, n_min=4, n_max=4, cb_min=2, cb_max=4,
                 x_min=2, x_max=2, util_lo=0.5, util_hi=0.5, p_acc=0.3),
    "cfg2": dict(_BASE, n_sys=1_000_000, seed=0x9AA40002, n_min=8, n_max=16, cb_min=3, cb_max=8,
                 x_min=4, x_max=4, util_mode=1, util_lo=0.3, util_hi=0.9, util_step=0.1,
                 util_n=7, p_acc=0.5),
    "cfg3": dict(_BASE, n_sys=4_000_000, seed=0x9AA40003, n_min=2, n_max=64, n_geom_p=1.0 / 9.0,
                 cb_min=1, cb_max=12, x_min=2, x_max=8, util_lo=0.2, util_hi=0.95, p_acc=0.5),
    "cfg4": dict(_BASE, n_sys=10_000, seed=0x9AA40004, n_min=16, n_max=16, cb_min=2, cb_max=4,
                 x_min=2, x_max=2, util_lo=0.7, util_hi=0.7, p_acc=0.3),
    # the search workload with its 16 chains spread over 16 single-executor cores and
    # 0.05-1 ms segments: here some candidate orders pass the admission test
    "cfg4s": dict(_BASE, n_sys=10_000, seed=0x9AA40014, n_min=16, n_max=16, cb_min=2, cb_max=4,
                  x_min=16, x_max=16, exec_per_core=1, util_lo=0.7, util_hi=0.7, p_acc=0.3,
                  a_min=50_000, a_max=1_000_000),
}


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        lib.paam_gen_count.argtypes = [P(GenParams), ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 4
        lib.paam_gen_count.restype = None
        lib.paam_gen_fill.argtypes = [P(GenParams), ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 16
        lib.paam_gen_fill.restype = None
        lib.paam_gen_perms.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        lib.paam_gen_perms.restype = None
        lib.paam_gen_assign_wfd.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 5 + [
            ctypes.c_int32, ctypes.c_void_p]
        lib.paam_gen_assign_wfd.restype = None
        _lib = lib
        return lib


def build() -> str:
    """Compile the generator with gcc (portable C, no arch-specific flags)."""
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _offs(counts) -> np.ndarray:
    o = np.zeros(len(counts) + 1, np.int64)
    np.cumsum(counts, out=o[1:])
    return o


def _expand(starts: np.ndarray, ends: np.ndarray) -> np.ndarray:
    """Concatenation of arange(starts[i], ends[i]) without a Python loop."""
    starts = np.asarray(starts, np.int64)
    lens = np.asarray(ends, np.int64) - starts
    nz = lens > 0
    s_nz, l_nz = starts[nz], lens[nz]
    total = int(l_nz.sum())
    if total == 0:
        return np.zeros(0, np.int64)
    step = np.ones(total, np.int64)
    first = np.zeros(len(l_nz), np.int64)
    np.cumsum(l_nz[:-1], out=first[1:])
    step[0] = s_nz[0]
    # at each run start, jump from the previous run's last value to this run's start
    step[first[1:]] = s_nz[1:] - (s_nz[:-1] + l_nz[:-1] - 1)
    return np.cumsum(step)


@dataclass
class Systems:
    """A batch of systems in SoA/CSR form (host numpy arrays).

    Offsets are int64 with a closing sentinel; chain-local executor indices
    refer to the system's executor range ``sys_exec_off[s] ..``.
    """
    sys_chain_off: np.ndarray
    chain_cb_off: np.ndarray
    cb_seg_off: np.ndarray
    T: np.ndarray
    D: np.ndarray
    prio: np.ndarray
    exec: np.ndarray
    spin: np.ndarray
    E: np.ndarray
    A: np.ndarray
    acc: np.ndarray
    sys_exec_off: np.ndarray
    exec_core: np.ndarray
    exec_prio: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def n_sys(self) -> int:
        return len(self.sys_chain_off) - 1

    @property
    def n_chain(self) -> int:
        return len(self.T)

    @property
    def n_cb(self) -> int:
        return len(self.E)

    @property
    def n_seg(self) -> int:
        return len(self.A)

    @property
    def n_exec(self) -> int:
        return len(self.exec_core)

    def chains_per_system(self) -> np.ndarray:
        return np.diff(self.sys_chain_off)

    def nbytes(self) -> int:
        arrs = [self.sys_chain_off, self.chain_cb_off, self.cb_seg_off, self.T, self.D, self.prio,
                self.exec, self.spin, self.E, self.A, self.acc, self.sys_exec_off, self.exec_core]
        if self.exec_prio is not None:
            arrs.append(self.exec_prio)
        return int(sum(a.nbytes for a in arrs))

    def subset(self, idx) -> "Systems":
        """Systems ``idx`` (in the given order) re-packed into a fresh batch."""
        idx = np.asarray(idx, dtype=np.int64)
        sc, cbo, so, xo = self.sys_chain_off, self.chain_cb_off, self.cb_seg_off, self.sys_exec_off
        chains = _expand(sc[idx], sc[idx + 1])
        cbs = _expand(cbo[chains], cbo[chains + 1])
        segs = _expand(so[cbs], so[cbs + 1])
        execs = _expand(xo[idx], xo[idx + 1])
        return Systems(
            sys_chain_off=_offs(sc[idx + 1] - sc[idx]), chain_cb_off=_offs(cbo[chains + 1] - cbo[chains]),
            cb_seg_off=_offs(so[cbs + 1] - so[cbs]),
            T=self.T[chains], D=self.D[chains], prio=self.prio[chains],
            exec=self.exec[chains], spin=self.spin[chains], E=self.E[cbs],
            A=self.A[segs], acc=self.acc[segs], sys_exec_off=_offs(xo[idx + 1] - xo[idx]),
            exec_core=self.exec_core[execs],
            exec_prio=None if self.exec_prio is None else self.exec_prio[execs],
            meta=dict(self.meta, subset=True),
        )

    def chain_index(self, idx) -> np.ndarray:
        """Global chain indices of systems ``idx`` in subset order."""
        idx = np.asarray(idx, dtype=np.int64)
        return _expand(self.sys_chain_off[idx], self.sys_chain_off[idx + 1])


def params(cfg: str | dict = "cfg1", **overrides) -> GenParams:
    d = dict(CONFIGS[cfg]) if isinstance(cfg, str) else dict(cfg)
    d.update(overrides)
    p = GenParams()
    for name, _ in GenParams._fields_:
        if name == "pad_":
            continue
        setattr(p, name, d[name])
    return p


def generate(cfg: str | dict = "cfg1", threads: int | None = None, **overrides) -> Systems:
    """Generate a batch.  Deterministic in (cfg, overrides); thread count free."""
    lib = _load()
    p = params(cfg, **overrides)
    n = int(p.n_sys)
    threads = threads or min(32, os.cpu_count() or 1)
    n_chain = np.zeros(n, np.int32)
    n_cb = np.zeros(n, np.int32)
    n_seg = np.zeros(n, np.int32)
    n_exec = np.zeros(n, np.int32)
    bounds = np.linspace(0, n, threads + 1).astype(np.int64)
    ranges = [(int(bounds[i]), int(bounds[i + 1])) for i in range(threads) if bounds[i] < bounds[i + 1]]
    with ThreadPoolExecutor(len(ranges) or 1) as ex:
        list(ex.map(lambda r: lib.paam_gen_count(ctypes.byref(p), r[0], r[1], _ptr(n_chain), _ptr(n_cb),
                                                 _ptr(n_seg), _ptr(n_exec)), ranges))

    def excl(counts):
        o = np.zeros(n + 1, np.int64)
        np.cumsum(counts, out=o[1:])
        return o

    sys_chain_off, sys_exec_off = excl(n_chain), excl(n_exec)
    sys_cb, sys_seg = excl(n_cb), excl(n_seg)
    NC, NB, NS, NX = int(sys_chain_off[-1]), int(sys_cb[-1]), int(sys_seg[-1]), int(sys_exec_off[-1])
    chain_cb_off = np.empty(NC + 1, np.int64)
    cb_seg_off = np.empty(NB + 1, np.int64)
    chain_cb_off[NC] = NB
    cb_seg_off[NB] = NS
    T = np.empty(NC, np.int64)
    D = np.empty(NC, np.int64)
    prio = np.empty(NC, np.int32)
    ex_ = np.empty(NC, np.int32)
    spin = np.empty(NC, np.uint8)
    E = np.empty(NB, np.int64)
    A = np.empty(NS, np.int64)
    acc = np.empty(NS, np.int32)
    exec_core = np.empty(NX, np.int32)
    exec_prio = np.empty(NX, np.int32)
    with ThreadPoolExecutor(len(ranges) or 1) as ex:
        list(ex.map(lambda r: lib.paam_gen_fill(
            ctypes.byref(p), r[0], r[1], _ptr(sys_chain_off), _ptr(sys_exec_off), _ptr(sys_cb),
            _ptr(sys_seg), _ptr(chain_cb_off), _ptr(cb_seg_off), _ptr(T), _ptr(D), _ptr(prio),
            _ptr(ex_), _ptr(spin), _ptr(E), _ptr(A), _ptr(acc), _ptr(exec_core), _ptr(exec_prio)),
            ranges))
    meta = {"cfg": cfg if isinstance(cfg, str) else "custom", **overrides}
    return Systems(sys_chain_off, chain_cb_off, cb_seg_off, T, D, prio, ex_, spin, E, A, acc,
                   sys_exec_off, exec_core, exec_prio, meta)


def permutations(seed: int, n_of_sys: np.ndarray, K: int, nmax: int | None = None,
                 first_slot: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """Random candidate priority orders.

    ``out[s, k, :n_s]`` is a permutation of ``0..n_s-1`` (a rank order: entry
    c is the rank of chain c, 0 = highest) for slots ``first_slot..K-1``;
    entries past ``n_s`` are -1.  Earlier slots are left as they are.
    """
    lib = _load()
    n_of_sys = np.ascontiguousarray(n_of_sys, dtype=np.int32)
    S = len(n_of_sys)
    nmax = int(nmax or (n_of_sys.max() if S else 1))
    if out is None:
        out = np.zeros((S, K, nmax), np.int16)
    assert out.shape == (S, K, nmax) and out.dtype == np.int16 and out.flags.c_contiguous
    lib.paam_gen_perms(seed, 0, S, K, first_slot, _ptr(n_of_sys), nmax, _ptr(out))
    return out


def candidate_ranks(sy: Systems, K: int, seed: int, nmax: int | None = None) -> np.ndarray:
    """Candidate chain priority orders for the priority-assignment search.

    ``out[s, k, c]`` is the rank (0 = highest priority) of chain c of system s
    in candidate k; entries past the system's chain count are -1.  Slot 0 is
    the system's own order (its given priorities: criticality-as-priority),
    slot 1 is deadline-monotonic (shorter deadline first, ties by chain index),
    slots 2.. are seeded random permutations.
    """
    n = sy.chains_per_system().astype(np.int32)
    S = sy.n_sys
    nmax = int(nmax or (n.max() if S else 1))
    out = np.full((S, K, nmax), -1, np.int16)
    if K > 2:
        permutations(seed, n, K, nmax, first_slot=2, out=out)
    sysid = np.repeat(np.arange(S), n)
    local = np.arange(sy.n_chain) - sy.sys_chain_off[sysid]

    def ranks_by(keys):
        order = np.lexsort(keys + (sysid,))  # within each system, ascending keys
        r = np.empty(sy.n_chain, np.int64)
        r[order] = np.arange(sy.n_chain) - sy.sys_chain_off[sysid[order]]
        return r

    if K > 0:
        out[sysid, 0, local] = ranks_by((-sy.prio.astype(np.int64),))
    if K > 1:
        out[sysid, 1, local] = ranks_by((local, sy.D))
    return out


def assign_accelerators(sy: Systems, n_units: int, threads: int | None = None) -> Systems:
    """The same systems with their accelerator segments spread over n_units
    units of the accelerator by worst-fit decreasing utilisation (A / T), per
    system, as the PAAM server assigns them at registration."""
    assert 1 <= n_units <= 64
    lib = _load()
    acc = np.zeros(len(sy.A), np.int32)
    threads = threads or min(32, os.cpu_count() or 1)
    bounds = np.linspace(0, sy.n_sys, threads + 1).astype(np.int64)
    ranges = [(int(bounds[i]), int(bounds[i + 1])) for i in range(threads) if bounds[i] < bounds[i + 1]]
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in (sy.sys_chain_off, sy.chain_cb_off, sy.cb_seg_off,
                                                                sy.T, sy.A)]
    with ThreadPoolExecutor(len(ranges) or 1) as ex:
        list(ex.map(lambda r: lib.paam_gen_assign_wfd(r[0], r[1], *[_ptr(a) for a in arrs], int(n_units),
                                                      _ptr(acc)), ranges))
    return Systems(**{**sy.__dict__, "acc": acc, "meta": dict(sy.meta, accelerator_units=int(n_units))})


def split_end_to_end(sy: Systems, seed: int, max_sub: int = 3):
    """Group each system's chains into end-to-end chains of sub-chains (the
    workload shape of chains that span several executors).

    System s uses one group size k_s, uniform in 1..min(max_sub, executors),
    and groups consecutive chains; the members of a group get the period of
    its first chain (deadline D* = that period, also each member's D) and
    consecutive executors, so each sub-chain runs on its own executor.
    Executor priorities are left to be derived (criticality-as-priority).
    Returns (systems, e2e_off, e2e_chain, D_e2e); sub-chains are contiguous.
    """
    rng = np.random.default_rng(seed)
    n = sy.chains_per_system()
    nx = np.diff(sy.sys_exec_off)
    k = np.minimum(rng.integers(1, max_sub + 1, size=sy.n_sys), np.maximum(nx, 1))
    sysid = np.repeat(np.arange(sy.n_sys), n)
    local = np.arange(sy.n_chain) - sy.sys_chain_off[sysid]
    kc = k[sysid]
    first = sy.sys_chain_off[sysid] + (local // kc) * kc
    T = sy.T[first].copy()
    ex = ((sy.exec[first].astype(np.int64) + local % kc) % nx[sysid]).astype(np.int32)
    out = Systems(sy.sys_chain_off, sy.chain_cb_off, sy.cb_seg_off, T, T.copy(), sy.prio, ex, sy.spin, sy.E,
                  sy.A, sy.acc, sy.sys_exec_off, sy.exec_core, None, dict(sy.meta, e2e_split=int(max_sub)))
    starts = np.nonzero(local % kc == 0)[0]
    e2e_off = np.append(starts, sy.n_chain).astype(np.int64)
    return out, e2e_off, np.arange(sy.n_chain, dtype=np.int64), T[starts].copy()


from .tiny import tiny_system, tiny_batch  # noqa: E402  (pure-Python small-integer systems)
