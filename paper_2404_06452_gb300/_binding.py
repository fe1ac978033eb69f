"""Thin ctypes binding of ``include/paam_rta.h`` (argument marshalling only).

Every computation runs in ``libpaam_rta.so``.  PyTorch supplies device
memory and streams.  If the library is missing the import fails loudly; there
is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaam_rta.so")

PAAM_OK = 0
PAAM_ST_SCHED, PAAM_ST_OVERRUN, PAAM_ST_DEP, PAAM_ST_ITERCAP = 0, 1, 2, 3
PAAM_MAX_CHAINS = 64

_c_void_p = ctypes.c_void_p


class SystemsView(ctypes.Structure):
    _fields_ = [
        ("n_sys", ctypes.c_int64), ("n_chain", ctypes.c_int64), ("n_cb", ctypes.c_int64),
        ("n_seg", ctypes.c_int64), ("n_exec", ctypes.c_int64),
        ("sys_chain_off", _c_void_p), ("chain_cb_off", _c_void_p), ("cb_seg_off", _c_void_p),
        ("T", _c_void_p), ("D", _c_void_p), ("prio", _c_void_p), ("exec", _c_void_p), ("spin", _c_void_p),
        ("E", _c_void_p), ("A", _c_void_p), ("acc", _c_void_p), ("sys_exec_off", _c_void_p),
        ("exec_core", _c_void_p), ("exec_prio", _c_void_p), ("is_device", ctypes.c_int32),
        ("reserved_", ctypes.c_int32),
    ]


class AnalysisOpts(ctypes.Structure):
    _fields_ = [("n_buckets", ctypes.c_int32), ("blocking_mode", ctypes.c_int32),
                ("eps_ns", ctypes.c_int64), ("kappa_ns", ctypes.c_int64)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch_rows", ctypes.c_int32), ("lr", ctypes.c_float),
                ("weight_decay", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("seed", ctypes.c_uint64), ("n_buckets", ctypes.c_int32),
                ("reserved_", ctypes.c_int32), ("kappa_ns", ctypes.c_int64),
                ("epoch_loss", ctypes.POINTER(ctypes.c_float))]


class PaamError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        sig = {
            "paam_create": (ctypes.c_int, [P(_c_void_p), ctypes.c_int]),
            "paam_destroy": (None, [_c_void_p]),
            "paam_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "paam_rta_load_systems": (ctypes.c_int, [_c_void_p, P(SystemsView), _c_void_p, P(_c_void_p)]),
            "paam_batch_n_sys": (ctypes.c_int64, [_c_void_p]),
            "paam_batch_n_chain": (ctypes.c_int64, [_c_void_p]),
            "paam_batch_free": (None, [_c_void_p]),
            "paam_rta_analyze_batch": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                      _c_void_p, _c_void_p, _c_void_p]),
            "paam_launch_count": (ctypes.c_uint64, []),
            "paam_rta_num_launch_configs": (ctypes.c_int, []),
            "paam_rta_autotune": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                 _c_void_p, ctypes.c_int]),
            "paam_rta_set_launch_config": (ctypes.c_int, [_c_void_p, ctypes.c_int]),
            "paam_rta_get_launch_config": (ctypes.c_int, [_c_void_p]),
            "paam_rta_analyze_noalloc": (ctypes.c_int, [P(SystemsView), P(AnalysisOpts), _c_void_p, _c_void_p,
                                                        _c_void_p, _c_void_p]),
            "paam_rta_search_ordered": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                       ctypes.c_int32, ctypes.c_int32, _c_void_p, ctypes.c_int32,
                                                       ctypes.c_int32, _c_void_p, _c_void_p, _c_void_p]),
            "paam_model_create": (ctypes.c_int, [_c_void_p, ctypes.c_uint64, P(_c_void_p)]),
            "paam_model_free": (None, [_c_void_p]),
            "paam_model_num_params": (ctypes.c_int64, []),
            "paam_model_get_params": (ctypes.c_int, [_c_void_p, _c_void_p]),
            "paam_model_set_params": (ctypes.c_int, [_c_void_p, _c_void_p]),
            "paam_model_save": (ctypes.c_int, [_c_void_p, ctypes.c_char_p]),
            "paam_model_load": (ctypes.c_int, [_c_void_p, ctypes.c_char_p, P(_c_void_p)]),
            "paam_surrogate_train": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, P(TrainOpts),
                                                    P(_c_void_p)]),
            "paam_surrogate_infer": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, ctypes.c_int32,
                                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                    ctypes.c_int32, _c_void_p, _c_void_p, _c_void_p]),
            "paam_surrogate_predict": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_int32,
                                                      ctypes.c_int64, _c_void_p, _c_void_p]),
            "paam_surrogate_search": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _c_void_p,
                                                     _c_void_p]),
            "paam_surrogate_grad": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, _c_void_p, ctypes.c_int32,
                                                   _c_void_p, _c_void_p]),
            "paam_surrogate_features": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _c_void_p,
                                                       _c_void_p]),
            "paam_tc_gemm_bf16": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _c_void_p, _c_void_p]),
            "paam_diag_gelu": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_int64, _c_void_p]),
            "paam_diag_divisor": (ctypes.c_int, [_c_void_p, _c_void_p, _c_void_p, ctypes.c_int64, _c_void_p]),
            "paam_measure_preemption": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_void_p,
                                                       _c_void_p]),
            "paam_rta_end_to_end": (ctypes.c_int, [_c_void_p, _c_void_p, ctypes.c_int64, _c_void_p, _c_void_p,
                                                   _c_void_p, ctypes.c_int64, _c_void_p, _c_void_p, _c_void_p,
                                                   _c_void_p, _c_void_p]),
            "paam_rta_search_priorities": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                          _c_void_p, _c_void_p, _c_void_p]),
            "paam_rta_audsley_order": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), ctypes.c_int32,
                                                      _c_void_p, _c_void_p]),
            "paam_rta_autotune_search": (ctypes.c_int, [_c_void_p, _c_void_p, P(AnalysisOpts), _c_void_p,
                                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _c_void_p,
                                                        _c_void_p, ctypes.c_int]),
            "paam_rta_analyze_host": (ctypes.c_int, [_c_void_p, P(SystemsView), P(AnalysisOpts), ctypes.c_int32,
                                                     ctypes.c_int64, _c_void_p, _c_void_p, _c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def exported_symbols() -> list:
    """Names this binding expects the library to export."""
    return ["paam_create", "paam_destroy", "paam_strerror", "paam_rta_load_systems", "paam_batch_n_sys",
            "paam_batch_n_chain", "paam_batch_free", "paam_rta_analyze_batch", "paam_launch_count",
            "paam_rta_num_launch_configs", "paam_rta_autotune", "paam_rta_set_launch_config",
            "paam_rta_get_launch_config", "paam_rta_analyze_noalloc", "paam_rta_search_priorities",
            "paam_tc_gemm_bf16", "paam_rta_search_ordered", "paam_model_create", "paam_model_free",
            "paam_model_num_params", "paam_model_get_params", "paam_model_set_params", "paam_model_save",
            "paam_model_load", "paam_surrogate_train", "paam_surrogate_infer", "paam_surrogate_predict", "paam_surrogate_search",
            "paam_surrogate_grad", "paam_surrogate_features", "paam_diag_gelu", "paam_diag_divisor", "paam_rta_end_to_end",
            "paam_measure_preemption", "paam_rta_audsley_order", "paam_rta_analyze_host",
            "paam_rta_autotune_search"]


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().paam_launch_count())


def strerror(code: int) -> str:
    try:
        return lib().paam_strerror(code).decode()
    except ImportError:
        return str(code)


def _check(rc: int, what: str):
    if rc != PAAM_OK:
        raise PaamError(rc, what)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _ptr(x) -> int | None:
    """Address of a numpy array or a torch tensor (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer {type(x)}")


class Context:
    """A library context bound to one CUDA device (``paam_create``)."""

    def __init__(self, device: int = 0):
        h = _c_void_p()
        _check(lib().paam_create(ctypes.byref(h), int(device)), "paam_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().paam_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A validated device copy of systems (``paam_rta_load_systems``)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    @property
    def n_sys(self) -> int:
        return int(lib().paam_batch_n_sys(self.handle))

    @property
    def n_chain(self) -> int:
        return int(lib().paam_batch_n_chain(self.handle))

    def free(self):
        if self.handle:
            lib().paam_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


_VIEW_FIELDS = ["sys_chain_off", "chain_cb_off", "cb_seg_off", "T", "D", "prio", "exec", "spin", "E", "A",
                "acc", "sys_exec_off", "exec_core", "exec_prio"]


def make_view(sy, is_device: bool) -> tuple:
    """A ``SystemsView`` over the arrays of ``sy`` (attributes named as in the
    header); returns (view, keepalive)."""
    v = SystemsView()
    keep = []
    for f in _VIEW_FIELDS:
        a = getattr(sy, f, None)
        keep.append(a)
        setattr(v, f, _ptr(a))
    v.n_sys = len(sy.sys_chain_off) - 1
    v.n_chain = len(sy.T)
    v.n_cb = len(sy.E)
    v.n_seg = len(sy.A)
    v.n_exec = len(sy.exec_core)
    v.is_device = 1 if is_device else 0
    return v, keep


def paam_rta_load_systems(ctx: Context, sy, stream=None, is_device: bool | None = None) -> Batch:
    if is_device is None:
        is_device = hasattr(sy.T, "is_cuda") and bool(sy.T.is_cuda)
    v, keep = make_view(sy, is_device)
    h = _c_void_p()
    _check(lib().paam_rta_load_systems(ctx.handle, ctypes.byref(v), _stream_ptr(stream), ctypes.byref(h)),
           "paam_rta_load_systems")
    del keep
    return Batch(ctx, h)


def analysis_opts(n_buckets: int = 1, eps: int = 0, kappa: int = 0, blocking_mode: int = 0) -> AnalysisOpts:
    return AnalysisOpts(int(n_buckets), int(blocking_mode), int(eps), int(kappa))


def paam_rta_analyze_batch(ctx: Context, batch: Batch, opts: AnalysisOpts, R, status, verdict=None,
                           stream=None):
    _check(lib().paam_rta_analyze_batch(ctx.handle, batch.handle, ctypes.byref(opts), _ptr(R), _ptr(status),
                                        _ptr(verdict), _stream_ptr(stream)), "paam_rta_analyze_batch")


def paam_rta_num_launch_configs() -> int:
    return int(lib().paam_rta_num_launch_configs())


def paam_rta_autotune(ctx: Context, batch: Batch, opts: AnalysisOpts, stream=None) -> tuple:
    """Time every launch configuration on ``batch``; keep the fastest.
    Returns (chosen index, list of per-configuration milliseconds)."""
    n = paam_rta_num_launch_configs()
    times = (ctypes.c_float * n)()
    rc = lib().paam_rta_autotune(ctx.handle, batch.handle, ctypes.byref(opts), _stream_ptr(stream), times, n)
    if rc < 0:
        raise PaamError(rc, "paam_rta_autotune")
    return rc, [float(t) for t in times]


def paam_rta_set_launch_config(batch: Batch, index: int):
    _check(lib().paam_rta_set_launch_config(batch.handle, int(index)), "paam_rta_set_launch_config")


def paam_rta_get_launch_config(batch: Batch) -> int:
    return int(lib().paam_rta_get_launch_config(batch.handle))


PAAM_NOALLOC_MAX_SYS = 65536


def paam_rta_analyze_noalloc(sy, opts: AnalysisOpts, R, status, verdict=None, stream=None):
    """Allocation-free analysis of device-resident tables ``sy`` (attributes
    named as in the header, torch CUDA tensors) into caller-owned outputs."""
    v, keep = make_view(sy, True)
    _check(lib().paam_rta_analyze_noalloc(ctypes.byref(v), ctypes.byref(opts), _ptr(R), _ptr(status),
                                          _ptr(verdict), _stream_ptr(stream)), "paam_rta_analyze_noalloc")
    del keep


def paam_rta_search_priorities(ctx: Context, batch: Batch, opts: AnalysisOpts, ranks, stop_at_first: bool,
                               cand_ok, first_ok, stream=None):
    """Exact search over candidate rank orders ``ranks`` ([S, K, nmax] int16,
    device tensor); fills ``first_ok`` [S] and optionally ``cand_ok`` [S, K]."""
    S, K, nmax = ranks.shape
    _check(lib().paam_rta_search_priorities(ctx.handle, batch.handle, ctypes.byref(opts), _ptr(ranks), int(K),
                                            int(nmax), 1 if stop_at_first else 0, _ptr(cand_ok), _ptr(first_ok),
                                            _stream_ptr(stream)), "paam_rta_search_priorities")


def paam_rta_autotune_search(ctx: Context, batch: Batch, opts: AnalysisOpts, ranks, stop_at_first: bool = False,
                             stream=None) -> tuple:
    """Time every launch configuration on the search over ``ranks`` ([S, K,
    nmax] int16 device tensor); keep the fastest.  Returns (index, ms list)."""
    S, K, nmax = ranks.shape
    n = paam_rta_num_launch_configs()
    times = (ctypes.c_float * n)()
    rc = lib().paam_rta_autotune_search(ctx.handle, batch.handle, ctypes.byref(opts), _ptr(ranks), int(K), int(nmax),
                                        1 if stop_at_first else 0, _stream_ptr(stream), times, n)
    _check(min(rc, 0), "paam_rta_autotune_search")
    return rc, list(times)


def paam_rta_analyze_host(ctx: Context, sy, opts: AnalysisOpts, R, status, verdict=None, launch_config: int = -1,
                          chunk_systems: int = 0):
    """Pipelined analysis of host arrays ``sy`` (numpy or page-locked torch
    CPU tensors) into host outputs ``R`` [n_chain] int64, ``status``
    [n_chain] uint8 and optionally ``verdict`` [n_sys] uint8."""
    v, keep = make_view(sy, False)
    _check(lib().paam_rta_analyze_host(ctx.handle, ctypes.byref(v), ctypes.byref(opts), int(launch_config),
                                       int(chunk_systems), _ptr(R), _ptr(status), _ptr(verdict)),
           "paam_rta_analyze_host")
    del keep


def paam_rta_audsley_order(ctx: Context, batch: Batch, opts: AnalysisOpts, ranks_out, stream=None):
    """Audsley-style seed order of every system into ``ranks_out`` ([S, nmax]
    int16 device tensor; rank 0 highest, -1 beyond each system's chains)."""
    nmax = ranks_out.shape[1]
    _check(lib().paam_rta_audsley_order(ctx.handle, batch.handle, ctypes.byref(opts), int(nmax), _ptr(ranks_out),
                                        _stream_ptr(stream)), "paam_rta_audsley_order")


def paam_tc_gemm_bf16(A, B, C, err, stream=None):
    """C = A @ B^T on the tensor cores (A [M, K], B [N, K] bf16; C [M, N] fp32)."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().paam_tc_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), int(M), int(N), int(K), _ptr(err),
                                   _stream_ptr(stream)), "paam_tc_gemm_bf16")


def paam_rta_end_to_end(ctx: Context, batch: Batch, e2e_off, e2e_chain, D_e2e, eps_prime: int, R, status,
                        R_e2e, status_e2e, stream=None):
    """End-to-end bounds of chains made of sub-chains (device arrays)."""
    n = int(D_e2e.numel())
    _check(lib().paam_rta_end_to_end(ctx.handle, batch.handle, n, _ptr(e2e_off), _ptr(e2e_chain), _ptr(D_e2e),
                                     int(eps_prime), _ptr(R), _ptr(status), _ptr(R_e2e), _ptr(status_e2e),
                                     _stream_ptr(stream)), "paam_rta_end_to_end")


PREEMPTION_KERNELS = ("MatMul", "Reduction", "VectorAdd", "Histogram")


def paam_measure_preemption(kind: int, iters: int, device: int = 0) -> tuple:
    """Per-iteration preemption delays and baselines in microseconds (numpy)."""
    delay = np.zeros(iters, np.float32)
    base = np.zeros(iters, np.float32)
    _check(lib().paam_measure_preemption(int(device), int(kind), int(iters), delay.ctypes.data, base.ctypes.data),
           "paam_measure_preemption")
    return delay, base


def paam_diag_gelu(z, gelu=None, grad=None, stream=None):
    """The network's activation and its derivative at device fp32 ``z``."""
    _check(lib().paam_diag_gelu(_ptr(z), _ptr(gelu), _ptr(grad), int(z.numel()), _stream_ptr(stream)),
           "paam_diag_gelu")


def paam_diag_divisor(T, m, l, stream=None):
    """Multiply-shift divisor {m, l} of Lemma 1's arrival count for every
    device uint32 period in ``T`` (written to device uint32 ``m`` and ``l``)."""
    n = int(T.numel())
    if m.numel() != n or l.numel() != n:
        raise ValueError("paam_diag_divisor: T, m and l must have the same length")
    _check(lib().paam_diag_divisor(_ptr(T), _ptr(m), _ptr(l), n, _stream_ptr(stream)), "paam_diag_divisor")


def paam_rta_search_ordered(ctx: Context, batch: Batch, opts: AnalysisOpts, ranks, order, stop_at_first: bool,
                            cand_ok, first_ok, stream=None):
    """Search visiting candidates ``order[s, j]`` (device int32 [S, K]) of
    ``ranks`` ([S, Kc, nmax] int16) in that order."""
    S, Kc, nmax = ranks.shape
    K = order.shape[1]
    _check(lib().paam_rta_search_ordered(ctx.handle, batch.handle, ctypes.byref(opts), _ptr(ranks), int(Kc),
                                         int(nmax), _ptr(order), int(K), 1 if stop_at_first else 0, _ptr(cand_ok),
                                         _ptr(first_ok), _stream_ptr(stream)), "paam_rta_search_ordered")


class Model:
    """A surrogate ranking model (``paam_model_*``)."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    @staticmethod
    def create(ctx: Context, seed: int = 0) -> "Model":
        h = _c_void_p()
        _check(lib().paam_model_create(ctx.handle, ctypes.c_uint64(seed), ctypes.byref(h)), "paam_model_create")
        return Model(ctx, h)

    @staticmethod
    def load(ctx: Context, path: str) -> "Model":
        h = _c_void_p()
        _check(lib().paam_model_load(ctx.handle, path.encode(), ctypes.byref(h)), "paam_model_load")
        return Model(ctx, h)

    def save(self, path: str):
        _check(lib().paam_model_save(self.handle, path.encode()), "paam_model_save")

    def get_params(self) -> np.ndarray:
        out = np.empty(int(lib().paam_model_num_params()), np.float32)
        _check(lib().paam_model_get_params(self.handle, out.ctypes.data), "paam_model_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == int(lib().paam_model_num_params())
        _check(lib().paam_model_set_params(self.handle, p.ctypes.data), "paam_model_set_params")

    def free(self):
        if self.handle:
            lib().paam_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def train_opts(epochs=1, batch_rows=8192, lr=1e-3, weight_decay=1e-4, beta1=0.9, beta2=0.999, adam_eps=1e-8,
               seed=0, n_buckets=1, kappa=0, epoch_loss=None) -> TrainOpts:
    o = TrainOpts(int(epochs), int(batch_rows), float(lr), float(weight_decay), float(beta1), float(beta2),
                  float(adam_eps), ctypes.c_uint64(seed).value, int(n_buckets), 0, int(kappa), None)
    if epoch_loss is not None:
        o.epoch_loss = epoch_loss.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return o


def paam_surrogate_train(ctx: Context, batch: Batch, R, status, opts: TrainOpts, model: "Model | None" = None):
    h = _c_void_p(model.handle.value if model is not None else None)
    _check(lib().paam_surrogate_train(ctx.handle, batch.handle, _ptr(R), _ptr(status), ctypes.byref(opts),
                                      ctypes.byref(h)), "paam_surrogate_train")
    return model if model is not None else Model(ctx, h)


def paam_surrogate_search(ctx: Context, model: Model, batch: Batch, opts: AnalysisOpts, ranks, first_ok,
                          n_pinned: int = 0, stream=None):
    """The exact search guided by the network over the candidates ``ranks``
    ([S, K, nmax] device int16): the first ``n_pinned`` slots, then the others in
    the network's order, each system stopping at its first admitted candidate;
    ``first_ok`` ([S] device int32) gets that candidate or -1."""
    S, K, nmax = ranks.shape
    _check(lib().paam_surrogate_search(ctx.handle, model.handle, batch.handle, ctypes.byref(opts), _ptr(ranks),
                                       int(K), int(nmax), int(n_pinned), _ptr(first_ok), _stream_ptr(stream)),
           "paam_surrogate_search")


def paam_surrogate_infer(ctx: Context, model: Model, batch: Batch, ranks, top_k: int, ranked, scores=None,
                         n_buckets: int = 1, kappa: int = 0, stream=None, n_pinned: int = 0):
    """Rank the candidates ``ranks`` ([S, K, nmax]) by the network's score into
    ``ranked`` ([S, top_k]); the first ``n_pinned`` slots rank ahead of all."""
    S, K, nmax = ranks.shape
    _check(lib().paam_surrogate_infer(ctx.handle, model.handle, batch.handle, _ptr(ranks), int(K), int(nmax),
                                      int(n_buckets), int(kappa), int(n_pinned), int(top_k), _ptr(ranked),
                                      _ptr(scores), _stream_ptr(stream)), "paam_surrogate_infer")


def paam_surrogate_predict(ctx: Context, model: Model, batch: Batch, pred, n_buckets: int = 1, kappa: int = 0,
                           stream=None):
    _check(lib().paam_surrogate_predict(ctx.handle, model.handle, batch.handle, int(n_buckets), int(kappa),
                                        _ptr(pred), _stream_ptr(stream)), "paam_surrogate_predict")


def paam_surrogate_grad(ctx: Context, model: Model, X, L) -> tuple:
    rows = X.shape[0]
    g = np.empty(int(lib().paam_model_num_params()), np.float32)
    loss = ctypes.c_float(0.0)
    _check(lib().paam_surrogate_grad(ctx.handle, model.handle, _ptr(X), _ptr(L), int(rows), g.ctypes.data,
                                     ctypes.byref(loss)), "paam_surrogate_grad")
    return g, float(loss.value)


def paam_surrogate_features(ctx: Context, batch: Batch, X, ranks=None, n_buckets: int = 1, kappa: int = 0,
                            stream=None):
    if ranks is None:
        K, nmax = 1, 0
    else:
        _, K, nmax = ranks.shape
    _check(lib().paam_surrogate_features(ctx.handle, batch.handle, _ptr(ranks), int(K), int(nmax), int(n_buckets),
                                         int(kappa), _ptr(X), _stream_ptr(stream)), "paam_surrogate_features")
