"""Convenience wrappers over the C ABI that allocate outputs with PyTorch."""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from . import _binding as B

_FIELDS = ["sys_chain_off", "chain_cb_off", "cb_seg_off", "T", "D", "prio", "exec", "spin", "E", "A", "acc",
           "sys_exec_off", "exec_core", "exec_prio"]


def to_device(sy, device="cuda", pin: bool = False):
    """Copy the arrays of a host batch to torch tensors on ``device`` (or to
    pinned host tensors when ``pin``).  Returns an attribute namespace."""
    import torch

    out = SimpleNamespace()
    for f in _FIELDS:
        a = getattr(sy, f, None)
        if a is None:
            setattr(out, f, None)
            continue
        t = torch.from_numpy(np.ascontiguousarray(a))
        t = t.pin_memory() if pin else t.to(device)
        setattr(out, f, t)
    return out


def analyze(ctx: B.Context, batch: B.Batch, n_buckets: int = 1, eps: int = 0, kappa: int = 0, stream=None,
            blocking_mode: int = 0):
    """Run ``paam_rta_analyze_batch`` into fresh torch device tensors."""
    import torch

    dev = torch.device("cuda", ctx.device)
    R = torch.empty(batch.n_chain, dtype=torch.int64, device=dev)
    st = torch.empty(batch.n_chain, dtype=torch.uint8, device=dev)
    v = torch.empty(batch.n_sys, dtype=torch.uint8, device=dev)
    B.paam_rta_analyze_batch(ctx, batch, B.analysis_opts(n_buckets, eps, kappa, blocking_mode), R, st, v,
                             stream=stream)
    return R, st, v


def search(ctx: B.Context, batch: B.Batch, ranks, n_buckets: int = 1, eps: int = 0, kappa: int = 0,
           stop_at_first: bool = False, want_cand_ok: bool = True, stream=None, blocking_mode: int = 0):
    """Run ``paam_rta_search_priorities`` on device rank rows; returns torch
    tensors (first_ok [S], cand_ok [S, K] or None)."""
    import torch

    dev = torch.device("cuda", ctx.device)
    S, K, _ = ranks.shape
    first_ok = torch.empty(S, dtype=torch.int32, device=dev)
    cand_ok = torch.empty((S, K), dtype=torch.uint8, device=dev) if want_cand_ok else None
    B.paam_rta_search_priorities(ctx, batch, B.analysis_opts(n_buckets, eps, kappa, blocking_mode), ranks,
                                 stop_at_first,
                                 cand_ok, first_ok, stream=stream)
    return first_ok, cand_ok


def audsley_order(ctx: B.Context, batch: B.Batch, nmax: int, n_buckets: int = 1, eps: int = 0, kappa: int = 0,
                  blocking_mode: int = 0, stream=None):
    """Run ``paam_rta_audsley_order``; returns the seed ranks as a torch
    tensor [S, nmax] (int16, rank 0 highest, -1 beyond each system's chains)."""
    import torch

    ranks = torch.empty((batch.n_sys, nmax), dtype=torch.int16, device=torch.device("cuda", ctx.device))
    B.paam_rta_audsley_order(ctx, batch, B.analysis_opts(n_buckets, eps, kappa, blocking_mode), ranks,
                             stream=stream)
    return ranks
