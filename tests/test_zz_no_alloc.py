"""The allocation-free entry point against the allocating one.

paam_rta_analyze_noalloc is for callers that cannot allocate memory when they
run an admission test; it keeps its bookkeeping in a fixed device array of the
library.  This file checks, through the C ABI, that two calls in a row give
exactly the results of paam_rta_load_systems + paam_rta_analyze_batch (the
analysis is integer-exact, so the tolerance is zero) -- with one accelerator
and with three, under both blocking readings, on the default stream and on a
caller's stream -- that the calls leave the free device memory and PyTorch's
allocator statistics unchanged, and that an oversized batch is refused.  It
is named to run last and works alone in a fresh process as well.
"""
import random

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _workload():
    import paam_gen as g
    from paam_gen import tiny

    a = g.generate("cfg3", n_sys=3000)  # 2..64 chains: exercises the wide-configuration list
    rng = random.Random(5)
    big_t = [tiny.tiny_system(rng, n_min=2, n_max=20, cb_max=4, x_max=4, periods=tuple(range(2**31, 2**34, 2**28)),
                              e_max=2**26, a_max=2**25, p_seg=0.5, p_spin=0.5) for _ in range(100)]
    b = tiny.to_systems(big_t)  # periods beyond the 32-bit fast path: exercises the int64 list
    parts = [a.subset(np.arange(0, 1500)), b, a.subset(np.arange(1500, 3000))]

    def cat_off(name):
        offs, base = [np.zeros(1, np.int64)], 0
        for s in parts:
            o = getattr(s, name)
            offs.append(o[1:] + base)
            base += o[-1]
        return np.concatenate(offs)

    cat = lambda f: np.concatenate([getattr(s, f) for s in parts])
    return g.Systems(cat_off("sys_chain_off"), cat_off("chain_cb_off"), cat_off("cb_seg_off"), cat("T"), cat("D"),
                     cat("prio"), cat("exec"), cat("spin"), cat("E"), cat("A"), cat("acc"), cat_off("sys_exec_off"),
                     cat("exec_core"), cat("exec_prio"))


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = _workload()
    params = dict(n_buckets=2, eps=198_000, kappa=41_210)
    ctx = pkg.Context(0)
    batch = pkg.paam_rta_load_systems(ctx, sy)
    R0, st0, v0 = pkg.analyze(ctx, batch, **params)
    torch.cuda.synchronize()
    dev = pkg.to_device(sy)
    opts = pkg.analysis_opts(**params)
    R = torch.empty_like(R0)
    st = torch.empty_like(st0)
    v = torch.empty_like(v0)
    for call in range(2):
        R.fill_(-7)
        st.fill_(9)
        v.fill_(9)
        torch.cuda.synchronize()
        before = _alloc_snapshot(torch)
        pkg.paam_rta_analyze_noalloc(dev, opts, R, st, v)
        torch.cuda.synchronize()
        if call == 1:  # after the first call's one-time set-up nothing else may be taken
            assert _alloc_snapshot(torch) == before
        assert torch.equal(R, R0), f"call {call}: R differs"
        assert torch.equal(st, st0), f"call {call}: status differs"
        assert torch.equal(v, v0), f"call {call}: verdict differs"
    batch.free()
    ctx.close()


def _alloc_snapshot(torch):
    st = torch.cuda.memory_stats()
    pool = {k: v for k, v in st.items() if k.startswith(("allocated_bytes.all.current", "reserved_bytes.all.current",
                                                          "active_bytes.all.current"))}
    return torch.cuda.mem_get_info()[0], pool


@pytest.mark.parametrize("blocking_mode", [0, 1])
def test_noalloc_several_accelerators_on_a_caller_stream(blocking_mode):
    """The safe blocking reading and the literal one on a batch whose segments
    are spread over three accelerator units (the caller's acc table is read
    in place), enqueued on the caller's own stream: two calls in a row, each
    bit-identical to the allocating path, neither taking device memory from
    the driver or from PyTorch's caching allocator."""
    import torch

    import paam_gen as g
    import paper_2404_06452_gb300 as pkg

    sy = g.assign_accelerators(_workload(), 3)
    assert sy.acc.max() == 2
    params = dict(n_buckets=2, eps=198_000, kappa=41_210)
    ctx = pkg.Context(0)
    batch = pkg.paam_rta_load_systems(ctx, sy)
    R0, st0, v0 = pkg.analyze(ctx, batch, blocking_mode=blocking_mode, **params)
    torch.cuda.synchronize()
    dev = pkg.to_device(sy)
    opts = pkg.analysis_opts(blocking_mode=blocking_mode, **params)
    stream = torch.cuda.Stream()
    R = torch.empty_like(R0)
    st = torch.empty_like(st0)
    v = torch.empty_like(v0)
    for call in range(2):
        R.fill_(-7)
        st.fill_(9)
        v.fill_(9)
        torch.cuda.synchronize()
        before = _alloc_snapshot(torch)
        pkg.paam_rta_analyze_noalloc(dev, opts, R, st, v, stream=stream)
        stream.synchronize()
        if call == 1:
            assert _alloc_snapshot(torch) == before
        assert torch.equal(R, R0), f"call {call}: R differs"
        assert torch.equal(st, st0), f"call {call}: status differs"
        assert torch.equal(v, v0), f"call {call}: verdict differs"
    batch.free()
    ctx.close()


def test_noalloc_rejects_oversized_batch():
    import torch

    import paam_gen as g
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg1", n_sys=pkg.PAAM_NOALLOC_MAX_SYS + 1)
    dev = pkg.to_device(sy)
    R = torch.empty(sy.n_chain, dtype=torch.int64, device="cuda")
    st = torch.empty(sy.n_chain, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.PaamError) as ei:
        pkg.paam_rta_analyze_noalloc(dev, pkg.analysis_opts(), R, st)
    assert ei.value.code == -2
