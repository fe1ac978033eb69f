"""The pipelined analysis of host arrays (``paam_rta_analyze_host``): the same
results as loading the batch and analysing it on the device, for every chunk
size and launch configuration, with several accelerators and the safe
blocking reading, and the load-time errors raised from any chunk."""
import numpy as np
import pytest

import oracle
import paam_gen as g

from gpu_util import assert_same, ctx, gpu_analyze

pytestmark = pytest.mark.gpu


def _host(sy, chunk=0, cfg=-1, **p):
    import paper_2404_06452_gb300 as pkg

    R = np.empty(sy.n_chain, np.int64)
    st = np.empty(sy.n_chain, np.uint8)
    v = np.empty(sy.n_sys, np.uint8)
    pkg.paam_rta_analyze_host(ctx(), sy, pkg.analysis_opts(**p), R, st, v, launch_config=cfg, chunk_systems=chunk)
    return dict(R=R, status=st, verdict=v)


@pytest.mark.parametrize("chunk", [0, 1, 777, 50_000])
def test_same_as_device_batch(chunk):
    sy = g.generate("cfg2", n_sys=120_000)
    ref = gpu_analyze(sy)
    assert_same(_host(sy, chunk), ref)


def test_full_workload_pinned_and_every_launch_config():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg2")  # 1M systems, 12M chains
    pinned = pkg.to_device(sy, pin=True)
    ref = gpu_analyze(sy)
    R = np.empty(sy.n_chain, np.int64)
    st = np.empty(sy.n_chain, np.uint8)
    v = np.empty(sy.n_sys, np.uint8)
    for cfg in range(pkg.paam_rta_num_launch_configs()):
        R[:] = -7
        pkg.paam_rta_analyze_host(ctx(), pinned, pkg.analysis_opts(), R, st, v, launch_config=cfg)
        assert_same(dict(R=R, status=st, verdict=v), ref)


def test_uneven_sizes_and_options_against_oracle():
    sy = g.generate("cfg3", n_sys=40_000)
    p = dict(n_buckets=3, eps=1000, kappa=500)
    got = _host(sy, 5_000, **p)
    idx = np.r_[0:200, 19_900:20_100, 39_800:40_000]
    sub = sy.subset(idx)
    ref = oracle.analyze(sub, threads=8, **p)
    ci = sy.chain_index(idx)
    assert np.array_equal(got["R"][ci], ref["R"]) and np.array_equal(got["status"][ci], ref["status"])
    assert np.array_equal(got["verdict"][idx], ref["verdict"])
    assert_same(got, gpu_analyze(sy, **p))


@pytest.mark.parametrize("blocking_mode", [0, 1])
def test_several_accelerators_and_safe_blocking(blocking_mode):
    sy = g.assign_accelerators(g.generate("cfg2", n_sys=30_000, p_spin=0.3), 3)
    assert_same(_host(sy, 4_096, blocking_mode=blocking_mode), gpu_analyze(sy, blocking_mode=blocking_mode))


def test_invalid_system_in_a_later_chunk_is_rejected():
    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg2", n_sys=20_000)
    bad = sy.subset(np.arange(sy.n_sys))
    c = int(bad.sys_chain_off[15_000])
    bad.D[c] = bad.T[c] + 1  # D > T in system 15,000
    with pytest.raises(pkg.PaamError):
        _host(bad, 2_000)
    # a broken closing offset is caught on the host before any copy
    bad2 = sy.subset(np.arange(sy.n_sys))
    bad2.sys_chain_off[-1] += 1
    with pytest.raises(pkg.PaamError):
        _host(bad2)


def test_automatic_chunks_reject_an_invalid_system_in_the_last_chunk():
    import paper_2404_06452_gb300 as pkg

    # 200,000 systems: automatic chunks of halving size, the last one small
    sy = g.generate("cfg2", n_sys=200_000)
    assert_same(_host(sy), gpu_analyze(sy))
    bad = sy.subset(np.arange(sy.n_sys))
    c = int(bad.sys_chain_off[199_990])
    bad.D[c] = bad.T[c] + 1  # D > T near the end of the batch
    with pytest.raises(pkg.PaamError):
        _host(bad)
