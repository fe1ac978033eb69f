"""``paam_rta_load_systems`` refuses a system whose iteration bound
L = sum_h ceil(Dmax / T_h) + 2 exceeds PAAM_MAX_ITER (PAAM_E_RANGE), so no
analysis kernel ever runs on it; a system exactly at the bound is accepted and
its longest recurrence (about PAAM_MAX_ITER steps) ends without reaching the
kernels' iteration cap."""
import numpy as np
import pytest

import oracle
from paam_gen import tiny

from gpu_util import assert_same, ctx, gpu_analyze

pytestmark = pytest.mark.gpu

MAX_ITER = 1 << 20


def _system(X):
    """Chain 0 (T = D = X, E = 0) under chain 1 (T = D = 1, E = 1) on one
    executor: L = ceil(X / X) + ceil(X / 1) + 2 = X + 3, and chain 0's
    recurrence climbs one unit per step until it passes X."""
    return dict(chains=[dict(T=X, D=X, prio=0, exec=0, spin=0, cbs=[(0, [])]),
                        dict(T=1, D=1, prio=1, exec=0, spin=0, cbs=[(1, [])])],
                execs=[dict(core=0, prio=0)])


def test_over_budget_system_refused_at_load():
    import paper_2404_06452_gb300 as pkg

    ok = tiny.to_systems([_system(1000)])
    for X in (MAX_ITER - 2, MAX_ITER, 1 << 30):
        bad = tiny.to_systems([_system(1000), _system(X), _system(50)])
        with pytest.raises(pkg.PaamError) as ei:
            pkg.paam_rta_load_systems(ctx(), bad)
        assert ei.value.code == -2  # PAAM_E_RANGE
        assert L_of(bad)[1] > MAX_ITER
    b = pkg.paam_rta_load_systems(ctx(), ok)
    b.free()


def L_of(sy):
    n = np.diff(sy.sys_chain_off)
    out = []
    for s in range(sy.n_sys):
        T = sy.T[sy.sys_chain_off[s]:sy.sys_chain_off[s + 1]]
        D = sy.D[sy.sys_chain_off[s]:sy.sys_chain_off[s + 1]]
        out.append(int(sum(-(-int(D.max()) // int(t)) for t in T)) + 2 if n[s] else 2)
    return out


def test_system_at_the_bound_runs_to_overrun():
    X = MAX_ITER - 3  # L = MAX_ITER exactly
    sy = tiny.to_systems([_system(X), _system(64)])
    assert L_of(sy)[0] == MAX_ITER
    ref = oracle.analyze(sy)
    assert ref["status"].tolist() == [1, 0, 1, 0]  # chain 0 passes its deadline, chain 1 meets its own
    it = oracle.iterations(sy)
    assert it["max_loop"][0] == X + 1  # one step per unit up to X + 1
    out = gpu_analyze(sy)
    assert_same(out, ref)
    assert not np.any(out["status"] == 3)  # PAAM_ST_ITERCAP
