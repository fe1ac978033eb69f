"""End-to-end bounds of chains spanning several executors on the GPU against
the oracle: bit-exact R* and status."""
import numpy as np
import pytest

import oracle
import paam_gen as g
from oracle.end_to_end import end_to_end

from gpu_util import ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps_prime", [0, 198_000])
def test_end_to_end_matches_oracle(eps_prime):
    import torch

    import paper_2404_06452_gb300 as pkg

    sy, off, chain, D = g.split_end_to_end(g.generate("cfg2", n_sys=100_000), 9)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    R, st, _ = pkg.analyze(ctx(), b, eps=5_000)
    Re = torch.empty(len(D), dtype=torch.int64, device="cuda")
    se = torch.empty(len(D), dtype=torch.uint8, device="cuda")
    t = lambda a: torch.from_numpy(a).cuda()
    pkg.paam_rta_end_to_end(ctx(), b, t(off), t(chain), t(D), eps_prime, R, st, Re, se)
    torch.cuda.synchronize()
    ref = oracle.analyze(sy, eps=5_000, threads=8)
    Rr, sr = end_to_end(ref["R"], ref["status"], off, chain, D, eps_prime)
    assert np.array_equal(Re.cpu().numpy(), Rr) and np.array_equal(se.cpu().numpy(), sr)
    assert len(set(sr.tolist())) == 3  # every status occurs
    b.free()


def test_end_to_end_rejects_bad_index():
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg1", n_sys=10)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    R, st, _ = pkg.analyze(ctx(), b)
    off = torch.tensor([0, 2], dtype=torch.int64, device="cuda")
    chain = torch.tensor([0, sy.n_chain], dtype=torch.int64, device="cuda")  # one past the end
    D = torch.tensor([10**9], dtype=torch.int64, device="cuda")
    Re = torch.empty(1, dtype=torch.int64, device="cuda")
    se = torch.empty(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.PaamError):
        pkg.paam_rta_end_to_end(ctx(), b, off, chain, D, 0, R, st, Re, se)
    b.free()


def test_preemption_measurement_runs_every_kernel_kind():
    """The preemption-cost measurement: finite per-iteration delays and
    positive baselines for each of the four kernel kinds; bad arguments are
    refused before any device work."""
    import paper_2404_06452_gb300 as pkg

    for kind in range(4):
        delay, base = pkg.paam_measure_preemption(kind, 20)
        assert np.all(np.isfinite(delay)) and np.all(base > 0), (kind, delay, base)
        assert np.all(delay > -base)  # the contended run cannot be shorter than nothing
    with pytest.raises(pkg.PaamError):
        pkg.paam_measure_preemption(4, 10)
