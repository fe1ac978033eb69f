"""The surrogate network's GPU kernels against float64 oracles, and what the
trained network does for the priority search.

Tolerances: features are fp32 ratios stored as bf16 (relative 2^-8); the
network runs bf16 weights and activations with fp32 accumulation through four
layers, so gradients are compared in relative L2 norm within 3e-2."""
import numpy as np
import pytest

import oracle
import paam_gen as g
from oracle import features as ofeat
from oracle import mlp

from gpu_util import ctx

pytestmark = pytest.mark.gpu


def _bf16_to_f64(t):
    import torch

    return t.to(torch.float32).cpu().numpy().astype(np.float64)


def _features(sy, ranks=None, n_buckets=1, kappa=0):
    import torch

    import paper_2404_06452_gb300 as pkg

    b = pkg.paam_rta_load_systems(ctx(), sy)
    K = 1 if ranks is None else ranks.shape[1]
    X = torch.empty((sy.n_sys * K, 1024), dtype=torch.bfloat16, device="cuda")
    r = None if ranks is None else torch.from_numpy(ranks).cuda()
    pkg.paam_surrogate_features(ctx(), b, X, ranks=r, n_buckets=n_buckets, kappa=kappa)
    torch.cuda.synchronize()
    b.free()
    return _bf16_to_f64(X)


def test_features_match_oracle():
    sy = g.generate("cfg3", n_sys=150)
    got = _features(sy, n_buckets=2, kappa=30_000)
    ref = ofeat.features(sy, n_buckets=2, kappa=30_000)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-3)
    assert np.all(got[ref == 0] == 0)
    sy4 = g.generate("cfg4s", n_sys=40)
    ranks = g.candidate_ranks(sy4, 6, 4)
    got = _features(sy4, ranks)
    ref = ofeat.features(sy4, ranks)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-3)


@pytest.mark.parametrize("case", ["seg16", "seg32", "many_chains", "many_executors"])
def test_candidate_features_paths(case):
    """Candidate mode: 16- and 32-lane segments per candidate order (up to 16 /
    32 chains, several buckets, more candidates than segments per block), and
    the per-item kernel for systems beyond 32 chains or 32 executors."""
    if case == "seg16":
        sy = g.generate("cfg2", n_sys=30, seed=76)
    elif case == "seg32":
        sy = g.generate("cfg3", n_sys=40, seed=77, n_max=32)
        assert sy.chains_per_system().max() > 16
    elif case == "many_chains":
        sy = g.generate("cfg3", n_sys=40, seed=77)
        assert sy.chains_per_system().max() > 32
    else:
        sy = g.generate("cfg4s", n_sys=12, x_min=40, x_max=40, seed=78)
    ranks = g.candidate_ranks(sy, 37, 5)
    got = _features(sy, ranks, n_buckets=3, kappa=20_000)
    ref = ofeat.features(sy, ranks, n_buckets=3, kappa=20_000)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-3)
    assert np.all(got[ref == 0] == 0)


def test_candidate_features_invalid_row_is_zero():
    sy = g.generate("cfg4s", n_sys=5)
    ranks = g.candidate_ranks(sy, 4, 3)
    ranks[2, 1, 3] = ranks[2, 1, 4]  # not a permutation
    ranks[4, 3, 0] = 99              # out of range
    got = _features(sy, ranks).reshape(5, 4, 1024)
    assert np.all(got[2, 1] == 0) and np.all(got[4, 3] == 0)
    ok = np.ones((5, 4), bool)
    ok[2, 1] = ok[4, 3] = False
    ref = ofeat.features(sy, np.where(ok[:, :, None], ranks, g.candidate_ranks(sy, 4, 3))).reshape(5, 4, 1024)
    assert np.all(np.abs(got[ok] - ref[ok]) <= 2.0 ** -8 * np.abs(ref[ok]) + 2e-3)


def _bf16_round(a):
    import torch

    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _oracle_net(params, X):
    """The float64 network on bf16 weights (as the tensor cores see them)."""
    q, o = params.astype(np.float64).copy(), 0
    for fin, fout in mlp.SIZES:
        q[o:o + fin * fout] = _bf16_round(q[o:o + fin * fout])
        o += fin * fout + fout
    return mlp.forward(q, X)[0]


def test_infer_and_predict_scores_match_oracle_network():
    """Inference reads only the feature columns a batch can fill (16 per chain
    slot of its largest system); its scores and the per-chain predictions
    still follow the full 1024-input network."""
    import torch

    import paper_2404_06452_gb300 as pkg

    p = _random_params(11)
    m = pkg.Model.create(ctx(), 2)
    m.set_params(p)
    for cfg, K, nb in (("cfg4s", 20, 1), ("cfg1", 7, 2)):
        sy = g.generate(cfg, n_sys=30)
        ranks = g.candidate_ranks(sy, K, 8)
        b = pkg.paam_rta_load_systems(ctx(), sy)
        r = torch.from_numpy(ranks).cuda()
        ranked = torch.empty((sy.n_sys, 3), dtype=torch.int32, device="cuda")
        scores = torch.empty((sy.n_sys, K), dtype=torch.float32, device="cuda")
        pkg.paam_surrogate_infer(ctx(), m, b, r, 3, ranked, scores, n_buckets=nb)
        pred = torch.empty((sy.n_sys, 64), dtype=torch.float32, device="cuda")
        pkg.paam_surrogate_predict(ctx(), m, b, pred, n_buckets=nb)
        torch.cuda.synchronize()
        n = sy.chains_per_system()
        Y = _oracle_net(p, _bf16_round(ofeat.features(sy, ranks, n_buckets=nb))).reshape(sy.n_sys, K, 64)
        want = np.stack([np.maximum(Y[s, :, :n[s]].max(axis=1), 0.0) for s in range(sy.n_sys)])
        got = scores.cpu().numpy()
        assert np.all(np.abs(got - want) <= 3e-2 * (np.abs(want) + 1.0)), np.abs(got - want).max()
        Yp = _oracle_net(p, _bf16_round(ofeat.features(sy, n_buckets=nb)))
        gp = pred.cpu().numpy()
        for s in range(sy.n_sys):
            assert np.all(np.abs(gp[s, :n[s]] - Yp[s, :n[s]]) <= 3e-2 * (np.abs(Yp[s, :n[s]]) + 1.0))
        b.free()
    m.free()


def test_infer_at_scale_matches_oracle_network():
    """100,000 candidate rows (a ragged last 128-row tile) take the persistent
    weight-stationary layers with the TMA-store epilogue; sampled systems'
    scores follow the float64 network."""
    import torch

    import paper_2404_06452_gb300 as pkg

    p = _random_params(5)
    m = pkg.Model.create(ctx(), 3)
    m.set_params(p)
    sy = g.generate("cfg4s", n_sys=400)
    K = 250
    ranks = g.candidate_ranks(sy, K, 12)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = torch.from_numpy(ranks).cuda()
    ranked = torch.empty((sy.n_sys, 4), dtype=torch.int32, device="cuda")
    scores = torch.empty((sy.n_sys, K), dtype=torch.float32, device="cuda")
    pkg.paam_surrogate_infer(ctx(), m, b, r, 4, ranked, scores)
    torch.cuda.synchronize()
    got = scores.cpu().numpy()
    idx = np.r_[0:8, 196:204, 392:400]  # first, middle and last rows of the batch
    sub = sy.subset(idx)
    n = sub.chains_per_system()
    Y = _oracle_net(p, _bf16_round(ofeat.features(sub, ranks[idx]))).reshape(len(idx), K, 64)
    want = np.stack([np.maximum(Y[s, :, :n[s]].max(axis=1), 0.0) for s in range(len(idx))])
    assert np.all(np.abs(got[idx] - want) <= 3e-2 * (np.abs(want) + 1.0)), np.abs(got[idx] - want).max()
    # the ranking is the score order
    rk = ranked.cpu().numpy()
    for s in range(sy.n_sys):
        assert np.all(np.diff(got[s, rk[s]]) >= 0)
    b.free()
    m.free()


def test_infer_in_two_chunks_matches_oracle_network():
    """5.12M candidate rows run as two chunks of whole systems; systems on both
    sides of the boundary, and the last ones, follow the float64 network."""
    import torch

    import paper_2404_06452_gb300 as pkg

    p = _random_params(6)
    m = pkg.Model.create(ctx(), 4)
    m.set_params(p)
    sy = g.generate("cfg1", n_sys=20_000)
    K = 256
    ranks = g.candidate_ranks(sy, K, 13)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = torch.from_numpy(ranks).cuda()
    ranked = torch.empty((sy.n_sys, 2), dtype=torch.int32, device="cuda")
    scores = torch.empty((sy.n_sys, K), dtype=torch.float32, device="cuda")
    pkg.paam_surrogate_infer(ctx(), m, b, r, 2, ranked, scores)
    torch.cuda.synchronize()
    got = scores.cpu().numpy()
    idx = np.r_[9_994:10_006, 19_994:20_000]
    sub = sy.subset(idx)
    n = sub.chains_per_system()
    Y = _oracle_net(p, _bf16_round(ofeat.features(sub, ranks[idx]))).reshape(len(idx), K, 64)
    want = np.stack([np.maximum(Y[s, :, :n[s]].max(axis=1), 0.0) for s in range(len(idx))])
    assert np.all(np.abs(got[idx] - want) <= 3e-2 * (np.abs(want) + 1.0)), np.abs(got[idx] - want).max()
    assert np.all(np.isfinite(got))
    b.free()
    m.free()


def _random_params(seed):
    rng = np.random.default_rng(seed)
    out = []
    for fin, fout in mlp.SIZES:
        out.append(rng.uniform(-1, 1, fin * fout) * np.sqrt(6.0 / fin))
        out.append(rng.uniform(-0.1, 0.1, fout))
    return np.concatenate(out).astype(np.float32)


def test_gradients_match_oracle():
    """Gradients of one 8,192-row minibatch (the training shape: 19 split-K
    slices of the first layer's weight gradient) element by element.  The
    reference is the network with its storage in bf16 (weights, kept
    pre-activations, activations and back-propagated gradients rounded where
    the kernels store them) and exact sums; what is left is the kernels' fp32
    accumulation, bounded by K * 2^-24 times the sum of the products'
    magnitudes (K <= 8,192 rows: 2^-11), plus a rare bf16 rounding that
    falls the other way.  The fp32 parameters' float64 gradient is checked as
    well, per block in relative L2 norm."""
    import torch

    import paper_2404_06452_gb300 as pkg

    p = _random_params(5)
    m = pkg.Model.create(ctx(), 1)
    m.set_params(p)
    rng = np.random.default_rng(6)
    rows = 8192
    X = torch.from_numpy(rng.uniform(0, 1.5, (rows, 1024)).astype(np.float32)).to(torch.bfloat16)
    L = rng.uniform(0, 2, (rows, 64)).astype(np.float32)
    L[rng.uniform(size=L.shape) < 0.3] = -1.0
    grads, loss = pkg.paam_surrogate_grad(ctx(), m, X.cuda(), torch.from_numpy(L).cuda())
    Xd = X.to(torch.float32).numpy().astype(np.float64)
    ref_loss, ref = mlp.loss_and_grad(p.astype(np.float64), Xd, L)
    ref16_loss, ref16, scale = mlp.loss_and_grad_bf16(p.astype(np.float64), Xd, L)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    assert abs(loss - ref16_loss) <= 1e-3 * ref16_loss
    got = grads.astype(np.float64)
    tol = 2.0 ** -11 * scale + 1e-12
    bad = np.nonzero(np.abs(got - ref16) > tol)[0]
    assert len(bad) == 0, (len(bad), bad[:5], got[bad[:5]], ref16[bad[:5]], tol[bad[:5]])
    # the bound is far below the gradients themselves: a zeroed or misplaced
    # element would exceed it
    assert np.median(np.abs(ref16) / (tol + 1e-30)) > 8
    o = 0
    for fin, fout in mlp.SIZES:
        for size in (fin * fout, fout):
            a, b = got[o:o + size], ref[o:o + size]
            assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-7, (o, np.linalg.norm(a - b) / np.linalg.norm(b))
            o += size
    m.free()


def _trained_model(cfg="cfg4s", n_sys=20000, epochs=6, seed=1):
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate(cfg, n_sys=n_sys, seed=12345)
    # vary the priority orders the network sees: random permutations per system
    rng = np.random.default_rng(seed)
    for s in range(sy.n_sys):
        c0, c1 = sy.sys_chain_off[s], sy.sys_chain_off[s + 1]
        sy.prio[c0:c1] = rng.permutation(c1 - c0)
    sy.exec_prio = None
    b = pkg.paam_rta_load_systems(ctx(), sy)
    R, st, _ = pkg.analyze(ctx(), b)
    losses = np.zeros(epochs, np.float32)
    m = pkg.paam_surrogate_train(ctx(), b, R, st, pkg.train_opts(epochs=epochs, batch_rows=2048, lr=2e-3, seed=seed,
                                                                    epoch_loss=losses))
    torch.cuda.synchronize()
    return m, b, sy, R, st, losses


def test_training_reduces_loss_and_predicts():
    import torch

    import paper_2404_06452_gb300 as pkg

    m, b, sy, R, st, losses = _trained_model()
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.6 * losses[0], losses
    pred = torch.empty((sy.n_sys, 64), dtype=torch.float32, device="cuda")
    pkg.paam_surrogate_predict(ctx(), m, b, pred)
    torch.cuda.synchronize()
    Rn, stn, D = R.cpu().numpy(), st.cpu().numpy(), sy.D
    y = np.where(stn == 0, np.minimum(Rn / D, 2.0), 2.0)
    n = sy.chains_per_system()
    p = pred.cpu().numpy()[np.repeat(np.arange(sy.n_sys), n), np.arange(sy.n_chain) - np.repeat(sy.sys_chain_off[:-1], n)]
    mae = np.abs(p - y).mean()
    assert mae < 0.7 * np.abs(y - y.mean()).mean(), mae
    m.free()
    b.free()


def test_training_is_bit_reproducible():
    """The weight gradients are split over the minibatch rows into slices
    summed in a fixed order, so two trainings with the same seed and data give
    the same parameters bit for bit."""
    import torch

    import paper_2404_06452_gb300 as pkg

    sy = g.generate("cfg2", n_sys=40_000)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    R, st, _ = pkg.analyze(ctx(), b)
    torch.cuda.synchronize()
    params = []
    for _ in range(2):
        m = pkg.paam_surrogate_train(ctx(), b, R, st, pkg.train_opts(epochs=2, batch_rows=4096, lr=2e-3, seed=9),
                                     None)
        params.append(m.get_params())
        m.free()
    b.free()
    assert np.array_equal(params[0].view(np.uint32), params[1].view(np.uint32))


def test_infer_ranks_by_score_and_guided_search_is_exact():
    import torch

    import paper_2404_06452_gb300 as pkg

    m, btrain, *_ = _trained_model()
    btrain.free()
    sy = g.generate("cfg4s", n_sys=400)
    K, top = 64, 8
    ranks = g.candidate_ranks(sy, K, 9)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    r = torch.from_numpy(ranks).cuda()
    ranked = torch.empty((sy.n_sys, top), dtype=torch.int32, device="cuda")
    scores = torch.empty((sy.n_sys, K), dtype=torch.float32, device="cuda")
    pkg.paam_surrogate_infer(ctx(), m, b, r, top, ranked, scores)
    torch.cuda.synchronize()
    sc = scores.cpu().numpy()
    want = np.argsort(sc, axis=1, kind="stable")[:, :top]
    assert np.array_equal(ranked.cpu().numpy(), want)
    # pinned seed slots come first, in slot order, then the scored ones
    pinned = torch.empty_like(ranked)
    pkg.paam_surrogate_infer(ctx(), m, b, r, top, pinned, n_pinned=3)
    torch.cuda.synchronize()
    rest = 3 + np.argsort(sc[:, 3:], axis=1, kind="stable")[:, :top - 3]
    assert np.array_equal(pinned.cpu().numpy(), np.concatenate([np.tile([0, 1, 2], (sy.n_sys, 1)), rest], axis=1))
    # guided search: confirm the top candidates exactly
    first = torch.empty(sy.n_sys, dtype=torch.int32, device="cuda")
    cand = torch.empty((sy.n_sys, K), dtype=torch.uint8, device="cuda")
    pkg.paam_rta_search_ordered(ctx(), b, pkg.analysis_opts(), r, ranked, False, cand, first)
    torch.cuda.synchronize()
    ex = oracle.search(sy, ranks, threads=8)
    guided_ok = cand.cpu().numpy()
    assert not np.any(guided_ok & (ex["cand_ok"] == 0))  # zero false accepts
    found = (first.cpu().numpy() >= 0)
    has = ex["first_ok"] >= 0
    assert not np.any(found & ~has)
    recall = found[has].mean()
    # the same budget spent on a random order of the candidates
    rng = np.random.default_rng(2)
    rand_order = np.stack([rng.permutation(K)[:top] for _ in range(sy.n_sys)])
    rand_found = np.array([ex["cand_ok"][s, rand_order[s]].any() for s in range(sy.n_sys)])
    assert recall >= rand_found[has].mean(), (recall, rand_found[has].mean())
    m.free()
    b.free()


@pytest.mark.parametrize("which", ["trained", "untrained"])
def test_exact_guided_search_gives_the_exhaustive_verdicts(which):
    """paam_surrogate_search (pinned seeds, then the network's order, each system
    stopping at its first admitted candidate) admits exactly the systems the
    exhaustive search admits, each with a candidate the oracle admits, and a
    system admitted by a pinned seed with its lowest such slot; the network's
    quality changes only the time (an untrained network gives the same verdicts).
    Mixed sizes (cfg3, up to 64 chains) and a batch of 16-chain systems."""
    import torch

    import paper_2404_06452_gb300 as pkg

    if which == "trained":
        m, btrain, *_ = _trained_model()
        btrain.free()
    else:
        m = pkg.Model.create(ctx(), seed=3)
    for sy, K, pinned in ((g.generate("cfg4s", n_sys=600), 64, 2), (g.generate("cfg3", n_sys=300, seed=4), 16, 1)):
        ranks = g.candidate_ranks(sy, K, 11, nmax=int(sy.chains_per_system().max()))
        b = pkg.paam_rta_load_systems(ctx(), sy)
        r = torch.from_numpy(ranks).cuda()
        first = torch.full((sy.n_sys,), -7, dtype=torch.int32, device="cuda")
        pkg.paam_surrogate_search(ctx(), m, b, pkg.analysis_opts(), r, first, n_pinned=pinned)
        torch.cuda.synchronize()
        f = first.cpu().numpy()
        ex = oracle.search(sy, ranks, threads=8)
        has = ex["first_ok"] >= 0
        assert np.array_equal(f >= 0, has)
        assert np.all(f >= -1) and np.all(f < K)
        idx = np.nonzero(f >= 0)[0]
        assert np.all(ex["cand_ok"][idx, f[idx]] == 1)  # every admitted candidate is admissible
        seeded = ex["cand_ok"][:, :pinned].any(axis=1)
        assert np.array_equal(f[seeded], ex["cand_ok"][seeded, :pinned].argmax(axis=1))
        b.free()
    m.free()


def test_checkpoint_roundtrip(tmp_path):
    import torch

    import paper_2404_06452_gb300 as pkg

    m = pkg.Model.create(ctx(), 3)
    m.set_params(_random_params(8))
    path = str(tmp_path / "model.bin")
    m.save(path)
    m2 = pkg.Model.load(ctx(), path)
    assert np.array_equal(m.get_params(), m2.get_params())
    sy = g.generate("cfg2", n_sys=300)
    b = pkg.paam_rta_load_systems(ctx(), sy)
    p1 = torch.empty((sy.n_sys, 64), dtype=torch.float32, device="cuda")
    p2 = torch.empty_like(p1)
    pkg.paam_surrogate_predict(ctx(), m, b, p1)
    pkg.paam_surrogate_predict(ctx(), m2, b, p2)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    m.free()
    m2.free()
    b.free()
