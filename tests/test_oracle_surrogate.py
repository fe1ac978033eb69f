"""Pins of the surrogate's float64 oracles: backpropagation against central
finite differences, and the features against a hand-derived case."""
import json
import os

import numpy as np

from oracle import features as ofeat
from oracle import mlp
from paam_gen import tiny

HERE = os.path.dirname(os.path.abspath(__file__))


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = sum(a * b + b for a, b in mlp.SIZES)
    p = rng.uniform(-1, 1, P) * 0.05
    X = rng.uniform(0, 1, (3, 1024))
    L = rng.uniform(0, 2, (3, 64))
    L[:, 40:] = -1
    _, g = mlp.loss_and_grad(p, X, L)
    # one coordinate in each weight and bias block, plus random ones
    idx = list(rng.choice(P, 30, replace=False))
    o = 0
    for fin, fout in mlp.SIZES:
        idx += [o + 7, o + fin * fout + 3]
        o += fin * fout + fout
    for i in idx:
        e = np.zeros(P)
        e[i] = 1e-6
        fd = (mlp.loss_and_grad(p + e, X, L)[0] - mlp.loss_and_grad(p - e, X, L)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-9, (i, fd, g[i])


def test_masked_entries_do_not_contribute():
    rng = np.random.default_rng(1)
    P = sum(a * b + b for a, b in mlp.SIZES)
    p = rng.uniform(-1, 1, P) * 0.05
    X = rng.uniform(0, 1, (4, 1024))
    L = rng.uniform(0, 2, (4, 64))
    L2 = L.copy()
    L[:, 10:] = -1
    L2[:, 10:] = -1
    L2[:, 20] = -5.0  # any negative value masks
    assert np.allclose(mlp.loss_and_grad(p, X, L)[1], mlp.loss_and_grad(p, X, L2)[1])


def test_features_hand_case():
    with open(os.path.join(HERE, "golden", "hand_features.json")) as f:
        case = json.load(f)
    d = dict(chains=[dict(c, cbs=[(e, a) for e, a in c["cbs"]]) for c in case["system"]["chains"]],
             execs=case["system"]["execs"])
    sy = tiny.to_systems([d])
    got = ofeat.system_features(sy, 0)
    want = np.zeros(64 * 16)
    for c, row in enumerate(case["features"]):
        want[c * 16:(c + 1) * 16] = row
    assert np.allclose(got, want, atol=1e-12)
    # the same order given as ranks (chain 0 first) with derived executor priorities
    got2 = ofeat.system_features(sy, 0, rank_row=np.array([0, 1]))
    assert np.allclose(got2, want, atol=1e-12)
