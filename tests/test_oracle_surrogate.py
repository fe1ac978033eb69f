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


def test_bf16_rounding_definition():
    """Round to nearest with ties to even on the 8-bit significand of
    bfloat16 (Intel BF16 specification; IEEE 754 roundTiesToEven): values
    checked against their binary expansions."""
    x = np.array([1.0, 1 + 2 ** -8, 1 + 2 ** -7, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 65504.0, 2 ** -130,
                  -(1 + 5 * 2 ** -9), 0.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 65536.0, 2 ** -130,
                     -(1 + 2 ** -7), 0.0])
    assert np.array_equal(mlp.bf16(x), want)
    r = np.random.default_rng(3).uniform(-1e3, 1e3, 10000)
    y = mlp.bf16(r)
    assert np.array_equal(mlp.bf16(y), y)  # idempotent
    assert np.all(np.abs(y - r) <= (2.0 ** -8 + 2.0 ** -23) * np.abs(r))  # half an ulp of 8 bits (after float32)


def test_bf16_storage_network_is_the_same_function_up_to_rounding():
    """With every stored value rounded to bf16 the loss and gradients stay
    within a few bf16 roundings of the float64 network; the magnitude sums it
    returns bound each gradient element, and they equal the exact gradient
    where every product has one sign."""
    rng = np.random.default_rng(4)
    P = sum(a * b + b for a, b in mlp.SIZES)
    p = rng.uniform(-1, 1, P) * 0.05
    X = mlp.bf16(rng.uniform(0, 1, (256, 1024)))
    L = rng.uniform(0, 2, (256, 64))
    L[:, 40:] = -1
    l64, g64 = mlp.loss_and_grad(p, X, L)
    l16, g16, scale = mlp.loss_and_grad_bf16(p, X, L)
    assert abs(l16 - l64) <= 2e-2 * l64
    assert np.linalg.norm(g16 - g64) <= 3e-2 * np.linalg.norm(g64)
    assert np.all(np.abs(g16) <= scale * (1 + 1e-12))
    # the first layer's inputs are all >= 0, so its bias gradient's magnitude sum
    # is |sum| exactly when a column of the back-propagated gradient keeps one sign
    o = 1024 * 256
    gb, sb = g16[o:o + 256], scale[o:o + 256]
    assert np.all((np.abs(gb) < sb) | np.isclose(np.abs(gb), sb))
