"""Pins of the learned-control-variate reference (oracle/qsel_mlp.py): the
backward pass against central finite differences, bfloat16 rounding and GELU
against known values, the features against closed forms on the grid."""
import math

import numpy as np
import pytest

import qsel_inputs as qi
from oracle import qsel_mlp as m
from oracle import qsel_oracle as o
from tests.models import grid_model, theta


def _params(seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, 0.4, (64, 14)), "b1": rng.normal(0, 0.1, 64),
            "W2": rng.normal(0, 0.2, (64, 64)), "b2": rng.normal(0, 0.1, 64),
            "W3": rng.normal(0, 0.2, (1, 64)), "b3": rng.normal(0, 0.1, 1),
            "mu": rng.normal(0, 1, 14), "scale": rng.uniform(0.5, 2.0, 14)}


def test_backward_matches_central_differences():
    P = _params()
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (7, 14))
    y = rng.normal(0, 1, 7)
    _, g = m.loss_and_grad(P, X, y, bf16=False)
    h = 1e-6
    for name, idx in (("W1", (3, 5)), ("b1", (7,)), ("W2", (10, 20)), ("b2", (63,)), ("W3", (0, 11)), ("b3", (0,))):
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][idx] += h
        Pm[name][idx] -= h
        fd = (m.loss_and_grad(Pp, X, y, False)[0] - m.loss_and_grad(Pm, X, y, False)[0]) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), name


def test_bf16_rounding_and_gelu_values():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie (to even: 1), 1 + 3*2^-9 rounds up to 1 + 2^-7
    np.testing.assert_array_equal(m.bf16_round([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.0, 0.0]),
                                  [1.0, 1.0, 1 + 2 ** -7, -2.0, 0.0])
    assert m.gelu(np.array([0.0]))[0] == 0.0
    assert abs(m.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    assert abs(m.gelu(np.array([10.0]))[0] - 10.0) < 1e-12


def test_features_closed_forms_on_grid():
    mdl = grid_model(6, 5, obs_frac=0.3)
    th = theta(0.5, 1.3, 0.8)
    ss = o.balanced_slab_start(5, 2)          # parts [0,3) and [3,5)
    F = m.features(mdl, th, ss, 1)
    Q = o.precision(mdl, th).toarray()
    n_s = 36
    np.testing.assert_allclose(F[:, 0], np.log(np.diag(Q)), rtol=1e-13)
    # boundary distance on a 6x6 grid: min(x, y, 5 - x, 5 - y)
    xs, ys = np.divmod(np.arange(n_s), 6)
    bd = np.minimum(np.minimum(xs, ys), np.minimum(5 - xs, 5 - ys))
    np.testing.assert_array_equal(F[:n_s, 10], bd)
    # ext = [0,4) sep {4}; ext = [2,5) sep {1}
    np.testing.assert_array_equal(F[::n_s, 9], [4, 3, 2, 2, 3])
    np.testing.assert_allclose(F[0, 11:14], th)
    r = 2 * n_s + 14
    row = np.abs(Q[r].copy())
    row[r] = 0
    top = np.sort(row[row > 0])[::-1][:8]
    np.testing.assert_allclose(F[r, 1:9], np.log(top), rtol=1e-13)


def test_feature_distance_caps():
    # 20x20 grid: the boundary distance min(x, y, 19 - x, 19 - y) reaches 9,
    # capped at 8; one part has no separator, so every slab gets the cap
    mdl = grid_model(20, 3, obs_frac=0.3)
    th = theta(0.5, 1.3, 0.8)
    F = m.features(mdl, th, [0, 3], 1)
    xs, ys = np.divmod(np.arange(400), 20)
    bd = np.minimum(np.minimum(np.minimum(xs, ys), np.minimum(19 - xs, 19 - ys)), 8)
    assert bd.max() == 8 and (np.minimum(np.minimum(xs, ys), np.minimum(19 - xs, 19 - ys)) == 9).any()
    np.testing.assert_array_equal(F[:400, 10], bd)
    np.testing.assert_array_equal(F[::400, 9], [m.SEPARATOR_CAP] * 3)
    # 40 slabs in 2 parts with overlap 1: ext [0,21) sep {21}; slab 0 is 21 away, capped
    sep = m.separator_distance(40, o.balanced_slab_start(40, 2), 1)
    assert sep[0] == m.SEPARATOR_CAP and sep[19] == 2 and sep[20] == 2 and sep[39] == m.SEPARATOR_CAP
