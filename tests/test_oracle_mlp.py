"""Pins of the oracle's learned-model reference (oracle/mlp.py): the analytic
loss gradient equals central finite differences of the loss, and the features
map the solver's domain onto the unit square."""
import numpy as np
import pytest

from oracle import mlp


def test_parameter_count_matches_architecture():
    assert mlp.NPARAM == 2 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4417


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, mlp.NPARAM)
    y = np.exp(rng.uniform(-3, 6, 40))
    P = rng.integers(2, 33, 40)
    x = mlp.features(y, P)
    t = rng.uniform(0.2, 1.0, 40)
    _, g = mlp.loss_and_grad(theta, x, t)
    idx = np.r_[rng.choice(mlp.NPARAM, 60, replace=False), mlp.NPARAM - 1, 0, 200]
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, x, t)[0] - mlp.loss_and_grad(tm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_features_cover_unit_square():
    x = mlp.features(np.array([0.0, 1000.0]), np.array([2, 32]))
    assert np.allclose(x, [[0.0, 0.0], [1.0, 1.0]])
    assert mlp.dsilu(0.0) == pytest.approx(0.5)
