"""Pins of the oracle's MAP by EM (Section 2.1, eqs. beta_it and adapt_weights).

For the double exponential (a = inf) every EM weight is 1/c, so the MAP is the L1-penalised
logistic regression of X_std on y with penalty 1/c: scikit-learn's solver gives it
independently. For finite a the EM fixed point must be a stationary point of the log
posterior l(beta) + sum_j log p(beta_j | a, c): d/dbeta_j = 0 where beta_j != 0, and
|dl/dbeta_j| <= (a+1)/(a c) where beta_j = 0 (the prior's cusp). And EM never lowers the
log posterior of its start.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1106_0322_gb300 import synth


def _xstd(G):
    G = G.astype(np.float64)
    return (G - G.mean(0)) / G.std(0)


def _grad_loglik(X, y, b):
    eta = X @ b
    return X.T @ (y - 1.0 / (1.0 + np.exp(-eta)))


def _logpost(X, y, b, a, c):
    eta = X @ b
    ll = np.sum(y * eta - (np.maximum(eta, 0) + np.log1p(np.exp(-np.abs(eta)))))
    x = np.abs(b)
    lp = np.sum(-np.log(2 * c) - x / c) if math.isinf(a) else np.sum(-np.log(2 * c) - (a + 1) * np.log1p(x / (a * c)))
    return ll + lp


@pytest.mark.parametrize("c", [0.02, 0.1, 1.0])
def test_double_exponential_map_is_l1_logistic_regression(c):
    lm = pytest.importorskip("sklearn.linear_model")
    reg = synth.make_region(400, 12, 0.9, (0.6, -0.4, 0.3), seed=31)
    X, y = _xstd(reg.G), reg.y.astype(np.float64)
    b, _ = oracle.map_em(reg.G, reg.y, math.inf, c, np.zeros(12))
    sk = lm.LogisticRegression(penalty="l1", C=c, fit_intercept=False, solver="liblinear", tol=1e-10, max_iter=100000)
    sk.fit(X, reg.y)
    ref = sk.coef_.ravel()
    assert np.max(np.abs(b - ref)) < 2e-4 * max(1.0, np.max(np.abs(ref)))
    assert np.array_equal(b == 0.0, np.abs(ref) < 1e-6)


@pytest.mark.parametrize("a,c", [(1.0, 0.01), (4.0, 0.05), (2.0, 0.5)])
def test_em_fixed_point_is_stationary_and_improves(a, c):
    reg = synth.make_region(300, 10, 0.9, (0.6, -0.5), seed=32)
    X, y = _xstd(reg.G), reg.y.astype(np.float64)
    rng = np.random.default_rng(4)
    b0 = rng.normal(0, 0.2, 10)
    b, lp = oracle.map_em(reg.G, reg.y, a, c, b0)
    assert abs(lp - _logpost(X, y, b, a, c)) < 1e-8 * abs(lp)
    assert lp >= _logpost(X, y, b0, a, c) - 1e-9
    g = _grad_loglik(X, y, b)
    nz = b != 0.0
    wj = (a + 1) / (a * c + np.abs(b))
    assert np.all(np.abs(g[nz] - wj[nz] * np.sign(b[nz])) < 1e-6 * np.maximum(1.0, wj[nz]))
    assert np.all(np.abs(g[~nz]) <= (a + 1) / (a * c) * (1 + 1e-9))
