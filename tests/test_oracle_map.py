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


# ------------------------------------------------------------------ the MAP path (Section 4.1)
@pytest.mark.parametrize("seed", [1, 2])
def test_map_path_of_the_double_exponential_is_l1_regression_at_every_scale(seed):
    """With the double exponential the log posterior is concave: each step has one mode,
    whichever start EM takes. So every kept mode is scikit-learn's L1 logistic regression at
    that step's c_t (a wrong scale index or a wrong step's mode fails this)."""
    lm = pytest.importorskip("sklearn.linear_model")
    reg = synth.make_region(300, 8, 0.9, (0.6, -0.4), seed=30 + seed)
    X = _xstd(reg.G)
    T = 6
    sched = np.exp(np.linspace(0.0, -3.5, T))  # diffuse to sparse, as the paper sweeps
    rng = np.random.default_rng(seed)
    best = rng.normal(0, 0.3, (T, 8))
    m, lp, ch = oracle.map_path(reg.G, reg.y, math.inf, sched, best)
    for t, c in enumerate(sched):
        sk = lm.LogisticRegression(penalty="l1", C=c, fit_intercept=False, solver="liblinear", tol=1e-10,
                                   max_iter=100000)
        sk.fit(X, reg.y)
        ref = sk.coef_.ravel()
        assert np.max(np.abs(m[t] - ref)) < 2e-4 * max(1.0, np.max(np.abs(ref))), t
        assert abs(lp[t] - _logpost(X, reg.y.astype(np.float64), m[t], math.inf, c)) < 1e-8 * abs(lp[t])


def _grid_logpost_1d(x, y, a, c, lo, hi, k):
    b = np.linspace(lo, hi, k)
    out = np.empty(k)
    for s in range(0, k, 4096):
        bb = b[s:s + 4096]
        eta = np.outer(x, bb)
        ll = (y[:, None] * eta - (np.maximum(eta, 0) + np.log1p(np.exp(-np.abs(eta))))).sum(0)
        out[s:s + 4096] = ll - np.log(2 * c) - (a + 1) * np.log1p(np.abs(bb) / (a * c))
    return b, out


def test_map_path_keeps_the_better_of_two_modes():
    """One marker, Gt(1, c) prior: the log posterior has a mode at 0 (once c is small enough)
    and a slab mode near the effect. With every step's best particle at 0, EM from it finds
    the spike and EM from the previous MAP stays on the slab while the slab is a mode, so the
    two candidates are the two local modes and keeping the better one must give the global
    maximum at every c_t, found here by brute force on a grid. Keeping the worse mode, or
    comparing at the wrong scale, fails this; the rule must pick each start at some step."""
    rng = np.random.default_rng(8)
    n = 400
    g = rng.binomial(2, 0.3, n).astype(np.int8)
    x = (g - g.mean()) / g.std()
    y = (rng.random(n) < 1.0 / (1.0 + np.exp(-0.35 * x))).astype(np.uint8)
    G = g[:, None]
    a = 1.0
    T = 24
    sched = np.exp(np.linspace(0.0, -7.0, T))
    m, lp, ch = oracle.map_path(G, y, a, sched, np.zeros((T, 1)))
    yd = y.astype(np.float64)
    picked_spike = picked_slab = False
    for t, c in enumerate(sched):
        b, f = _grid_logpost_1d(x, yd, a, c, -0.2, 1.5, 170001)
        # the premise: at most two local maxima (the spike and one slab) on this grid
        interior = (f[1:-1] > f[:-2]) & (f[1:-1] >= f[2:])
        assert interior.sum() <= 2, t
        k = int(np.argmax(f))
        assert abs(m[t, 0] - b[k]) < 2e-5 + 1e-3 * abs(b[k]), (t, m[t, 0], b[k])
        assert abs(lp[t] - f[k]) < 1e-6 * abs(f[k]), t
        if t > 0 and ch[t]:
            picked_slab = True
        if t > 0 and not ch[t] and m[t, 0] == 0.0 and m[t - 1, 0] != 0.0:
            picked_spike = True
    assert picked_slab and picked_spike, ch


def test_recorded_best_particle_has_the_highest_posterior_density():
    """or_run's per-step best particle against a brute-force argmax over the final particles
    of a one-step run, with l and log p from the pinned oracle functions."""
    reg = synth.make_region(200, 6, 0.9, (0.5, -0.3), seed=36)
    sched = np.array([0.05])
    out = oracle.run(reg.G, reg.y, 2.0, sched, 300, 3, seed=4, keep_particles=True, keep_best=True)
    B = out["final_beta"]
    score = oracle.loglik(reg.G, reg.y, B) + oracle.prior_logpdf(2.0, 0.05, B).reshape(B.shape).sum(1)
    k = int(np.argmax(score))
    assert np.array_equal(out["best"][0], B[k])
