"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each test checks one oracle function against something other than itself:
published known-answer values, closed forms derived from the paper's densities,
quadrature, a second representation of the same quantity (the scale mixture
of Section 2), brute force on tiny inputs, or a library routine.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from paper_1106_0322_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert out.tolist() == r[6:10]


def test_normals_are_standard_normal():
    z = np.concatenate([oracle.normals(11, i, 3, 2, 64) for i in range(2000)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.02
    # Kolmogorov-Smirnov against N(0,1)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct (particle, t, m) give different streams
    a = oracle.normals(11, 5, 3, 2, 16)
    b = oracle.normals(11, 5, 3, 3, 16)
    c = oracle.normals(12, 5, 3, 2, 16)
    assert not np.allclose(a, b) and not np.allclose(a, c)


# ------------------------------------------------------------------------- prior
PRIOR_CASES = [(1.0, 1.0), (1.0, 0.01), (4.0, 0.3), (2.0, 5.0), (16.0, 0.05), (math.inf, 0.2)]


@pytest.mark.parametrize("a,c", PRIOR_CASES)
def test_prior_integrates_to_one(a, c):
    f = lambda b: math.exp(oracle.prior_logpdf(a, c, [b])[0])
    # symmetric: integrate over [0, inf) twice; split at the scale to help quad
    left, _ = integrate.quad(f, 0, a * c if math.isfinite(a) else c, limit=400)
    right, _ = integrate.quad(f, a * c if math.isfinite(a) else c, np.inf, limit=400)
    assert abs(2 * (left + right) - 1.0) < 1e-7


@pytest.mark.parametrize("a,c", [(1.0, 1.0), (4.0, 0.3), (2.0, 5.0)])
def test_prior_tail_closed_form(a, c):
    # integrating eq. gent_prior: P(|beta| > x) = (1 + x/(a c))^(-a)
    f = lambda b: math.exp(oracle.prior_logpdf(a, c, [b])[0])
    for x in [0.1 * c, c, 7.0 * c]:
        tail, _ = integrate.quad(f, x, np.inf, limit=400)
        assert abs(2 * tail - (1 + x / (a * c)) ** (-a)) < 1e-8


@pytest.mark.parametrize("a,c", [(4.0, 0.3), (3.0, 2.0)])
def test_prior_moments(a, c):
    f = lambda b: math.exp(oracle.prior_logpdf(a, c, [b])[0])
    m1, _ = integrate.quad(lambda b: b * f(b), 0, np.inf, limit=400)
    m2, _ = integrate.quad(lambda b: b * b * f(b), 0, np.inf, limit=400)
    assert abs(2 * m1 - a * c / (a - 1)) < 1e-7 * a * c
    assert abs(2 * m2 - 2 * a * a * c * c / ((a - 1) * (a - 2))) < 1e-6 * a * a * c * c


@pytest.mark.parametrize("a,c", [(1.0, 1.0), (4.0, 0.3), (2.0, 0.05)])
def test_prior_scale_mixture(a, c):
    # Section 2, eq. scalemix: beta | tau ~ DE(0, tau), tau ~ IG(a, b) with b = a c
    b = a * c
    ig = stats.invgamma(a, scale=b)
    for beta in [0.0, 0.3 * c, c, 4.0 * c]:
        g = lambda tau: 1.0 / (2 * tau) * math.exp(-abs(beta) / tau) * ig.pdf(tau)
        val = integrate.quad(g, 0, b, limit=400)[0] + integrate.quad(g, b, np.inf, limit=400)[0]
        assert abs(math.log(val) - oracle.prior_logpdf(a, c, [beta])[0]) < 1e-7


def test_prior_double_exponential_limit():
    # a (log p_a(x) - log p_DE(x)) -> x^2/(2c^2) - x/c as a -> infinity
    c = 0.7
    x = np.array([0.1, 0.5, 1.3])
    de = oracle.prior_logpdf(math.inf, c, x)
    assert np.allclose(de, -np.log(2 * c) - x / c, rtol=0, atol=1e-15)
    limit = x ** 2 / (2 * c * c) - x / c
    prev = None
    for a in [1e3, 1e4, 1e5]:
        d = a * (oracle.prior_logpdf(a, c, x) - de)
        err = np.max(np.abs(d - limit))
        if prev is not None:
            assert err < prev / 5
        prev = err
    assert prev < 1e-3
    # Gt(1,1) and DE(0,1) agree at 0 (both -log 2) and Gt(1,1) is heavier in the tail
    assert oracle.prior_logpdf(1.0, 1.0, [0.0])[0] == pytest.approx(-math.log(2), abs=1e-15)
    assert oracle.prior_logpdf(1.0, 1.0, [6.0])[0] > oracle.prior_logpdf(math.inf, 1.0, [6.0])[0]


@pytest.mark.parametrize("a,c", [(1.0, 0.01), (4.0, 0.5), (math.inf, 0.2)])
def test_prior_sampler_matches_cdf(a, c):
    x = oracle.prior_sample(123, a, c, 20000, 2)
    mag = np.abs(x).ravel()
    if math.isfinite(a):
        cdf = lambda t: 1.0 - (1.0 + t / (a * c)) ** (-a)
    else:
        cdf = lambda t: 1.0 - np.exp(-t / c)
    assert stats.kstest(mag, cdf).pvalue > 1e-3
    assert abs(np.mean(x > 0) - 0.5) < 0.02


# ------------------------------------------------------------------- likelihood
def _tiny(n=7, p=3, seed=3):
    reg = synth.make_region(n, p, 0.5, (0.8,), seed=seed)
    return reg.G, reg.y


def test_standardise_matches_numpy():
    G, _ = _tiny(40, 6)
    m, s = oracle.standardise(G)
    assert np.allclose(m, G.mean(axis=0), atol=1e-15)
    assert np.allclose(s, G.std(axis=0, ddof=0), atol=1e-15)


def test_loglik_at_zero_and_symmetry():
    reg = synth.make_region(300, 12, 0.9, (0.5,), seed=5)
    B = np.zeros((1, 12))
    assert oracle.loglik(reg.G, reg.y, B)[0] == pytest.approx(-300 * math.log(2), rel=1e-14)
    B = synth.random_particles(5, 12, 0.3, seed=1).astype(np.float64)
    l1 = oracle.loglik(reg.G, reg.y, B)
    l2 = oracle.loglik(reg.G, (1 - reg.y).astype(np.uint8), -B)
    assert np.allclose(l1, l2, rtol=1e-13, atol=0)


def test_loglik_brute_force_product():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    G, y = _tiny(7, 3, seed=9)
    n, p = G.shape
    B = np.array([[0.3, -1.2, 0.05], [2.0, 0.0, -0.7], [-4.0, 3.0, 1.0]])
    got = oracle.loglik(G, y, B)
    Gm = [[mpmath.mpf(int(v)) for v in row] for row in G]
    for k in range(B.shape[0]):
        prod = mpmath.mpf(1)
        for i in range(n):
            eta = mpmath.mpf(0)
            for j in range(p):
                col = [Gm[r][j] for r in range(n)]
                mean = sum(col) / n
                sd = mpmath.sqrt(sum((v - mean) ** 2 for v in col) / n)
                eta += (Gm[i][j] - mean) / sd * mpmath.mpf(B[k, j])
            pi = 1 / (1 + mpmath.exp(-eta))
            prod *= pi if y[i] == 1 else (1 - pi)
        assert abs(float(mpmath.log(prod)) - got[k]) < 1e-12


def test_gradient_central_differences():
    reg = synth.make_region(150, 8, 0.9, (0.5, -0.3), seed=4)
    B = synth.random_particles(3, 8, 0.4, seed=2).astype(np.float64)
    ll, g = oracle.loglik_grad(reg.G, reg.y, B)
    assert np.allclose(ll, oracle.loglik(reg.G, reg.y, B), rtol=1e-15, atol=0)
    h = 1e-4
    for k in range(3):
        for j in range(8):
            Bp = B[k:k + 1].copy()
            Bm = B[k:k + 1].copy()
            Bp[0, j] += h
            Bm[0, j] -= h
            fd = (oracle.loglik(reg.G, reg.y, Bp)[0] - oracle.loglik(reg.G, reg.y, Bm)[0]) / (2 * h)
            assert abs(fd - g[k, j]) < 1e-6 * max(1.0, abs(g[k, j]))


def test_gradient_at_zero():
    reg = synth.make_region(120, 5, 0.9, (0.5,), seed=6)
    _, g = oracle.loglik_grad(reg.G, reg.y, np.zeros((1, 5)))
    X = (reg.G - reg.G.mean(0)) / reg.G.std(0)
    assert np.allclose(g[0], X.T @ (reg.y - 0.5), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- incremental weight
@pytest.mark.parametrize("a", [1.0, 4.0, math.inf])
def test_incremental_weight(a):
    beta = synth.random_particles(1, 40, 0.2, seed=8)[0].astype(np.float64)
    assert oracle.log_incr_weight(a, 0.3, 0.3, beta) == 0.0
    # closed form with no cancellation (algebraically equal to the difference of log priors)
    cp, cn = 0.31, 0.29
    x = np.abs(beta)
    if math.isfinite(a):
        ref = np.sum(-np.log(cn / cp) - (a + 1) * np.log1p(x * (cp - cn) / (cn * (a * cp + x))))
    else:
        ref = np.sum(-np.log(cn / cp) - x * (1 / cn - 1 / cp))
    assert oracle.log_incr_weight(a, cp, cn, beta) == pytest.approx(ref, rel=1e-9, abs=1e-12)
    # telescoping along a path
    path = [0.5, 0.4, 0.2, 0.15]
    tot = sum(oracle.log_incr_weight(a, path[i], path[i + 1], beta) for i in range(3))
    ref = oracle.prior_logpdf(a, path[-1], beta).sum() - oracle.prior_logpdf(a, path[0], beta).sum()
    assert tot == pytest.approx(ref, rel=1e-12, abs=1e-10)


# ---------------------------------------------------------------------- LSE/ESS
def test_lse_ess():
    rng = np.random.default_rng(0)
    lw = rng.normal(size=1000) * 3 - 50
    lse, ess = oracle.lse_ess(lw)
    assert lse == pytest.approx(special.logsumexp(lw), rel=1e-14)
    w = np.exp(lw - lse)
    assert ess == pytest.approx(w.sum() ** 2 / (w ** 2).sum(), rel=1e-12)
    assert oracle.lse_ess(lw + 123.0)[1] == pytest.approx(ess, rel=1e-12)
    assert oracle.lse_ess(np.full(512, -7.0))[1] == pytest.approx(512.0, rel=1e-14)
    one_hot = np.full(64, -np.inf)
    one_hot[17] = 0.0
    assert oracle.lse_ess(one_hot)[1] == 1.0


# -------------------------------------------------------------------- resampling
def _brute_systematic(W, u):
    C = np.array([math.fsum(W[: i + 1]) for i in range(W.size)])
    N = W.size
    out = []
    for k in range(N):
        t = (k + u) / N
        hits = np.nonzero(C > t)[0]
        out.append(hits[0] if hits.size else N - 1)
    return np.array(out, np.int32), C


@pytest.mark.parametrize("N", [1, 7, 256, 1000, 4099])
def test_resampling_definition(N):
    rng = np.random.default_rng(N)
    W = rng.gamma(0.3, size=N)
    W /= W.sum()
    u = float(rng.random())
    idx = oracle.resample_systematic(W, u)
    ref, C = _brute_systematic(W, u)
    Cb = oracle.cumsum_blocked(W)
    assert np.max(np.abs(Cb - C)) < 1e-14
    # identical except where a target sits within rounding of a cumulative sum
    t = (np.arange(N) + u) / N
    near = np.array([np.min(np.abs(C - tt)) < 1e-13 for tt in t])
    assert np.all((idx == ref) | near)
    assert np.all(np.diff(idx) >= 0)
    counts = np.bincount(idx, minlength=N)
    assert np.all(counts >= np.floor(N * W) - 1) and np.all(counts <= np.ceil(N * W) + 1)


def test_resampling_equal_weights_identity():
    for N in [1, 5, 256, 1024, 3000]:
        W = np.full(N, 1.0 / N)
        # u = 0 puts every target exactly on a cumulative sum, where rounding
        # decides the strict comparison; away from that tie the map is the identity.
        for u in [1e-6, 0.25, 0.999999]:
            assert np.array_equal(oracle.resample_systematic(W, u), np.arange(N, dtype=np.int32))


def test_resampling_one_hot():
    W = np.zeros(100)
    W[42] = 1.0
    assert np.all(oracle.resample_systematic(W, 0.5) == 42)


# -------------------------------------------------------------------- quantiles
def test_weighted_quantile_brute_force():
    rng = np.random.default_rng(1)
    for N in [1, 2, 9, 100, 1001]:
        v = np.round(rng.normal(size=N), 1)  # many ties
        W = rng.random(N)
        W /= W.sum()
        qs = np.array([0.05, 0.5, 0.95])
        got = oracle.weighted_quantile(v, W, qs)
        order = np.lexsort((np.arange(N), v))
        cum = np.cumsum(W[order])
        for q, g in zip(qs, got):
            k = np.nonzero(cum >= q)[0]
            k = k[0] if k.size else N - 1
            # allow the neighbour when the cumulative sum is within rounding of q
            ok = {v[order][k]}
            if k > 0 and abs(cum[k - 1] - q) < 1e-12:
                ok.add(v[order][k - 1])
            if k + 1 < N and abs(cum[k] - q) < 1e-12:
                ok.add(v[order][k + 1])
            assert g in ok
    # equal weights: order statistics
    v = np.arange(10.0)[::-1].copy()
    assert oracle.weighted_quantile(v, np.full(10, 0.1), [0.05, 0.5, 0.95]).tolist() == [0.0, 4.0, 9.0]
