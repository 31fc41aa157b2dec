"""Grid quadrature of the SPA posteriors for p <= 2 (test helper).

pi_c(beta) is proportional to exp(l(beta)) * prod_j p(beta_j | a, c), with the
logistic log-likelihood of Section 2 on standardised genotypes (Section 3) and the
Gt(a, c) prior of eq. gent_prior. This module evaluates it independently of the
oracle and the CUDA library (numpy only). It uses tensor-product Gauss-Legendre rules
on sub-intervals whose break points sit at 0 (the prior's cusp), geometrically
close to 0 (the prior's scale a*c), at +-Delta (the concentration thresholds) and
on a regular grid covering the likelihood.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import logsumexp


def axis_rule(c_values, L=3.0, deltas=(0.05, 0.1), nodes=10, lin_step=0.05):
    bp = {0.0, L}
    cmin = min(c_values)
    x = cmin * 1e-4
    while x < L:
        bp.add(x)
        x *= 3.0
    for d in deltas:
        bp.add(d)
    for v in np.arange(lin_step, L, lin_step):
        bp.add(float(v))
    pos = np.array(sorted(b for b in bp if 0.0 <= b <= L))
    g, w = np.polynomial.legendre.leggauss(nodes)
    xs, ws = [], []
    for a0, a1 in zip(pos[:-1], pos[1:]):
        h = 0.5 * (a1 - a0)
        xs.append(a0 + h * (g + 1.0))
        ws.append(h * w)
    xp = np.concatenate(xs)
    wp = np.concatenate(ws)
    x = np.concatenate([-xp[::-1], xp])
    w = np.concatenate([wp[::-1], wp])
    return x, w


def log_prior(beta, a, c):
    b = np.abs(beta)
    if math.isinf(a):
        return -np.log(2 * c) - b / c
    return -np.log(2 * c) - (a + 1.0) * np.log1p(b / (a * c))


def loglik_grid(G, y, betas):
    """l(beta) for a (K, p) array of coefficient vectors."""
    G = G.astype(np.float64)
    X = (G - G.mean(0)) / G.std(0)
    out = np.empty(betas.shape[0])
    step = 4096
    for s in range(0, betas.shape[0], step):
        eta = betas[s:s + step] @ X.T
        out[s:s + step] = eta @ y.astype(np.float64) - np.logaddexp(0.0, eta).sum(axis=1)
    return out


class Posterior:
    """Quadrature of pi_c for every c in `cs`; p must be 1 or 2."""

    def __init__(self, G, y, a, cs, L=3.0, deltas=(0.05, 0.1), nodes=10, lin_step=0.05):
        p = G.shape[1]
        if p not in (1, 2):
            raise ValueError("quadrature only for p <= 2")
        self.p, self.a, self.cs = p, a, np.asarray(cs, dtype=np.float64)
        x, w = axis_rule(self.cs, L=L, deltas=deltas, nodes=nodes, lin_step=lin_step)
        self.x, self.w = x, w
        if p == 1:
            pts = x[:, None]
            lw = np.log(w)
        else:
            X1, X2 = np.meshgrid(x, x, indexing="ij")
            pts = np.stack([X1.ravel(), X2.ravel()], axis=1)
            lw = (np.log(w)[:, None] + np.log(w)[None, :]).ravel()
        self.pts = pts
        self.ll = loglik_grid(G, y, pts)
        self.lw = lw

    def log_joint(self, c):
        return self.ll + log_prior(self.pts, self.a, c).sum(axis=1) + self.lw

    def log_z(self, c):
        return float(logsumexp(self.log_joint(c)))

    def weights(self, c):
        lj = self.log_joint(c)
        return np.exp(lj - logsumexp(lj))

    def mean(self, c):
        return self.weights(c) @ self.pts

    def conc(self, c, delta):
        W = self.weights(c)
        inside = np.abs(self.pts) < delta
        return 1.0 - W @ inside

    def cdf(self, c, j, v):
        """P(beta_j <= v) with linear interpolation of the marginal between nodes."""
        W = self.weights(c)
        xs = self.pts[:, j]
        order = np.argsort(xs, kind="stable")
        xs_s = xs[order]
        cw = np.cumsum(W[order])
        return float(np.interp(v, xs_s, cw))
