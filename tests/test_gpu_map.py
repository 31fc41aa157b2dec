"""MAP by EM on the GPU (Section 2.1) and the MAP path along a sweep (Section 4.1).

From the same starting point the GPU's EM (FP32 proximal-gradient inner solves) and the
oracle's (FP64 coordinate descent to convergence) follow the same EM iterates up to the
inner solves' accuracy and must reach the same local mode. Along a sweep the MAP at each
step must be a stationary point of that step's log posterior.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1106_0322_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spa():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as mod

    return mod


def _xstd(G):
    G = G.astype(np.float64)
    return (G - G.mean(0)) / G.std(0)


def _logpost(X, y, b, a, c):
    eta = X @ b
    ll = np.sum(y * eta - (np.maximum(eta, 0) + np.log1p(np.exp(-np.abs(eta)))))
    x = np.abs(b)
    lp = np.sum(-np.log(2 * c) - x / c) if math.isinf(a) else np.sum(-np.log(2 * c) - (a + 1) * np.log1p(x / (a * c)))
    return ll + lp


@pytest.mark.parametrize("a,c", [(1.0, 0.02), (4.0, 0.1), (math.inf, 0.05), (2.0, 1.0)])
def test_map_matches_oracle(spa, a, c):
    reg = synth.make_region(500, 24, 0.9, (0.6, -0.5, 0.3), seed=41)
    rng = np.random.default_rng(5)
    starts = np.stack([np.zeros(24), rng.normal(0, 0.3, 24), rng.laplace(0, 0.05, 24)]).astype(np.float32)
    with spa.Region(reg.G, reg.y, a) as r:
        g, glp = r.map(starts, c, max_em=500, tol=1e-6)
    X, y = _xstd(reg.G), reg.y.astype(np.float64)
    for s in range(starts.shape[0]):
        o, olp = oracle.map_em(reg.G, reg.y, a, c, starts[s].astype(np.float64), max_em=500, tol=1e-10)
        assert np.max(np.abs(g[s] - o)) < 2e-3 * max(1.0, np.max(np.abs(o))), s
        assert abs(glp[s] - olp) < 1e-4 * abs(olp) + 1e-3, s
        assert abs(glp[s] - _logpost(X, y, g[s].astype(np.float64), a, c)) < 1e-6 * abs(glp[s]) + 1e-6


def test_map_path_is_stationary_along_the_sweep(spa):
    reg = synth.make_region(400, 16, 0.9, (0.5, -0.4), seed=42)
    a = 4.0
    sched = synth.paper_schedule(1.0, 12, a, ratio=0.8)  # diffuse to sparse, as in the paper
    cfg = spa.make_config(map_path=True, init="resample_move", burn_in_steps=5)
    X, y = _xstd(reg.G), reg.y.astype(np.float64)
    with spa.Region(reg.G, reg.y, a, config=cfg) as r:
        r.run(sched, 512, 3, 7)
        m, lp = r.map_path(sched.size, max_em=500, tol=1e-6)
    assert np.all(np.isfinite(m)) and np.all(np.isfinite(lp))
    for t, c in enumerate(sched):
        b = m[t].astype(np.float64)
        assert abs(lp[t] - _logpost(X, y, b, a, c)) < 1e-6 * abs(lp[t]) + 1e-6
        eta = X @ b
        gr = X.T @ (y - 1.0 / (1.0 + np.exp(-eta)))
        w = (a + 1) / (a * c + np.abs(b))
        nz = b != 0.0
        # stationarity of l + log p where beta_j != 0; the cusp's subgradient bound at 0
        assert np.all(np.abs(gr[nz] - w[nz] * np.sign(b[nz])) < 5e-3 * np.maximum(1.0, w[nz])), t
        assert np.all(np.abs(gr[~nz]) <= (a + 1) / (a * c) * (1 + 1e-3) + 1e-3), t
    # the sparse end has the fewest non-zeros
    assert np.count_nonzero(m[-1]) <= np.count_nonzero(m[0])


@pytest.mark.parametrize("a,move", [(4.0, "rw"), (1.0, "site")])
def test_map_path_satisfies_its_recurrence(spa, a, move):
    """S_t is the better of the mode from step t's best particle and EM(c_t, S_{t-1}) (Section
    4.1): EM from S_{t-1} at c_t, run alone, either gives S_t bit for bit or a log posterior no
    higher than S_t's, and the parallel rounds reach that fixed point within T rounds."""
    reg = synth.make_region(300, 12, 0.9, (0.6, -0.5), seed=44)
    T = 24
    sched = synth.paper_schedule(1.0, T, a, ratio=0.8)
    cfg = spa.make_config(map_path=True, move=move, init="resample_move", burn_in_steps=3)
    with spa.Region(reg.G, reg.y, a, config=cfg) as r:
        r.run(sched, 256, 2, 8)
        m, lp = r.map_path(T, max_em=300, tol=1e-6)
        rounds = r.map_path_rounds()
        assert 1 <= rounds <= T
        for t in range(1, T):
            x, xlp = r.map(m[t - 1][None, :], float(sched[t]), max_em=300, tol=1e-6)
            if np.array_equal(x[0].view(np.uint32), m[t].view(np.uint32)):
                assert xlp[0] == lp[t]
            else:
                assert xlp[0] <= lp[t], t
        # a second call is the same computation
        m2, lp2 = r.map_path(T, max_em=300, tol=1e-6)
    assert np.array_equal(m.view(np.uint32), m2.view(np.uint32)) and np.array_equal(lp, lp2)


def test_map_path_needs_a_recorded_run(spa):
    reg = synth.make_region(200, 6, 0.9, (0.5,), seed=43)
    with spa.Region(reg.G, reg.y, 1.0) as r:
        r.run(synth.geometric_schedule(3), 64, 1, 1)
        with pytest.raises(spa.SpaError):
            r.map_path(3)


@pytest.mark.parametrize("seed", [44, 45])
def test_map_path_matches_the_oracle_walk_from_the_same_starts(spa, seed):
    """Section 4.1's rule, GPU (parallel rounds) against the oracle (the steps walked in
    order), from the same starts: the oracle's own sweep records each step's best particle
    (rounded to FP32, the form the GPU takes), and both sides run the path from those. The
    kept modes and their log posteriors must agree at every step, and the chained start must
    win with a mode of its own at some steps, so the comparison exercises the rule."""
    a = 1.0
    reg = synth.make_region(300, 12, 0.9, (0.6, -0.5), seed=seed)
    T = 20
    sched = synth.paper_schedule(1.0, T, a, ratio=0.8)  # diffuse to sparse, as in the paper
    out = oracle.run(reg.G, reg.y, a, sched, 512, 2, seed=8, cfg=oracle.make_config(init="mcmc", burn_in_steps=3),
                     keep_best=True)
    best = out["best"].astype(np.float32)
    om, olp, och = oracle.map_path(reg.G, reg.y, a, sched, best.astype(np.float64), max_em=300, tol=1e-8)
    with spa.Region(reg.G, reg.y, a) as r:
        gm, glp = r.map_path_given(sched, best, max_em=300, tol=1e-6)
        assert 1 <= r.map_path_rounds() <= T
    own_mode = 0
    for t in range(T):
        scale = max(1.0, np.max(np.abs(om[t])))
        assert np.max(np.abs(gm[t] - om[t])) < 2e-3 * scale, t
        assert abs(glp[t] - olp[t]) < 1e-5 * abs(olp[t]) + 1e-4, t
        A, _ = oracle.map_em(reg.G, reg.y, a, float(sched[t]), best[t].astype(np.float64), max_em=300, tol=1e-8)
        if och[t] and np.max(np.abs(A - om[t])) > 1e-3:
            own_mode += 1
    assert own_mode >= 2
