"""End-to-end pins of the oracle's SMC sweep (Section 4) against quadrature.

For p <= 2 every target pi_t can be integrated on a grid, so the oracle's
per-scale posterior means, concentrations V(Delta), quantiles and evidence
estimates Z_t (products of the Z_t/Z_{t-1} estimates, Section 4) are compared with
the quadrature values. The Monte Carlo standard error comes from independent seeds.
The fixed-scale runs follow the paper's validation recipe (Section 4.2): run MCMC at
one fixed scale and compare with the SMC sampler's answer there.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1106_0322_gb300 import synth
from tests.quadrature import Posterior

R_SEEDS = 8


def _zscores(est, truth, floor):
    est = np.asarray(est)
    m = est.mean(axis=0)
    se = est.std(axis=0, ddof=1) / math.sqrt(est.shape[0])
    return np.abs(m - truth) / (se + floor)


def _check(z, name):
    """Standardised errors: none beyond 6, and on average chi-square-like (E z^2 ~ 1.4
    for a t distribution with R - 1 = 7 degrees of freedom). A handful of comparisons is
    too few to average, so there only the maximum is bounded (by 4.5)."""
    z = np.asarray(z).ravel()
    if z.size < 20:
        assert np.max(z) < 4.5, f"{name}: max z {np.max(z):.2f}"
        return
    assert np.max(z) < 6.0, f"{name}: max z {np.max(z):.2f}"
    assert np.mean(z ** 2) < 3.0, f"{name}: mean z^2 {np.mean(z ** 2):.2f}"


def _runs(reg, a, sched, N, M, move="rw", init="prior_is", burn=0):
    cfg = oracle.make_config(move=move, init=init, burn_in_steps=burn)
    return [oracle.run(reg.G, reg.y, a, sched, N, M, seed=100 + s, cfg=cfg) for s in range(R_SEEDS)]


# (p, a, move, direction). "d2s" is the paper's direction (diffuse to sparse, b_t
# decreasing, Section 4) started by MCMC at the diffuse end (Section 4.1); "s2d" goes
# sparse to diffuse from prior importance sampling. The latter degenerates when the
# sparse-end posterior has a mode the prior rarely visits, so it is pinned on a
# region where it does not (p = 1, heavy-tailed a = 1).
#
# The last entry is the sparse end of the path, log c. For p = 2, a = 4 the posterior of
# the second coefficient splits into a spike at 0 and a slab near the effect as c falls,
# and with 4 random-walk moves per step at N = 2048 the SMC estimate of its mean is biased
# below log c ~ -4.5 (32 seeds: bias 0.06 at log c = -6, 0.018 at -5, none resolvable at
# -4.4): a property of the algorithm at this budget, so the quadrature pin stops there.
SWEEPS = [(1, 1.0, "rw", "s2d", 0.9, -6.0), (2, 4.0, "rw", "d2s", 0.9, -4.5), (2, 2.0, "mala", "d2s", 0.9, -6.0),
          (1, math.inf, "rw", "d2s", 0.9, -6.0), (2, 1.0, "rw", "d2s", 0.9, -6.0),
          (2, 4.0, "site", "d2s", 0.9, -4.5), (1, 1.0, "site", "s2d", 0.9, -6.0)]


@pytest.mark.parametrize("p,a,move,direction,rho,lo", SWEEPS)
def test_smc_sweep_matches_quadrature(p, a, move, direction, rho, lo):
    reg = synth.make_region(200, p, rho, (0.6,) * p, seed=2024 + p)
    sched = synth.geometric_schedule(16, lo, 0.0, sparse_to_diffuse=(direction == "s2d"))
    init = "prior_is" if direction == "s2d" else "mcmc"
    runs = _runs(reg, a, sched, N=2048, M=4, move=move, init=init, burn=25)
    post = Posterior(reg.G, reg.y, a, sched)
    T = sched.size
    truth_mean = np.array([post.mean(c) for c in sched])
    truth_conc = np.array([[post.conc(c, d) for d in (0.05, 0.1)] for c in sched])  # (T, 2, p)
    truth_logz = np.array([post.log_z(c) for c in sched])

    _check(_zscores([r["mean"] for r in runs], truth_mean, 2e-4), "mean")
    conc = np.stack([r["conc"].transpose(0, 2, 1) for r in runs])  # (R, T, D, p)
    _check(_zscores(conc, truth_conc, 2e-3), "conc")
    logz = np.stack([np.cumsum(r["log_z_inc"]) for r in runs])
    _check(_zscores(logz, truth_logz, 2e-3), "log Z")
    # the sampler did its work: resampling happened and moves were accepted
    assert all(r["resampled"].any() for r in runs)
    acc = np.mean([r["accept_rate"] for r in runs])
    assert 0.05 < acc < 0.95
    if p == 1:
        q_levels = (0.05, 0.5, 0.95)
        F = np.array([[[post.cdf(sched[t], 0, r["quantile"][t, 0, k]) for k in range(3)]
                       for t in range(T)] for r in runs])
        _check(_zscores(F, np.array(q_levels)[None, :], 2e-3), "quantiles")


@pytest.mark.parametrize("move,a", [("rw", 1.0), ("mala", 4.0), ("site", 2.0)])
def test_fixed_scale_mcmc_matches_quadrature(move, a):
    # Section 4.2: MCMC at a fixed scale, started with burn-in from prior draws.
    reg = synth.make_region(200, 2, 0.9, (0.5, -0.4), seed=77)
    c = 0.05
    sched = np.full(6, c)
    runs = _runs(reg, a, sched, N=2048, M=5, move=move, init="mcmc", burn=20)
    post = Posterior(reg.G, reg.y, a, [c])
    _check(_zscores([r["mean"][-1] for r in runs], post.mean(c), 2e-4), "fixed-c mean")
    conc = np.stack([r["conc"][-1].T for r in runs])
    truth = np.array([post.conc(c, d) for d in (0.05, 0.1)])
    _check(_zscores(conc, truth, 2e-3), "fixed-c conc")
    for r in runs:
        # constant scale: after the resample-move start no reweighting happens, so the
        # weights stay equal, nothing is resampled and Z_t / Z_{t-1} = 1
        assert not r["resampled"].any()
        assert np.allclose(r["ess"], 2048.0)
        assert np.all(r["log_z_inc"][1:] == 0.0)


def test_run_is_deterministic_and_thread_count_free():
    reg = synth.make_region(120, 6, 0.9, (0.5,), seed=3)
    sched = synth.geometric_schedule(5, -4.0, 0.0)
    r1 = oracle.run(reg.G, reg.y, 1.0, sched, 256, 2, seed=9, cfg=oracle.make_config(n_threads=1))
    r2 = oracle.run(reg.G, reg.y, 1.0, sched, 256, 2, seed=9, cfg=oracle.make_config(n_threads=4))
    for k in r1:
        assert np.array_equal(r1[k], r2[k]), k


def test_run_rejects_bad_input():
    reg = synth.make_region(50, 3, 0.9, (0.5,), seed=3)
    with pytest.raises(ValueError):
        oracle.run(reg.G, reg.y, 1.0, np.array([0.1, -0.2]), 16, 1, seed=1)
    with pytest.raises(ValueError):
        oracle.run(reg.G, reg.y, 0.0, np.array([0.1]), 16, 1, seed=1)
    G = reg.G.copy()
    G[:, 1] = 1
    with pytest.raises(ValueError):
        oracle.run(G, reg.y, 1.0, np.array([0.1]), 16, 1, seed=1)


@pytest.mark.slow
def test_bimodal_sparse_end_matches_quadrature_with_a_larger_budget():
    """The p = 2, a = 4 random-walk sweep down to log c = -6, where the default budget
    (T = 16 steps, N = 2048, 4 moves per step) leaves the slab coefficient's mean biased: with
    a finer schedule (T = 64, so the particle system changes less per step) and twice the
    particles and moves, the oracle matches quadrature of every pi_t over the whole path,
    the bimodal sparse end included (measured: the bias there falls from 0.035 to 0.003)."""
    reg = synth.make_region(200, 2, 0.9, (0.6,) * 2, seed=2024 + 2)
    a = 4.0
    sched = synth.geometric_schedule(64, -6.0, 0.0, sparse_to_diffuse=False)
    runs = _runs(reg, a, sched, N=4096, M=8, move="rw", init="mcmc", burn=25)
    post = Posterior(reg.G, reg.y, a, sched)
    truth_mean = np.array([post.mean(c) for c in sched])
    truth_conc = np.array([[post.conc(c, d) for d in (0.05, 0.1)] for c in sched])
    truth_logz = np.array([post.log_z(c) for c in sched])
    _check(_zscores([r["mean"] for r in runs], truth_mean, 2e-4), "mean")
    _check(_zscores(np.stack([r["conc"].transpose(0, 2, 1) for r in runs]), truth_conc, 2e-3), "conc")
    _check(_zscores(np.stack([np.cumsum(r["log_z_inc"]) for r in runs]), truth_logz, 2e-3), "log Z")
    # the slab coefficient's posterior at the sparse end is genuinely split: most of its mass
    # in the spike at 0, a tenth of it away from 0 (otherwise this would not test the
    # bimodal regime)
    v = post.conc(sched[-1], 0.05)
    assert 0.05 < np.max(v) < 0.5
