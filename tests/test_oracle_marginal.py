"""Pins of the oracle's scale-marginalised summaries (Section 4, eq. all_particles).

The mixture over the schedule's scales weighs step t by Z_t / Z_1. Pinned here by what
fixes it independently of its formula: equal evidence reduces it to the plain average over
steps; one step with overwhelming evidence reduces it to that step's summaries; the t = 0
evidence cancels; and for p = 1 the oracle's own sweep, run through it, matches grid
quadrature of the scale-marginalised posterior within Monte Carlo error.
"""
import numpy as np

import oracle
from paper_1106_0322_gb300 import synth
from tests.quadrature import Posterior
from tests.test_oracle_smc import _check, _zscores


def _inputs(T=7, p=5, D=2, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 2, T), rng.normal(0, 1, (T, p)), rng.uniform(0, 1, (T, p, D))


def test_equal_evidence_is_the_plain_average():
    _, mean, conc = _inputs()
    r = oracle.marginal(np.zeros(mean.shape[0]), mean, conc)
    assert np.allclose(r["post_c"], 1.0 / mean.shape[0], rtol=0, atol=1e-15)
    assert np.allclose(r["mean"], mean.mean(axis=0), rtol=1e-13, atol=1e-15)
    assert np.allclose(r["conc"], conc.mean(axis=0), rtol=1e-13, atol=1e-15)


def test_dominant_step_gives_its_summaries():
    _, mean, conc = _inputs(seed=1)
    inc = np.zeros(mean.shape[0])
    inc[4] = 800.0  # L_t = 800 for t >= 4, then back down at t = 5
    inc[5] = -800.0
    r = oracle.marginal(inc, mean, conc)
    assert abs(r["post_c"][4] - 1.0) < 1e-300 + 1e-15
    assert np.allclose(r["mean"], mean[4], rtol=1e-14, atol=0)
    assert np.allclose(r["conc"], conc[4], rtol=1e-14, atol=0)


def test_first_increment_cancels_and_weights_sum_to_one():
    inc, mean, conc = _inputs(seed=2)
    a = oracle.marginal(inc, mean, conc)
    inc2 = inc.copy()
    inc2[0] += 123.0
    b = oracle.marginal(inc2, mean, conc)
    assert np.array_equal(a["post_c"], b["post_c"])
    assert abs(a["post_c"].sum() - 1.0) < 1e-14
    # weights follow the running sums: w_t / w_s = exp(L_t - L_s)
    L = np.concatenate([[0.0], np.cumsum(inc[1:])])
    assert np.allclose(np.log(a["post_c"][1:] / a["post_c"][0]), L[1:] - L[0], rtol=1e-10, atol=1e-10)


def test_sweep_marginal_matches_quadrature():
    """p = 1, a = 1: the scale-marginalised posterior mean and V(0.1) from the oracle's sweep
    against sum_t Z(c_t) m(c_t) / sum_t Z(c_t) by quadrature (uniform prior on log c)."""
    reg = synth.make_region(200, 1, 0.9, (0.6,), seed=2025)
    sched = synth.geometric_schedule(16, -6.0, 0.0, sparse_to_diffuse=True)
    cfg = oracle.make_config(move="rw", init="prior_is")
    runs = [oracle.run(reg.G, reg.y, 1.0, sched, 2048, 4, seed=300 + s, cfg=cfg) for s in range(8)]
    post = Posterior(reg.G, reg.y, 1.0, sched)
    lz = np.array([post.log_z(c) for c in sched])
    w = np.exp(lz - lz.max())
    w /= w.sum()
    truth_mean = np.array([w @ np.array([post.mean(c)[0] for c in sched])])
    truth_conc = np.array([w @ np.array([post.conc(c, 0.1)[0] for c in sched])])
    margs = [oracle.marginal(r["log_z_inc"], r["mean"], r["conc"]) for r in runs]
    _check(_zscores([m["mean"] for m in margs], truth_mean, 2e-4), "marginal mean")
    _check(_zscores([m["conc"][:, 1] for m in margs], truth_conc, 2e-3), "marginal V(0.1)")
    _check(_zscores([m["post_c"] for m in margs], w, 2e-3), "p(c | X, y)")
