"""Sweep parity at the benchmarked shapes, in the launch configuration the benchmark times.

The hit-region workload (n = 2000, p = 200, N = 8192, M = 10 random-walk moves, a = 1) and
the MALA workload (the same shape, a = 2, M = 5 MALA moves driven by the tensor-core
adjoint) run on the GPU exactly as in bench.py -- same N, n, p and M, so the same tuned
n-tile width, particle-resident likelihood kernel, adjoint K-split and vectorised move path
-- for the first STEPS scale steps of their schedules. The oracle runs the same prefix.

SMC is randomized, so the two are compared in distribution over R seeds per side (the
two-sample standardised differences of the posterior means, the concentrations V(Delta) and
the cumulative log-evidence, with the reading of "within 3 Monte Carlo standard errors"
written out in _check). With the same seed both sides draw the same prior particles and the
same random streams, so the first step's evidence, ESS and resampling decision agree to the
likelihood's rounding.
"""
import numpy as np
import pytest

import oracle
from paper_1106_0322_gb300 import synth
from tests.test_gpu_parity import split_bound
from tests.test_gpu_sweep import _two_sample_z
from tests.test_oracle_smc import _check

pytestmark = pytest.mark.gpu

R = 8
STEPS = 6


@pytest.fixture(scope="module")
def spa():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as mod

    return mod


@pytest.mark.parametrize("name", ["hit-region", "mala"])
def test_benchmarked_workload_prefix_matches_oracle(spa, name):
    w = synth.WORKLOADS[name]
    reg = synth.workload_region(name)
    sched = synth.workload_schedule(name)[:STEPS]
    cfg = spa.make_config(move=w["move"])
    with spa.Region(reg.G, reg.y, w["nu"], config=cfg) as r:
        g = [r.run(sched, w["N"], w["M"], s) for s in range(1, R + 1)]
        same = r.run(sched, w["N"], w["M"], 5)
        assert r.loglik_tile_width() in (128, 224, 256)
    ocfg = oracle.make_config(move=w["move"])
    o = [oracle.run(reg.G, reg.y, w["nu"], sched, w["N"], w["M"], seed=100 + s, cfg=ocfg) for s in range(R)]
    _check(_two_sample_z([x["mean"] for x in g], [x["mean"] for x in o], 2e-4), f"{name} mean")
    _check(_two_sample_z([x["conc"] for x in g], [x["conc"] for x in o], 2e-3), f"{name} conc")
    _check(_two_sample_z([np.cumsum(x["log_z_inc"]) for x in g], [np.cumsum(x["log_z_inc"]) for x in o], 2e-3),
           f"{name} log Z")
    _check(_two_sample_z([x["accept_rate"] for x in g], [x["accept_rate"] for x in o], 2e-3), f"{name} acceptance")
    for x in g:
        assert np.all(x["ess"] >= 1.0) and np.all(x["ess"] <= w["N"] * (1 + 1e-9))
    # the same seed: identical prior draws at t = 0 (the prior is drawn in FP32 on the GPU),
    # so the evidence LSE(l) - log N moves by at most the largest per-particle likelihood
    # error d, whose split-BF16 bound is computed for these draws, and the ESS by a factor of
    # at most e^(4d) (each weight moves by e^(+-d))
    draws = spa.prior_sample(5, w["nu"], float(sched[0]), w["N"], w["p"])
    d = float(np.max(split_bound(reg.G, draws, w["p"])))
    ref = oracle.run(reg.G, reg.y, w["nu"], sched, w["N"], w["M"], seed=5, cfg=ocfg)
    assert abs(same["log_z_inc"][0] - ref["log_z_inc"][0]) <= d
    assert abs(same["ess"][0] - ref["ess"][0]) <= np.expm1(4 * d) * ref["ess"][0]
    if abs(ref["ess"][0] - 0.75 * w["N"]) > np.expm1(4 * d) * ref["ess"][0]:
        assert same["resampled"][0] == ref["resampled"][0]
