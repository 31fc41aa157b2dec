"""Failure detection through the C ABI, with no GPU fault (none of these traps, hangs or
faults the device).

- A bounded device wait that runs out: with SPA_FAULT=stall the likelihood kernel's MMA
  issuer waits on a barrier that nothing arrives at, under a 1 ms limit. The wait runs out,
  the kernel's other roles give up, drain their own copies, free TMEM and return, and the
  sweep reports SPA_ETIMEOUT. Without the stall the same context reproduces a clean sweep bit
  for bit, under the short limit and the default one.
- Host-side injection (SPA_FAULT): failed device allocations give SPA_ENOMEM, a NaN log-weight
  gives SPA_ENUMERIC; a NaN particle handed to the log-likelihood gives SPA_ENUMERIC; bad
  schedules and sizes give SPA_EINVAL. After each, the context runs a clean sweep again.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spa():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as spa

    return spa


@pytest.fixture(scope="module")
def region():
    from paper_1106_0322_gb300 import synth

    return synth.make_region(300, 12, 0.9, (0.5, -0.4), seed=21)


def _same(a, b):
    for k in ("mean", "quantile", "conc", "ess", "log_z_inc", "accept_rate", "resampled"):
        assert np.array_equal(a[k], b[k]), k


SCHED = np.exp(np.linspace(-5.0, 0.0, 5))


@pytest.mark.parametrize("move", ["rw", "mala"])
def test_a_wait_that_runs_out_reports_etimeout_and_the_context_recovers(spa, region, move, monkeypatch):
    cfg = spa.make_config(move=move)
    with spa.Region(region.G, region.y, 1.0, config=cfg) as r:
        ref = r.run(SCHED, 512, 2, seed=5)
        r.set_wait_limit(1_000_000)  # 1 ms
        monkeypatch.setenv("SPA_FAULT", "stall")
        with pytest.raises(spa.SpaError) as err:
            r.run(SCHED, 512, 2, seed=5)
        assert err.value.code == spa.SPA_ETIMEOUT
        assert "bounded device wait" in str(err.value)
        # the per-step entry points report it the same way
        with pytest.raises(spa.SpaError) as err:
            r.loglik(np.zeros((256, region.G.shape[1]), np.float32))
        assert err.value.code == spa.SPA_ETIMEOUT
        monkeypatch.delenv("SPA_FAULT")
        # with nothing stalled, the short limit does not end waits that complete
        _same(ref, r.run(SCHED, 512, 2, seed=5))
        r.set_wait_limit(0)  # back to the default
        _same(ref, r.run(SCHED, 512, 2, seed=5))
        ll = r.loglik(np.zeros((256, region.G.shape[1]), np.float32))
        assert np.allclose(ll, -region.G.shape[0] * np.log(2.0), rtol=1e-6)


def test_a_nan_particle_gives_enumeric(spa, region):
    p = region.G.shape[1]
    for prec in ("split_bf16", "fp32"):
        with spa.Region(region.G, region.y, 1.0, config=spa.make_config(precision=prec)) as r:
            B = np.zeros((64, p), np.float32)
            B[17, 3] = np.nan
            with pytest.raises(spa.SpaError) as err:
                r.loglik(B)
            assert err.value.code == spa.SPA_ENUMERIC
            B[17, 3] = 0.0
            ll = r.loglik(B)
            assert np.all(np.isfinite(ll))


def test_injected_nan_weight_gives_enumeric(spa, region, monkeypatch):
    with spa.Region(region.G, region.y, 1.0) as r:
        ref = r.run(SCHED, 512, 2, seed=9)
        monkeypatch.setenv("SPA_FAULT", "nan_weight")
        with pytest.raises(spa.SpaError) as err:
            r.run(SCHED, 512, 2, seed=9)
        assert err.value.code == spa.SPA_ENUMERIC
        monkeypatch.delenv("SPA_FAULT")
        _same(ref, r.run(SCHED, 512, 2, seed=9))


def test_injected_allocation_failure_gives_enomem(spa, region, monkeypatch):
    monkeypatch.setenv("SPA_FAULT", "alloc")
    with pytest.raises(spa.SpaError) as err:
        spa.Region(region.G, region.y, 1.0)
    assert err.value.code == spa.SPA_ENOMEM
    monkeypatch.delenv("SPA_FAULT")
    with spa.Region(region.G, region.y, 1.0) as r:
        ref = r.run(SCHED, 512, 2, seed=3)
        monkeypatch.setenv("SPA_FAULT", "alloc")
        with pytest.raises(spa.SpaError) as err:
            r.run(SCHED, 1024, 2, seed=3)  # a new particle count needs a new workspace
        assert err.value.code == spa.SPA_ENOMEM
        monkeypatch.delenv("SPA_FAULT")
        _same(ref, r.run(SCHED, 512, 2, seed=3))


def test_bad_schedules_and_sizes_give_einval(spa, region):
    with spa.Region(region.G, region.y, 1.0) as r:
        ref = r.run(SCHED, 512, 2, seed=4)
        for bad in ([0.1, 0.0, 1.0], [0.1, -1.0], [0.1, np.nan], [np.inf, 1.0]):
            with pytest.raises(spa.SpaError) as err:
                r.run(np.array(bad), 512, 2, seed=4)
            assert err.value.code == spa.SPA_EINVAL
        for N, M in ((0, 2), (512, -1), ((1 << 22) + 1, 2)):
            with pytest.raises(spa.SpaError) as err:
                r.run(SCHED, N, M, seed=4)
            assert err.value.code == spa.SPA_EINVAL
        _same(ref, r.run(SCHED, 512, 2, seed=4))
