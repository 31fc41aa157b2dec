"""The batched sweep: R regions captured into one CUDA graph (one branch per region).

Each branch runs the same kernels on the region's own buffers, every reduction has a fixed
order, and the only atomics are integer counters, so a region's results in the batch must
equal its own spa_run with the same seed bit for bit, whatever the other branches do.
"""
import numpy as np
import pytest

from paper_1106_0322_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spa():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as mod

    return mod


# (n, p, nu, N, T, M, move, precision): uneven shapes, p both a multiple of 4 and not
SHAPES = [
    (300, 7, 1.0, 256, 6, 2, "rw", "split_bf16"),
    (1200, 64, 2.0, 1024, 5, 3, "mala", "split_bf16"),
    (700, 33, 16.0, 512, 4, 2, "rw", "fp32"),
    (2000, 130, 4.0, 1024, 4, 2, "mala", "split_bf16"),
    (1000, 250, float("inf"), 768, 3, 2, "rw", "split_bf16"),
    (500, 20, 1.0, 384, 5, 1, "mala", "fp32"),
]


def _regions(spa):
    regs = []
    for k, (n, p, nu, N, T, M, move, prec) in enumerate(SHAPES):
        g = synth.make_region(n, p, 0.9, (0.4, -0.3), seed=700 + k)
        regs.append(spa.Region(g.G, g.y, nu, config=spa.make_config(move=move, precision=prec)))
    return regs


def test_batch_graph_matches_individual_runs(spa):
    regs = _regions(spa)
    scheds = [synth.geometric_schedule(s[4]) for s in SHAPES]
    Ns = [s[3] for s in SHAPES]
    Ms = [s[5] for s in SHAPES]
    try:
        b = spa.Batch(regs, scheds, Ns, Ms, list(range(11, 11 + len(SHAPES))))
        assert b.launch_count() > 0
        first = b.run()
        second = b.run(seeds=list(range(21, 21 + len(SHAPES))))
        b.close()
        for k, r in enumerate(regs):
            for seed, outs in ((11 + k, first), (21 + k, second)):
                ind = r.run(scheds[k], Ns[k], Ms[k], seed)
                for key in ind:
                    assert np.array_equal(ind[key], outs[k][key]), (k, seed, key)
    finally:
        for r in regs:
            r.close()


def test_batch_rejects_a_changed_context(spa):
    regs = _regions(spa)[:2]
    scheds = [synth.geometric_schedule(4), synth.geometric_schedule(4)]
    try:
        b = spa.Batch(regs, scheds, [256, 256], [1, 1], [1, 2])
        b.run()
        regs[1].set_config(spa.make_config(move="rw", precision="fp32", ess_frac=0.5))
        with pytest.raises(spa.SpaError) as e:
            b.run()
        assert e.value.code == spa.SPA_EINVAL
        b.close()
    finally:
        for r in regs:
            r.close()


def test_batch_argument_errors(spa):
    regs = _regions(spa)[:1]
    s = synth.geometric_schedule(3)
    try:
        with pytest.raises(spa.SpaError):
            spa.Batch([regs[0], regs[0]], [s, s], [64, 64], [1, 1], [1, 2])
        bad = s.copy()
        bad[1] = -1.0
        with pytest.raises(spa.SpaError):
            spa.Batch(regs, [bad], [64], [1], [1])
    finally:
        for r in regs:
            r.close()


# Regions that share T, N, M and the move kind can run in lock step (SPA_BATCH_MODE=lockstep):
# every likelihood evaluation of all regions is one grouped launch per tile class (n-tile width,
# resident particle operand or not). Uneven n and p, p on both sides of the resident limit
# (K <= 256).
LOCKSTEP = [(300, 7, 1.0), (1200, 64, 2.0), (2000, 130, 4.0), (1000, 300, float("inf")), (700, 33, 16.0),
            (500, 260, 1.0)]


@pytest.mark.parametrize("move", ["rw", "mala"])
def test_lockstep_batch_matches_individual_runs(spa, move, monkeypatch):
    monkeypatch.setenv("SPA_BATCH_MODE", "lockstep")
    regs = []
    for k, (n, p, nu) in enumerate(LOCKSTEP):
        g = synth.make_region(n, p, 0.9, (0.4, -0.3), seed=800 + k)
        regs.append(spa.Region(g.G, g.y, nu, config=spa.make_config(move=move)))
    R = len(regs)
    sched = synth.geometric_schedule(5)
    N, M = 512, 2
    try:
        b = spa.Batch(regs, [sched] * R, [N] * R, [M] * R, list(range(31, 31 + R)))
        first = b.run()
        second = b.run(seeds=list(range(41, 41 + R)))
        n_lock = b.launch_count()
        b.close()
        monkeypatch.setenv("SPA_BATCH_MODE", "branches")
        bb = spa.Batch(regs, [sched] * R, [N] * R, [M] * R, list(range(31, 31 + R)))
        branch = bb.run()
        n_branch = bb.launch_count()
        bb.close()
        # one grouped launch per tile class replaces R likelihood launches per evaluation
        assert n_lock < n_branch
        for k, r in enumerate(regs):
            for seed, outs in ((31 + k, first), (41 + k, second)):
                ind = r.run(sched, N, M, seed)
                for key in ind:
                    assert np.array_equal(ind[key], outs[k][key]), (k, seed, key)
            for key in branch[k]:
                assert np.array_equal(branch[k][key], first[k][key]), (k, key)
    finally:
        for r in regs:
            r.close()
