"""The synthetic inputs: the generator draws what the input recipe states.

Genotypes are sums of two haplotypes. Each haplotype thresholds an AR(1) latent Gaussian
chain along the markers at the minor-allele frequency, so each allele is Bernoulli(MAF),
the two alleles are independent (Hardy-Weinberg proportions), and linkage between markers
decays with distance. Phenotypes come from a logistic model on MAF-standardised
genotypes with case-control ascertainment, n // 2 cases. The schedules follow their
formulas, and the named workloads have the shapes their descriptions give.
"""
import math

import numpy as np
import pytest

from paper_1106_0322_gb300 import synth


def test_region_values_and_balance():
    reg = synth.make_region(301, 17, 0.9, (0.5, -0.4), seed=1)
    assert reg.G.shape == (301, 17) and reg.G.dtype == np.int8 and reg.G.flags["C_CONTIGUOUS"]
    assert set(np.unique(reg.G)) <= {0, 1, 2}
    assert reg.y.dtype == np.uint8 and set(np.unique(reg.y)) == {0, 1}
    assert int(reg.y.sum()) == 301 // 2
    assert np.all(reg.G.min(axis=0) < reg.G.max(axis=0))  # no monomorphic column
    assert np.all((reg.maf >= 0.05) & (reg.maf <= 0.5))
    assert reg.causal_idx.size == 2 and np.all(np.diff(reg.causal_idx) > 0)


def test_same_seed_same_region():
    a = synth.make_region(200, 12, 0.9, (0.5,), seed=7)
    b = synth.make_region(200, 12, 0.9, (0.5,), seed=7)
    c = synth.make_region(200, 12, 0.9, (0.5,), seed=8)
    assert np.array_equal(a.G, b.G) and np.array_equal(a.y, b.y) and np.array_equal(a.maf, b.maf)
    assert not np.array_equal(a.G, c.G)


def test_allele_frequencies_and_hardy_weinberg():
    """Without causal markers the labels carry no signal, so every column is a
    Binomial(2, MAF) draw: frequencies of 0, 1, 2 within 5 standard errors of
    (1-f)^2, 2f(1-f), f^2."""
    n = 30000
    reg = synth.make_region(n, 10, 0.9, (), seed=3)
    for j in range(reg.p):
        f = reg.maf[j]
        expect = np.array([(1 - f) ** 2, 2 * f * (1 - f), f * f])
        obs = np.bincount(reg.G[:, j], minlength=3) / n
        se = np.sqrt(expect * (1 - expect) / n)
        assert np.all(np.abs(obs - expect) < 5 * se + 1e-12), (j, obs, expect)


def test_linkage_decays_with_distance():
    reg = synth.make_region(8000, 40, 0.95, (), seed=4)
    C = np.corrcoef(reg.G.astype(np.float64), rowvar=False)
    near = np.mean([C[j, j + 1] for j in range(39)])
    mid = np.mean([C[j, j + 5] for j in range(35)])
    far = np.mean([C[j, j + 30] for j in range(10)])
    assert near > mid > far and near > 0.3 and abs(far) < 0.15


@pytest.mark.parametrize("beta", [1.0, -1.0])
def test_causal_marker_shifts_the_cases(beta):
    reg = synth.make_region(4000, 6, 0.5, (beta,), seed=5, causal_idx=[2])
    x = (reg.G[:, 2] - 2 * reg.maf[2]) / math.sqrt(2 * reg.maf[2] * (1 - reg.maf[2]))
    d = x[reg.y == 1].mean() - x[reg.y == 0].mean()
    assert np.sign(d) == np.sign(beta) and abs(d) > 0.3


def test_geometric_schedule():
    c = synth.geometric_schedule(9, -8.0, 0.0)
    assert np.allclose(np.log(c), np.linspace(-8.0, 0.0, 9), rtol=0, atol=1e-12)
    d = synth.geometric_schedule(9, -8.0, 0.0, sparse_to_diffuse=False)
    assert np.array_equal(d, c[::-1])
    assert synth.geometric_schedule(1, -3.0, 0.0).tolist() == [math.exp(-3.0)]


def test_paper_schedule():
    """b_t = b_1 0.98^(t-1), returned as c_t = b_t / a."""
    c = synth.paper_schedule(2.0, 450, 1.0)
    assert c[0] == 2.0 and np.allclose(c[1:] / c[:-1], 0.98, rtol=1e-14, atol=0)
    assert np.allclose(synth.paper_schedule(1.0, 250, 4.0) * 4.0, 0.98 ** np.arange(250), rtol=1e-14, atol=0)
    assert np.array_equal(synth.workload_schedule("paper-18q"), synth.paper_schedule(1.0, 250, 4.0))


def test_workload_shapes():
    w = synth.WORKLOADS
    assert (w["hit-region"]["n"], w["hit-region"]["p"], w["hit-region"]["N"], w["hit-region"]["T"],
            w["hit-region"]["M"], w["hit-region"]["move"]) == (2000, 200, 8192, 200, 10, "rw")
    assert (w["split-large"]["n"], w["split-large"]["p"], w["split-large"]["N"]) == (5000, 500, 16384)
    assert (w["mala"]["move"], w["mala"]["M"], w["mala"]["nu"]) == ("mala", 5, 2.0)
    assert (w["paper-18q"]["n"], w["paper-18q"]["p"], w["paper-18q"]["nu"], w["paper-18q"]["T"],
            w["paper-18q"]["M"], w["paper-18q"]["move"]) == (1859, 184, 4.0, 250, 5, "site")
    assert (w["paper-small"]["n"], w["paper-small"]["p"], w["paper-small"]["nu"], w["paper-small"]["T"]) == (
        500, 50, 1.0, 450)
    assert w["split-large"]["causal_beta"] == synth.PAPER_CAUSAL_BETA
    assert synth.workload_schedule("hit-region").size == 200


def test_batched_regions_ranges():
    regions = synth.batched_regions(R=4, seed=11)
    assert len(regions) == 4
    for reg, nu in regions:
        assert 1000 <= reg.n <= 5000 and reg.n % 2 == 0 and int(reg.y.sum()) == reg.n // 2
        assert 20 <= reg.p <= 500 and 0.8 <= reg.rho <= 0.97
        assert 1 <= reg.causal_idx.size <= 4 and nu in (1.0, 2.0, 4.0, 16.0)


def test_random_particles():
    B = synth.random_particles(1000, 30, 0.2, seed=2)
    assert B.shape == (1000, 30) and B.dtype == np.float32 and B.flags["C_CONTIGUOUS"]
    zeros = np.mean(B == 0.0)
    assert 0.03 < zeros < 0.07
    nz = np.abs(B[B != 0.0]).astype(np.float64)
    assert abs(nz.mean() - 0.2) < 0.01  # Laplace(0, b): E|x| = b
