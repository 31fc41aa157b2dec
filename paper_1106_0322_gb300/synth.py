"""Seeded synthetic hit regions: genotypes G in {0,1,2} and case-control phenotypes y.

The paper analyses real genotypes (Section 3: 1859 subjects x 184 SNPs from a
colorectal-cancer hit region on chromosome 18q) that are not distributed with it.
This module generates stand-ins with the same structure:

* markers in linkage disequilibrium: each haplotype is an AR(1) latent Gaussian
  chain along the markers, z_j = rho z_{j-1} + sqrt(1 - rho^2) e_j, and the allele
  at marker j is 1{z_j > Phi^{-1}(1 - MAF_j)}, MAF_j ~ U(0.05, 0.5); a genotype is
  the sum of two haplotypes, so it is Binomial(2, MAF_j) at each marker;
* pseudo-phenotypes as in Section 3: a few causal markers with non-zero
  coefficients on population-standardised genotypes, y ~ Bernoulli(logit^{-1}(eta)),
  eta = intercept + sum_k beta_k x_k, followed by case-control ascertainment
  (individuals are drawn until n/2 cases and n/2 controls are filled).

Nothing here evaluates the SPA method: it only draws inputs. Both the FP64 oracle
and the CUDA library consume its outputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import ndtri

# Causal effect sizes printed for the n=500 / p=50 data set (Section 5).
PAPER_CAUSAL_BETA = (-0.2538, 0.4578, -0.1873, -0.1498, 0.0996)


@dataclasses.dataclass
class Region:
    G: np.ndarray          # (n, p) int8, values 0/1/2, row-major
    y: np.ndarray          # (n,) uint8, 0/1
    maf: np.ndarray        # (p,) minor-allele frequencies used to draw G
    causal_idx: np.ndarray  # indices of non-zero coefficients
    causal_beta: np.ndarray
    rho: float
    seed: int

    @property
    def n(self) -> int:
        return int(self.G.shape[0])

    @property
    def p(self) -> int:
        return int(self.G.shape[1])


def _haplotypes(rng: np.random.Generator, count: int, rho: float, thr: np.ndarray) -> np.ndarray:
    """`count` haplotypes (count, p) of 0/1 alleles from AR(1) latent Gaussians."""
    p = thr.shape[0]
    z = rng.standard_normal(count)
    out = np.empty((count, p), dtype=np.int8)
    out[:, 0] = z > thr[0]
    innov = math.sqrt(max(0.0, 1.0 - rho * rho))
    for j in range(1, p):
        z = rho * z + innov * rng.standard_normal(count)
        out[:, j] = z > thr[j]
    return out


def make_region(n: int, p: int, rho: float, causal_beta, seed: int,
                causal_idx=None, intercept: float = -0.2,
                maf_range=(0.05, 0.5)) -> Region:
    """Draw one region with n individuals (n // 2 cases, n - n // 2 controls) and p markers.

    `causal_beta` are the non-zero coefficients on MAF-standardised genotypes;
    their marker indices are drawn without replacement unless `causal_idx` is given.
    Columns that come out monomorphic (possible only for tiny n) are redrawn.
    """
    if n < 2 or p < 1:
        raise ValueError("need n >= 2 and p >= 1")
    rng = np.random.default_rng(seed)
    maf = rng.uniform(maf_range[0], maf_range[1], size=p)
    thr = ndtri(1.0 - maf)
    causal_beta = np.asarray(causal_beta, dtype=np.float64)
    if causal_idx is None:
        k = min(len(causal_beta), p)
        causal_idx = np.sort(rng.choice(p, size=k, replace=False))
        causal_beta = causal_beta[:k]
    causal_idx = np.asarray(causal_idx, dtype=np.int64)
    sd_pop = np.sqrt(2.0 * maf * (1.0 - maf))

    want_case = n // 2
    want_ctrl = n - want_case
    cases, ctrls = [], []
    have_case = have_ctrl = 0
    while have_case < want_case or have_ctrl < want_ctrl:
        batch = max(256, 2 * n)
        g = _haplotypes(rng, batch, rho, thr) + _haplotypes(rng, batch, rho, thr)
        if causal_idx.size:
            xs = (g[:, causal_idx] - 2.0 * maf[causal_idx]) / sd_pop[causal_idx]
            eta = intercept + xs @ causal_beta
        else:
            eta = np.full(batch, intercept)
        prob = 1.0 / (1.0 + np.exp(-eta))
        is_case = rng.random(batch) < prob
        take_c = g[is_case][: want_case - have_case]
        take_k = g[~is_case][: want_ctrl - have_ctrl]
        cases.append(take_c)
        ctrls.append(take_k)
        have_case += take_c.shape[0]
        have_ctrl += take_k.shape[0]
    G = np.concatenate(cases + ctrls, axis=0).astype(np.int8)
    y = np.concatenate([np.ones(want_case, np.uint8), np.zeros(want_ctrl, np.uint8)])
    # Shuffle individuals so cases and controls are interleaved.
    perm = rng.permutation(n)
    G, y = np.ascontiguousarray(G[perm]), np.ascontiguousarray(y[perm])
    # Redraw any monomorphic column (sd = 0 is not standardisable).
    for j in range(p):
        tries = 0
        while G[:, j].min() == G[:, j].max():
            col = (rng.random((n, 2)) < maf[j]).sum(axis=1)
            G[:, j] = col.astype(np.int8)
            tries += 1
            if tries > 1000:
                raise RuntimeError("could not draw a polymorphic column")
    return Region(G=G, y=y, maf=maf, causal_idx=causal_idx, causal_beta=causal_beta,
                  rho=rho, seed=seed)


def geometric_schedule(T: int, log_c_lo: float = -8.0, log_c_hi: float = 0.0,
                       sparse_to_diffuse: bool = True) -> np.ndarray:
    """T prior scales c_t, geometric in c over log c in [log_c_lo, log_c_hi].

    The SPA plots of Section 5.1 span log c in (-8, 0).
    """
    if T < 1:
        raise ValueError("T >= 1")
    if T == 1:
        grid = np.array([log_c_lo])
    else:
        grid = np.linspace(log_c_lo, log_c_hi, T)
    c = np.exp(grid)
    return c if sparse_to_diffuse else c[::-1].copy()


def paper_schedule(b1: float, T: int, a: float, ratio: float = 0.98) -> np.ndarray:
    """The paper's scale sequence b_t = b_1 * ratio^(t-1) (Section 4.1), returned as c_t = b_t / a."""
    t = np.arange(T, dtype=np.float64)
    return (b1 * ratio ** t) / a


# Workloads shaped like the paper's hit regions (n individuals, p markers,
# LD rho, causal effects, Gt degrees of freedom nu = a, N particles, T scale
# steps, M moves per step, move kind).
WORKLOADS = {
    "plain-small": dict(n=200, p=10, rho=0.9, causal_beta=(0.5, 0.5), nu=1.0,
                        N=1024, T=50, M=5, move="rw", seed=1000),
    "hit-region": dict(n=2000, p=200, rho=0.95, causal_beta=(0.3, 0.5, -0.4), nu=1.0,
                       N=8192, T=200, M=10, move="rw", seed=1001),
    "split-large": dict(n=5000, p=500, rho=0.95, causal_beta=PAPER_CAUSAL_BETA, nu=1.0,
                        N=16384, T=200, M=10, move="rw", seed=1002),
    "mala": dict(n=2000, p=200, rho=0.95, causal_beta=(0.3, 0.5, -0.4), nu=2.0,
                 N=8192, T=200, M=5, move="mala", seed=1003),
    # The paper's own settings (Section 4.1, "Further details"): its single-coordinate
    # cycle (M = 5 cycles per step), its schedules b_t = b_1 0.98^(t-1) run from diffuse to
    # sparse, started by MCMC at the first scale (resample-move burn-in), on synthetic data
    # of its two data sets' shapes (n = 500 / p = 50 with a = 1 and T = 450; the 18q region,
    # n = 1859 / p = 184, with a = 4, b_1 = 1 and T = 250).
    "paper-small": dict(n=500, p=50, rho=0.95, causal_beta=PAPER_CAUSAL_BETA, nu=1.0,
                        N=8192, T=450, M=5, move="site", seed=1005, schedule=("paper", 2.0), burn_in=10),
    "paper-18q": dict(n=1859, p=184, rho=0.95, causal_beta=PAPER_CAUSAL_BETA, nu=4.0,
                      N=8192, T=250, M=5, move="site", seed=1006, schedule=("paper", 1.0), burn_in=10),
}


def workload_region(name: str) -> Region:
    w = WORKLOADS[name]
    return make_region(w["n"], w["p"], w["rho"], w["causal_beta"], w["seed"])


def workload_schedule(name: str) -> np.ndarray:
    """The workload's scale schedule c_t: geometric over log c in [-8, 0], sparse to
    diffuse, or the paper's b_t = b_1 0.98^(t-1) (as c_t = b_t / a) when it names one."""
    w = WORKLOADS[name]
    sch = w.get("schedule")
    if sch and sch[0] == "paper":
        return paper_schedule(sch[1], w["T"], w["nu"])
    return geometric_schedule(w["T"])


def batched_regions(R: int = 64, seed: int = 1004):
    """R uneven regions: n ~ U[1000, 5000] (balanced), p ~ U[20, 500], rho ~ U[0.8, 0.97],
    1-4 causal markers with beta ~ N(0, 0.2) (variance 0.2, Section 3), nu in {1, 2, 4, 16}."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(R):
        n = int(rng.integers(500, 2501)) * 2
        p = int(rng.integers(20, 501))
        rho = float(rng.uniform(0.8, 0.97))
        k = int(rng.integers(1, 5))
        beta = rng.normal(0.0, math.sqrt(0.2), size=k)
        nu = float(rng.choice([1.0, 2.0, 4.0, 16.0]))
        reg = make_region(n, p, rho, beta, seed=5000 + r)
        out.append((reg, nu))
    return out


def random_particles(N: int, p: int, scale: float, seed: int, dtype=np.float32) -> np.ndarray:
    """(N, p) particle matrix with Laplace-distributed entries of the given scale
    and some exact zeros; used as loglik/gradient test inputs."""
    rng = np.random.default_rng(seed)
    B = rng.laplace(0.0, scale, size=(N, p))
    B[rng.random((N, p)) < 0.05] = 0.0
    return np.ascontiguousarray(B.astype(dtype))
