"""FP64 CPU oracle for the SPA sweep (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. The CUDA library never does, and the
two share no code. ``spa_oracle.c`` restates the method of Lee, Caron, Doucet &
Holmes (arXiv:1106.0322) in plain double-precision loops. This module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spa_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction). Returns the .so path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrConfig(C.Structure):
    _fields_ = [
        ("move_kind", C.c_int32),
        ("init_mode", C.c_int32),
        ("burn_in_steps", C.c_int32),
        ("n_quantiles", C.c_int32),
        ("quantiles", C.c_double * 8),
        ("n_deltas", C.c_int32),
        ("deltas", C.c_double * 8),
        ("ess_frac", C.c_double),
        ("rw_scale", C.c_double),
        ("mala_h", C.c_double),
        ("sd_floor", C.c_double),
        ("site_sd", C.c_double),
        ("n_threads", C.c_int32),
    ]


class OrResult(C.Structure):
    _fields_ = [
        ("mean", C.POINTER(C.c_double)),
        ("quantile", C.POINTER(C.c_double)),
        ("conc", C.POINTER(C.c_double)),
        ("ess", C.POINTER(C.c_double)),
        ("log_z_inc", C.POINTER(C.c_double)),
        ("accept_rate", C.POINTER(C.c_double)),
        ("resampled", C.POINTER(C.c_uint8)),
        ("final_beta", C.POINTER(C.c_double)),
        ("final_logw", C.POINTER(C.c_double)),
        ("best", C.POINTER(C.c_double)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.POINTER
        lib.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        lib.or_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, P(C.c_double)]
        lib.or_standardise.argtypes = [P(C.c_int8), C.c_int64, C.c_int64, P(C.c_double), P(C.c_double)]
        lib.or_standardise.restype = C.c_int
        lib.or_loglik.argtypes = [P(C.c_int8), P(C.c_uint8), C.c_int64, C.c_int64, P(C.c_double),
                                  C.c_int64, P(C.c_double)]
        lib.or_loglik.restype = C.c_int
        lib.or_loglik_grad.argtypes = [P(C.c_int8), P(C.c_uint8), C.c_int64, C.c_int64, P(C.c_double),
                                       C.c_int64, P(C.c_double), P(C.c_double)]
        lib.or_loglik_grad.restype = C.c_int
        lib.or_prior_logpdf.argtypes = [C.c_double, C.c_double, P(C.c_double), C.c_int64, P(C.c_double)]
        lib.or_prior_draw.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_double, C.c_double]
        lib.or_prior_draw.restype = C.c_double
        lib.or_prior_sample.argtypes = [C.c_uint64, C.c_double, C.c_double, C.c_int64, C.c_int64, P(C.c_double)]
        lib.or_log_incr_weight.argtypes = [C.c_double, C.c_double, C.c_double, P(C.c_double), C.c_int64]
        lib.or_log_incr_weight.restype = C.c_double
        lib.or_lse_ess.argtypes = [P(C.c_double), C.c_int64, P(C.c_double), P(C.c_double)]
        lib.or_cumsum_blocked.argtypes = [P(C.c_double), C.c_int64, P(C.c_double)]
        lib.or_resample_systematic.argtypes = [P(C.c_double), C.c_int64, C.c_double, P(C.c_int32)]
        lib.or_resample_systematic.restype = C.c_int
        lib.or_weighted_quantile.argtypes = [P(C.c_double), P(C.c_double), C.c_int64, P(C.c_double),
                                             C.c_int, P(C.c_double)]
        lib.or_weighted_quantile.restype = C.c_int
        lib.or_run.argtypes = [P(C.c_int8), P(C.c_uint8), C.c_int64, C.c_int64, C.c_double, P(C.c_double),
                               C.c_int64, C.c_int64, C.c_int32, C.c_uint64, P(OrConfig), P(OrResult)]
        lib.or_run.restype = C.c_int
        lib.or_max_threads.restype = C.c_int
        lib.or_marginal.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double), C.c_int64, C.c_int64, C.c_int,
                                    P(C.c_double), P(C.c_double), P(C.c_double)]
        lib.or_marginal.restype = C.c_int
        lib.or_map.argtypes = [P(C.c_int8), P(C.c_uint8), C.c_int64, C.c_int64, C.c_double, C.c_double, P(C.c_double),
                               C.c_int32, C.c_double, P(C.c_double), P(C.c_double)]
        lib.or_map.restype = C.c_int
        lib.or_map_path.argtypes = [P(C.c_int8), P(C.c_uint8), C.c_int64, C.c_int64, C.c_double, P(C.c_double),
                                    C.c_int64, P(C.c_double), C.c_int32, C.c_double, P(C.c_double), P(C.c_double),
                                    P(C.c_uint8)]
        lib.or_map_path.restype = C.c_int
        _lib = lib
        return lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def normals(seed: int, particle: int, t: int, m: int, p: int) -> np.ndarray:
    out = np.zeros(p, np.float64)
    _load().or_normals(seed, particle, t, m, p, _p(out, C.c_double))
    return out


def standardise(G):
    G = np.ascontiguousarray(G, dtype=np.int8)
    n, p = G.shape
    m = np.zeros(p)
    s = np.zeros(p)
    rc = _load().or_standardise(_p(G, C.c_int8), n, p, _p(m, C.c_double), _p(s, C.c_double))
    if rc != 0:
        raise ValueError("monomorphic column")
    return m, s


def loglik(G, y, B) -> np.ndarray:
    G = np.ascontiguousarray(G, dtype=np.int8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.float64)
    n, p = G.shape
    N = B.shape[0]
    out = np.zeros(N)
    if _load().or_loglik(_p(G, C.c_int8), _p(y, C.c_uint8), n, p, _p(B, C.c_double), N,
                         _p(out, C.c_double)) != 0:
        raise ValueError("bad input")
    return out


def loglik_grad(G, y, B):
    G = np.ascontiguousarray(G, dtype=np.int8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    B = np.ascontiguousarray(B, dtype=np.float64)
    n, p = G.shape
    N = B.shape[0]
    ll = np.zeros(N)
    g = np.zeros((N, p))
    if _load().or_loglik_grad(_p(G, C.c_int8), _p(y, C.c_uint8), n, p, _p(B, C.c_double), N,
                              _p(ll, C.c_double), _p(g, C.c_double)) != 0:
        raise ValueError("bad input")
    return ll, g


def prior_logpdf(a: float, c: float, beta) -> np.ndarray:
    b = np.ascontiguousarray(beta, dtype=np.float64).ravel()
    out = np.zeros_like(b)
    _load().or_prior_logpdf(a, c, _p(b, C.c_double), b.size, _p(out, C.c_double))
    return out


def prior_sample(seed: int, a: float, c: float, N: int, p: int) -> np.ndarray:
    out = np.zeros((N, p))
    _load().or_prior_sample(C.c_uint64(seed), a, c, N, p, _p(out, C.c_double))
    return out


def log_incr_weight(a: float, c_prev: float, c_new: float, beta) -> float:
    b = np.ascontiguousarray(beta, dtype=np.float64).ravel()
    return float(_load().or_log_incr_weight(a, c_prev, c_new, _p(b, C.c_double), b.size))


def lse_ess(logw):
    lw = np.ascontiguousarray(logw, dtype=np.float64)
    lse = C.c_double()
    ess = C.c_double()
    _load().or_lse_ess(_p(lw, C.c_double), lw.size, C.byref(lse), C.byref(ess))
    return lse.value, ess.value


def cumsum_blocked(W) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros_like(W)
    _load().or_cumsum_blocked(_p(W, C.c_double), W.size, _p(out, C.c_double))
    return out


def resample_systematic(W, u: float) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    idx = np.zeros(W.size, np.int32)
    if _load().or_resample_systematic(_p(W, C.c_double), W.size, float(u), _p(idx, C.c_int32)) != 0:
        raise MemoryError
    return idx


def weighted_quantile(vals, W, qs) -> np.ndarray:
    v = np.ascontiguousarray(vals, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    q = np.ascontiguousarray(qs, dtype=np.float64)
    out = np.zeros(q.size)
    _load().or_weighted_quantile(_p(v, C.c_double), _p(W, C.c_double), v.size, _p(q, C.c_double),
                                 q.size, _p(out, C.c_double))
    return out


def max_threads() -> int:
    return int(_load().or_max_threads())


def map_em(G, y, a: float, c: float, beta0, max_em: int = 500, tol: float = 1e-10):
    """MAP by EM from beta0 (Section 2.1): returns (mode, log l + log p at the mode)."""
    G = np.ascontiguousarray(G, dtype=np.int8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    b0 = np.ascontiguousarray(beta0, dtype=np.float64)
    n, p = G.shape
    out = np.zeros(p)
    lp = C.c_double(0.0)
    if _load().or_map(_p(G, C.c_int8), _p(y, C.c_uint8), n, p, float(a), float(c), _p(b0, C.c_double), int(max_em),
                      float(tol), _p(out, C.c_double), C.byref(lp)) != 0:
        raise ValueError("or_map: bad input")
    return out, lp.value


def map_path(G, y, a: float, sched, best, max_em: int = 500, tol: float = 1e-10):
    """The MAP path of Section 4.1 walked in step order from the per-step best particles
    best [T, p]: (modes [T, p], log posteriors [T], chained [T] = 1 where EM from the
    previous step's MAP was kept)."""
    G = np.ascontiguousarray(G, dtype=np.int8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    sched = np.ascontiguousarray(sched, dtype=np.float64)
    best = np.ascontiguousarray(best, dtype=np.float64)
    n, p = G.shape
    T = sched.size
    if best.shape != (T, p):
        raise ValueError("best must be T x p")
    out = np.zeros((T, p))
    lp = np.zeros(T)
    ch = np.zeros(T, np.uint8)
    if _load().or_map_path(_p(G, C.c_int8), _p(y, C.c_uint8), n, p, float(a), _p(sched, C.c_double), T,
                           _p(best, C.c_double), int(max_em), float(tol), _p(out, C.c_double), _p(lp, C.c_double),
                           _p(ch, C.c_uint8)) != 0:
        raise ValueError("or_map_path: bad input")
    return out, lp, ch


def marginal(log_z_inc, mean, conc) -> dict:
    """Scale-marginalised summaries (Section 4, eq. all_particles) from a sweep's per-step
    outputs: log_z_inc [T], mean [T, p], conc [T, p, D]. Returns post_c [T] (the weights
    Z_t/Z_1 normalised), mean [p] and conc [p, D] of the mixture over scales."""
    lz = np.ascontiguousarray(log_z_inc, dtype=np.float64)
    m = np.ascontiguousarray(mean, dtype=np.float64)
    c = np.ascontiguousarray(conc, dtype=np.float64)
    T, p = m.shape
    D = c.shape[2] if c.ndim == 3 else 0
    post = np.zeros(T)
    mo = np.zeros(p)
    co = np.zeros((p, max(D, 1)))
    if _load().or_marginal(_p(lz, C.c_double), _p(m, C.c_double), _p(c, C.c_double), T, p, D, _p(post, C.c_double),
                           _p(mo, C.c_double), _p(co, C.c_double)) != 0:
        raise ValueError("or_marginal: bad sizes")
    return {"post_c": post, "mean": mo, "conc": co[:, :D]}


def make_config(move: str = "rw", init: str = "prior_is", burn_in_steps: int = 0,
                quantiles=(0.05, 0.5, 0.95), deltas=(0.05, 0.1), ess_frac: float = 0.75,
                rw_scale: float = 2.38, mala_h: float = 1.65, sd_floor: float = 1e-3,
                site_sd: float = 0.5, n_threads: int = 0) -> OrConfig:
    cfg = OrConfig()
    cfg.move_kind = {"rw": 0, "mala": 1, "site": 2}[move]
    cfg.init_mode = {"prior_is": 0, "mcmc": 1}[init]
    cfg.burn_in_steps = burn_in_steps
    cfg.n_quantiles = len(quantiles)
    for i, q in enumerate(quantiles):
        cfg.quantiles[i] = q
    cfg.n_deltas = len(deltas)
    for i, d in enumerate(deltas):
        cfg.deltas[i] = d
    cfg.ess_frac = ess_frac
    cfg.rw_scale = rw_scale
    cfg.mala_h = mala_h
    cfg.sd_floor = sd_floor
    cfg.site_sd = site_sd
    cfg.n_threads = n_threads
    return cfg


def run(G, y, a: float, sched, N: int, M: int, seed: int, cfg: OrConfig | None = None,
        keep_particles: bool = False, keep_best: bool = False) -> dict:
    """Run the SMC sweep of Section 4 and return the per-scale outputs as numpy arrays."""
    if cfg is None:
        cfg = make_config()
    G = np.ascontiguousarray(G, dtype=np.int8)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    sched = np.ascontiguousarray(sched, dtype=np.float64)
    n, p = G.shape
    T = sched.size
    nq, nd = cfg.n_quantiles, cfg.n_deltas
    out = {
        "mean": np.zeros((T, p)),
        "quantile": np.zeros((T, p, nq)),
        "conc": np.zeros((T, p, nd)),
        "ess": np.zeros(T),
        "log_z_inc": np.zeros(T),
        "accept_rate": np.zeros(T),
        "resampled": np.zeros(T, np.uint8),
    }
    res = OrResult()
    res.mean = _p(out["mean"], C.c_double)
    res.quantile = _p(out["quantile"], C.c_double)
    res.conc = _p(out["conc"], C.c_double)
    res.ess = _p(out["ess"], C.c_double)
    res.log_z_inc = _p(out["log_z_inc"], C.c_double)
    res.accept_rate = _p(out["accept_rate"], C.c_double)
    res.resampled = _p(out["resampled"], C.c_uint8)
    if keep_particles:
        out["final_beta"] = np.zeros((N, p))
        out["final_logw"] = np.zeros(N)
        res.final_beta = _p(out["final_beta"], C.c_double)
        res.final_logw = _p(out["final_logw"], C.c_double)
    if keep_best:
        out["best"] = np.zeros((T, p))
        res.best = _p(out["best"], C.c_double)
    rc = _load().or_run(_p(G, C.c_int8), _p(y, C.c_uint8), n, p, float(a), _p(sched, C.c_double), T, N, M,
                        C.c_uint64(seed), C.byref(cfg), C.byref(res))
    if rc != 0:
        raise ValueError("oracle run failed (bad input)")
    return out


INF = math.inf
