"""Python binding of the GB300 SPA library (include/spa.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels (libspa.so, built in-tree by ``_build.build()``). If the library is missing
or cannot be loaded, every call raises; there is no CPU fallback.

Names follow the C ABI: ``Region`` wraps a ``spa_ctx`` (``spa_create`` /
``spa_destroy``) with ``run``, ``loglik``, ``grad``; the context-free calls are
module functions. ``LogLik`` is a ``torch.autograd.Function`` whose backward is the
hand-written adjoint (``spa_grad_device``).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import _build

SPA_OK, SPA_EINVAL, SPA_ENOMEM, SPA_ECUDA, SPA_ETIMEOUT, SPA_ENUMERIC, SPA_EUNSUPPORTED = range(7)
MOVE_RW, MOVE_MALA, MOVE_SITE = 0, 1, 2
PREC_SPLIT_BF16, PREC_FP32 = 0, 1
INIT_PRIOR_IS, INIT_RESAMPLE_MOVE = 0, 1
_CODES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENUMERIC", 6: "EUNSUPPORTED"}


class SpaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"SPA_{_CODES.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [
        ("move_kind", C.c_int32),
        ("precision", C.c_int32),
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
        ("map_path", C.c_int32),
        ("stream", C.c_void_p),
    ]


class Result(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("mean", "quantile", "conc", "ess", "log_z_inc", "accept_rate", "resampled")]


class BatchArgs(C.Structure):
    _fields_ = [("schedules", C.c_void_p), ("T", C.c_void_p), ("N", C.c_void_p),
                ("moves_per_step", C.c_void_p), ("seeds", C.c_void_p)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "spa_config_default": (None, [C.POINTER(Config)]),
    "spa_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_void_p)]),
    "spa_set_data": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "spa_set_config": (C.c_int, [C.c_void_p, C.POINTER(Config)]),
    "spa_get_config": (C.c_int, [C.c_void_p, C.POINTER(Config)]),
    "spa_destroy": (None, [C.c_void_p]),
    "spa_last_error": (C.c_char_p, [C.c_void_p]),
    "spa_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_uint64, C.POINTER(Result)]),
    "spa_run_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_uint64,
                                 C.POINTER(Result)]),
    "spa_sync": (C.c_int, [C.c_void_p]),
    "spa_run_batch": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(BatchArgs), C.c_void_p]),
    "spa_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(BatchArgs), C.POINTER(C.c_void_p)]),
    "spa_batch_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "spa_batch_launch_count": (C.c_int64, [C.c_void_p]),
    "spa_batch_destroy": (None, [C.c_void_p]),
    "spa_last_launch_count": (C.c_int64, [C.c_void_p]),
    "spa_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint64]),
    "spa_loglik_tile_width": (C.c_int, [C.c_void_p]),
    "spa_loglik_tile_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "spa_set_tile_config": (C.c_int, [C.c_void_p, C.c_int32]),
    "spa_map": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_int32, C.c_double, C.c_void_p,
                          C.c_void_p]),
    "spa_map_path": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_void_p, C.c_void_p]),
    "spa_map_path_rounds": (C.c_int, [C.c_void_p]),
    "spa_map_path_given": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_void_p,
                                     C.c_void_p]),
    "spa_loglik_repeat": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "spa_grad_repeat": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "spa_loglik": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "spa_loglik_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "spa_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p]),
    "spa_grad_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "spa_resample_systematic": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p]),
    "spa_resample_systematic_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p]),
    "spa_prior_logpdf": (C.c_int, [C.c_double, C.c_double, C.c_void_p, C.c_int64, C.c_void_p]),
    "spa_incr_weight": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_void_p, C.c_int64, C.c_int64,
                                  C.c_void_p]),
    "spa_lse_ess": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "spa_marginal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_void_p]),
    "spa_marginal_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "spa_summaries": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p,
                                C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "spa_philox4x32_10": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "spa_normals": (C.c_int, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, C.c_void_p]),
    "spa_prior_sample": (C.c_int, [C.c_uint64, C.c_double, C.c_double, C.c_int64, C.c_int64, C.c_void_p]),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libspa.so (raises if it is missing and build_if_missing is False)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"the CUDA library {_build.LIB} is not built: run __graft_entry__.build()")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _check(rc: int, ctx=None):
    if rc != SPA_OK:
        msg = load().spa_last_error(ctx)
        raise SpaError(rc, msg.decode() if msg else "")


def default_config() -> Config:
    cfg = Config()
    load().spa_config_default(C.byref(cfg))
    return cfg


def make_config(move: str = "rw", precision: str = "split_bf16", init: str = "prior_is", burn_in_steps: int = 0,
                quantiles=(0.05, 0.5, 0.95), deltas=(0.05, 0.1), ess_frac: float = 0.75, rw_scale: float = 2.38,
                mala_h: float = 1.65, sd_floor: float = 1e-3, site_sd: float = 0.5, map_path: bool = False,
                stream: int = 0) -> Config:
    cfg = default_config()
    cfg.move_kind = {"rw": MOVE_RW, "mala": MOVE_MALA, "site": MOVE_SITE}[move]
    cfg.precision = {"split_bf16": PREC_SPLIT_BF16, "fp32": PREC_FP32}[precision]
    cfg.init_mode = {"prior_is": INIT_PRIOR_IS, "resample_move": INIT_RESAMPLE_MOVE, "mcmc": INIT_RESAMPLE_MOVE}[init]
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
    cfg.map_path = 1 if map_path else 0
    cfg.stream = stream or None
    return cfg


class Region:
    """One hit region on the device: ``spa_create(G, y, n, p, nu)``."""

    def __init__(self, G, y, nu: float, config: Config | None = None):
        lib = load()
        self.G = np.ascontiguousarray(G, dtype=np.int8)
        self.y = np.ascontiguousarray(y, dtype=np.uint8)
        self.n, self.p = self.G.shape
        if self.y.shape != (self.n,):
            raise ValueError("y must have n entries")
        h = C.c_void_p()
        _check(lib.spa_create(_ptr(self.G), _ptr(self.y), self.n, self.p, float(nu), C.byref(h)))
        self._h = h
        self.nu = float(nu)
        if config is not None:
            self.set_config(config)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().spa_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_config(self, cfg: Config):
        _check(load().spa_set_config(self._h, C.byref(cfg)), self._h)

    def config(self) -> Config:
        cfg = Config()
        _check(load().spa_get_config(self._h, C.byref(cfg)), self._h)
        return cfg

    def set_data(self, G, y):
        G = np.ascontiguousarray(G, dtype=np.int8)
        y = np.ascontiguousarray(y, dtype=np.uint8)
        if G.shape != (self.n, self.p) or y.shape != (self.n,):
            raise ValueError("shape mismatch")
        _check(load().spa_set_data(self._h, _ptr(G), _ptr(y)), self._h)

    def run(self, schedule, N: int, moves_per_step: int, seed: int) -> dict:
        """Run the SMC sweep (spa_run) and return the per-scale outputs."""
        sched = np.ascontiguousarray(schedule, dtype=np.float64)
        T = sched.size
        cfg = self.config()
        out = _alloc_result(T, self.p, cfg.n_quantiles, cfg.n_deltas)
        res = _result_struct(out)
        _check(load().spa_run(self._h, _ptr(sched), T, int(N), int(moves_per_step), C.c_uint64(seed), C.byref(res)),
               self._h)
        return out

    def run_device(self, schedule_dev, N: int, moves_per_step: int, seed: int, out_dev: dict | None = None):
        """Enqueue a sweep with device-resident schedule and outputs (torch tensors)."""
        res = _result_struct(out_dev) if out_dev else None
        _check(load().spa_run_device(self._h, _ptr(schedule_dev), schedule_dev.numel(), int(N), int(moves_per_step),
                                     C.c_uint64(seed), C.byref(res) if res else None), self._h)

    def sync(self):
        _check(load().spa_sync(self._h), self._h)

    def last_launch_count(self) -> int:
        return int(load().spa_last_launch_count(self._h))

    def set_wait_limit(self, limit_ns: int = 0):
        """Bound of the tensor-core kernels' device waits (spa_set_wait_limit; 0: 4 s)."""
        _check(load().spa_set_wait_limit(self._h, C.c_uint64(int(limit_ns))), self._h)

    def map(self, beta0, c: float, max_em: int = 200, tol: float = 1e-5):
        """MAP by EM (Section 2.1) from each row of beta0 [S, p] at scale c: (modes [S, p],
        log posteriors [S])."""
        b0 = np.ascontiguousarray(np.atleast_2d(beta0), dtype=np.float32)
        S = b0.shape[0]
        out = np.zeros_like(b0)
        lp = np.zeros(S)
        _check(load().spa_map(self._h, _ptr(b0), S, float(c), int(max_em), float(tol), _ptr(out), _ptr(lp)), self._h)
        return out, lp

    def map_path(self, T: int, max_em: int = 200, tol: float = 1e-5):
        """The MAP path (Section 4.1) of the last run (config map_path=True): (map [T, p],
        log posteriors [T])."""
        out = np.zeros((T, self.p), np.float32)
        lp = np.zeros(T)
        _check(load().spa_map_path(self._h, int(T), int(max_em), float(tol), _ptr(out), _ptr(lp)), self._h)
        return out, lp

    def map_path_given(self, schedule, best, max_em: int = 200, tol: float = 1e-5):
        """The MAP path rule (Section 4.1) from given per-step starts best [T, p]: (map [T, p],
        log posteriors [T])."""
        sched = np.ascontiguousarray(schedule, dtype=np.float64)
        b = np.ascontiguousarray(best, dtype=np.float32)
        T = sched.size
        if b.shape != (T, self.p):
            raise ValueError("best must be T x p")
        out = np.zeros((T, self.p), np.float32)
        lp = np.zeros(T)
        _check(load().spa_map_path_given(self._h, _ptr(sched), _ptr(b), T, int(max_em), float(tol), _ptr(out),
                                         _ptr(lp)), self._h)
        return out, lp

    def map_path_rounds(self) -> int:
        """Rounds after the first that the last map_path took to reach its fixed point."""
        return int(load().spa_map_path_rounds(self._h))

    def loglik_tile_width(self) -> int:
        """n-tile width of the tensor-core likelihood kernel (0 before the first run)."""
        return int(load().spa_loglik_tile_width(self._h))

    def tile_config(self):
        """(configuration 0..6 or -1 before the first run, source: 0 fixed, 1 table, 2 timed)."""
        src = C.c_int32(0)
        cfg = int(load().spa_loglik_tile_config(self._h, C.byref(src)))
        return cfg, int(src.value)

    def set_tile_config(self, cfg: int):
        """Fix the likelihood kernel's tile configuration (-1: the table and tuner decide)."""
        _check(load().spa_set_tile_config(self._h, int(cfg)), self._h)

    def loglik_repeat(self, N: int, reps: int, stream: int = 0):
        _check(load().spa_loglik_repeat(self._h, int(N), int(reps), stream or None), self._h)

    def grad_repeat(self, N: int, reps: int, stream: int = 0):
        _check(load().spa_grad_repeat(self._h, int(N), int(reps), stream or None), self._h)

    def loglik(self, B) -> np.ndarray:
        B = np.ascontiguousarray(B, dtype=np.float32)
        N = B.shape[0]
        if B.shape != (N, self.p):
            raise ValueError("B must be N x p")
        out = np.zeros(N, np.float64)
        _check(load().spa_loglik(self._h, _ptr(B), N, _ptr(out)), self._h)
        return out

    def loglik_device(self, B, out, stream: int = 0):
        _check(load().spa_loglik_device(self._h, _ptr(B), B.shape[0], _ptr(out), stream or None), self._h)

    def grad(self, B, c: float = 0.0):
        B = np.ascontiguousarray(B, dtype=np.float32)
        N = B.shape[0]
        ll = np.zeros(N, np.float64)
        g = np.zeros((N, self.p), np.float32)
        _check(load().spa_grad(self._h, _ptr(B), N, float(c), _ptr(ll), _ptr(g)), self._h)
        return ll, g

    def grad_device(self, B, c: float, ll_out, grad_out, stream: int = 0):
        _check(load().spa_grad_device(self._h, _ptr(B), B.shape[0], float(c), _ptr(ll_out), _ptr(grad_out),
                                      stream or None), self._h)


def _alloc_result(T, p, nq, nd) -> dict:
    return {
        "mean": np.zeros((T, p)),
        "quantile": np.zeros((T, p, nq)),
        "conc": np.zeros((T, p, nd)),
        "ess": np.zeros(T),
        "log_z_inc": np.zeros(T),
        "accept_rate": np.zeros(T),
        "resampled": np.zeros(T, np.uint8),
    }


def _result_struct(out: dict) -> Result:
    r = Result()
    for k in ("mean", "quantile", "conc", "ess", "log_z_inc", "accept_rate", "resampled"):
        setattr(r, k, _ptr(out[k]) if out.get(k) is not None else None)
    return r


def _batch_args(regions, schedules, N, moves_per_step, seeds):
    R = len(regions)
    handles = (C.c_void_p * R)(*[r.handle.value for r in regions])
    scheds = [np.ascontiguousarray(s, dtype=np.float64) for s in schedules]
    sp = (C.c_void_p * R)(*[s.ctypes.data for s in scheds])
    keep = dict(handles=handles, scheds=scheds, sp=sp, T=np.array([s.size for s in scheds], np.int64),
                N=np.array(N, np.int64), M=np.array(moves_per_step, np.int32), S=np.array(seeds, np.uint64))
    args = BatchArgs(C.cast(sp, C.c_void_p), _ptr(keep["T"]), _ptr(keep["N"]), _ptr(keep["M"]), _ptr(keep["S"]))
    return args, keep


def _batch_outputs(regions, T):
    outs = [_alloc_result(T[r], regions[r].p, regions[r].config().n_quantiles, regions[r].config().n_deltas)
            for r in range(len(regions))]
    structs = (Result * len(regions))(*[_result_struct(o) for o in outs])
    return outs, structs


def run_batch(regions, schedules, N, moves_per_step, seeds) -> list:
    """spa_run_batch over several Regions; returns one output dict per region."""
    args, keep = _batch_args(regions, schedules, N, moves_per_step, seeds)
    outs, structs = _batch_outputs(regions, keep["T"])
    _check(load().spa_run_batch(keep["handles"], len(regions), C.byref(args), C.cast(structs, C.c_void_p)))
    return outs


class Batch:
    """spa_batch: the sweeps of several Regions captured into one CUDA graph (one branch
    per region, run concurrently), launched once per run()."""

    def __init__(self, regions, schedules, N, moves_per_step, seeds):
        self.regions = list(regions)
        args, keep = _batch_args(self.regions, schedules, N, moves_per_step, seeds)
        self._T = keep["T"]
        h = C.c_void_p()
        _check(load().spa_batch_create(keep["handles"], len(self.regions), C.byref(args), C.byref(h)))
        self.handle = h

    def run(self, seeds=None) -> list:
        outs, structs = _batch_outputs(self.regions, self._T)
        sp = None
        if seeds is not None:
            sarr = np.ascontiguousarray(seeds, dtype=np.uint64)
            assert sarr.size == len(self.regions)
            sp = _ptr(sarr)
        _check(load().spa_batch_run(self.handle, sp, C.cast(structs, C.c_void_p)))
        return outs

    def launch_count(self) -> int:
        return int(load().spa_batch_launch_count(self.handle))

    def close(self):
        if self.handle:
            load().spa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ context-free calls
def marginal(result: dict) -> dict:
    """spa_marginal on one sweep's outputs (a dict from Region.run): the posterior over the
    schedule's scales, post_c [T], and the scale-marginalised mean [p] and conc [p, D]."""
    lz = np.ascontiguousarray(result["log_z_inc"], dtype=np.float64)
    m = np.ascontiguousarray(result["mean"], dtype=np.float64)
    c = np.ascontiguousarray(result["conc"], dtype=np.float64)
    T, p = m.shape
    D = c.shape[2] if c.ndim == 3 else 0
    post = np.zeros(T)
    mo = np.zeros(p)
    co = np.zeros((p, max(D, 1)))
    _check(load().spa_marginal(_ptr(lz), _ptr(m), _ptr(c) if D else None, T, p, D, _ptr(post), _ptr(mo),
                               _ptr(co) if D else None))
    return {"post_c": post, "mean": mo, "conc": co[:, :D]}


def resample_systematic(W, u: float) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    idx = np.zeros(W.size, np.int32)
    _check(load().spa_resample_systematic(_ptr(W), W.size, float(u), _ptr(idx)))
    return idx


NOALLOC_RESAMPLE_MAX_N = 262144


def check_noalloc_buffers(W_dev, idx_dev):
    """Reject buffers the allocation-free resampling cannot take as they are: the kernel reads
    N contiguous doubles at W_dev's address and writes N int32 at idx_dev's, so anything else
    (another dtype, a strided view, host memory, two devices, a short index buffer) would give
    wrong ancestors or write past the caller's buffer. Raises ValueError."""
    import torch

    if W_dev.dtype != torch.float64:
        raise ValueError(f"W_dev must be float64, got {W_dev.dtype}")
    if idx_dev.dtype != torch.int32:
        raise ValueError(f"idx_dev must be int32, got {idx_dev.dtype}")
    if not (W_dev.is_cuda and idx_dev.is_cuda):
        raise ValueError("W_dev and idx_dev must be CUDA tensors")
    if W_dev.device != idx_dev.device:
        raise ValueError(f"W_dev and idx_dev are on different devices ({W_dev.device}, {idx_dev.device})")
    if W_dev.device.index is not None and W_dev.device.index != torch.cuda.current_device():
        raise ValueError(f"the buffers are on {W_dev.device}, the current device is {torch.cuda.current_device()}")
    if not (W_dev.is_contiguous() and idx_dev.is_contiguous()):
        raise ValueError("W_dev and idx_dev must be contiguous")
    if idx_dev.numel() != W_dev.numel():
        raise ValueError(f"idx_dev has {idx_dev.numel()} entries, W_dev {W_dev.numel()}: they must match")


def resample_systematic_noalloc(W_dev, u: float, idx_dev, stream: int = 0):
    """Allocation-free systematic resampling on device buffers (torch tensors): W_dev float64,
    idx_dev int32, both contiguous, on the current device and of the same length
    N <= NOALLOC_RESAMPLE_MAX_N. Enqueued on `stream`, which must be ordered after whatever
    wrote W_dev (the call does not synchronise)."""
    check_noalloc_buffers(W_dev, idx_dev)
    _check(load().spa_resample_systematic_noalloc(_ptr(W_dev), W_dev.numel(), float(u), _ptr(idx_dev),
                                                  stream or None))


def prior_logpdf(nu: float, c: float, beta) -> np.ndarray:
    b = np.ascontiguousarray(beta, dtype=np.float32).ravel()
    out = np.zeros(b.size, np.float64)
    _check(load().spa_prior_logpdf(float(nu), float(c), _ptr(b), b.size, _ptr(out)))
    return out


def incr_weight(nu: float, c_prev: float, c_new: float, B) -> np.ndarray:
    B = np.ascontiguousarray(B, dtype=np.float32)
    out = np.zeros(B.shape[0], np.float64)
    _check(load().spa_incr_weight(float(nu), float(c_prev), float(c_new), _ptr(B), B.shape[0], B.shape[1], _ptr(out)))
    return out


def lse_ess(logw):
    lw = np.ascontiguousarray(logw, dtype=np.float64)
    lse, ess = C.c_double(), C.c_double()
    _check(load().spa_lse_ess(_ptr(lw), lw.size, C.byref(lse), C.byref(ess)))
    return lse.value, ess.value


def summaries(B, W, quantiles=(0.05, 0.5, 0.95), deltas=(0.05, 0.1)):
    B = np.ascontiguousarray(B, dtype=np.float32)
    W = np.ascontiguousarray(W, dtype=np.float64)
    N, p = B.shape
    q = np.ascontiguousarray(quantiles, dtype=np.float64)
    d = np.ascontiguousarray(deltas, dtype=np.float64)
    mean = np.zeros(p)
    quant = np.zeros((p, q.size))
    conc = np.zeros((p, d.size))
    _check(load().spa_summaries(_ptr(B), _ptr(W), N, p, _ptr(q), q.size, _ptr(d), d.size, _ptr(mean), _ptr(quant),
                                _ptr(conc)))
    return mean, quant, conc


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _check(load().spa_philox4x32_10(_ptr(c), _ptr(k), c.shape[0], _ptr(out)))
    return out


def normals(seed: int, particle: int, t: int, m: int, p: int) -> np.ndarray:
    out = np.zeros(p, np.float32)
    _check(load().spa_normals(C.c_uint64(seed), particle, t, m, p, _ptr(out)))
    return out


def prior_sample(seed: int, nu: float, c: float, N: int, p: int) -> np.ndarray:
    out = np.zeros((N, p), np.float32)
    _check(load().spa_prior_sample(C.c_uint64(seed), float(nu), float(c), N, p, _ptr(out)))
    return out


# ---------------------------------------------------------- autograd wrapper
def _torch_loglik_function():
    import torch

    class LogLik(torch.autograd.Function):
        """l(B) for a CUDA (N, p) float32 tensor of particles; backward applies the adjoint
        kernel grad l = X^T (y - logit^{-1}(X beta)) (spa_grad_device)."""

        @staticmethod
        def forward(ctx, B, region: Region):
            B = B.detach().contiguous()
            out = torch.empty(B.shape[0], dtype=torch.float64, device=B.device)
            region.loglik_device(B, out, torch.cuda.current_stream().cuda_stream)
            ctx.save_for_backward(B)
            ctx.region = region
            return out

        @staticmethod
        def backward(ctx, g_out):
            (B,) = ctx.saved_tensors
            g = torch.empty_like(B)
            ll = torch.empty(B.shape[0], dtype=torch.float64, device=B.device)
            ctx.region.grad_device(B, 0.0, ll, g, torch.cuda.current_stream().cuda_stream)
            return g * g_out.to(g.dtype)[:, None], None

    return LogLik


def loglik_autograd(B, region: Region):
    """Differentiable log-likelihood of CUDA particles B (torch) in `region`."""
    return _torch_loglik_function().apply(B, region)


INF = math.inf
