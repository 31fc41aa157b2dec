"""Host-side checks of the C-ABI library that need no GPU: it builds, loads and exports
every entry point include/spa.h declares, and the ctypes structs match the header."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spa.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spa_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1106_0322_gb300 import _build

    _build.build()
    import paper_1106_0322_gb300 as spa

    return spa.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("spa_create", "spa_set_config", "spa_run", "spa_run_batch", "spa_destroy", "spa_last_error",
                     "spa_loglik", "spa_grad", "spa_resample_systematic", "spa_prior_logpdf"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1106_0322_gb300 as spa

    names = _declared()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(spa.EXPORTED)
    out = subprocess.run(["nm", "-D", "--defined-only", spa.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (spa_[a-z0-9_]+)$", out, flags=re.M))
    assert set(names) <= exported


def test_library_is_built_for_sm103a_only(lib):
    import paper_1106_0322_gb300 as spa

    out = subprocess.run(["cuobjdump", "--list-elf", spa.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout
    assert "sm_90" not in out.stdout and "sm_100." not in out.stdout


def test_struct_layouts_match_header():
    import ctypes as C

    import paper_1106_0322_gb300 as spa

    # int32 x5, double[8], int32, double[8], 4 doubles, pointer (LP64, natural alignment)
    assert C.sizeof(spa.Config) == 20 + 4 + 64 + 4 + 4 + 64 + 40 + 4 + 4 + 8
    assert C.sizeof(spa.Result) == 7 * 8
    assert C.sizeof(spa.BatchArgs) == 5 * 8


def test_default_config(lib):
    import paper_1106_0322_gb300 as spa

    cfg = spa.default_config()
    assert cfg.move_kind == spa.MOVE_RW and cfg.precision == spa.PREC_SPLIT_BF16
    assert cfg.n_quantiles == 3 and list(cfg.quantiles[:3]) == [0.05, 0.5, 0.95]
    assert cfg.n_deltas == 2 and list(cfg.deltas[:2]) == [0.05, 0.1]
    assert cfg.ess_frac == 0.75 and cfg.rw_scale == 2.38 and cfg.mala_h == 1.65


def test_null_arguments_are_rejected_without_a_gpu(lib):
    import ctypes as C

    import paper_1106_0322_gb300 as spa

    h = C.c_void_p()
    assert lib.spa_create(None, None, 10, 2, 1.0, C.byref(h)) == spa.SPA_EINVAL
    assert b"NULL" in lib.spa_last_error(None)
    assert lib.spa_run(None, None, 1, 1, 1, 0, None) == spa.SPA_EINVAL
    assert lib.spa_last_launch_count(None) == 0
    lib.spa_destroy(None)


def test_product_path_has_no_oracle_dependency():
    # the CUDA library and its binding never import or load the oracle
    pkg = os.path.join(ROOT, "paper_1106_0322_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "spa_oracle" not in text, f


class _FakeTensor:
    """Just the attributes the allocation-free resampling's argument checks read."""

    def __init__(self, dtype, is_cuda=True, device="cuda:0", contiguous=True, numel=16):
        import torch

        self.dtype = dtype
        self.is_cuda = is_cuda
        self.device = torch.device(device)
        self._contiguous = contiguous
        self._numel = numel

    def is_contiguous(self):
        return self._contiguous

    def numel(self):
        return self._numel


def test_noalloc_resampling_rejects_unusable_buffers(monkeypatch):
    import torch

    import paper_1106_0322_gb300 as spa

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    f64, i32 = torch.float64, torch.int32
    good_W, good_idx = _FakeTensor(f64), _FakeTensor(i32)
    spa.check_noalloc_buffers(good_W, good_idx)  # accepted
    cases = [
        (_FakeTensor(torch.float32), good_idx, "float64"),
        (good_W, _FakeTensor(torch.int64), "int32"),
        (torch.zeros(16, dtype=f64), torch.zeros(16, dtype=i32), "CUDA"),
        (good_W, _FakeTensor(i32, device="cuda:1"), "different devices"),
        (_FakeTensor(f64, device="cuda:1"), _FakeTensor(i32, device="cuda:1"), "current device"),
        (_FakeTensor(f64, contiguous=False), good_idx, "contiguous"),
        (good_W, _FakeTensor(i32, contiguous=False), "contiguous"),
        (good_W, _FakeTensor(i32, numel=15), "must match"),
        (good_W, _FakeTensor(i32, numel=17), "must match"),
    ]
    for W, idx, what in cases:
        with pytest.raises(ValueError, match=what):
            spa.check_noalloc_buffers(W, idx)
        # the public call rejects them before it reaches the library
        with pytest.raises(ValueError, match=what):
            spa.resample_systematic_noalloc(W, 0.5, idx)


def test_committed_tile_table_is_well_formed():
    """The likelihood kernel's tile table (written on a GB300 by paper_1106_0322_gb300/tune_tiles.py)
    lists, per shape, a configuration valid for that shape's kernel mode (configurations 3-6
    only with the particle operand resident: p + 1 <= 256; 6 only with a last k-block at
    most 32 columns wide) and the times it chose from."""
    import json

    path = os.path.join(ROOT, "paper_1106_0322_gb300", "tuning", "loglik_tiles.json")
    doc = json.load(open(path))
    assert doc["generated_by"] == "paper_1106_0322_gb300/tune_tiles.py"
    assert len(doc["entries"]) > 0
    for e in doc["entries"]:
        assert e["n"] > 0 and e["p"] > 0 and e["N_pad"] % 128 == 0
        assert 0 <= e["config"] <= 6
        assert e["config"] < 3 or e["p"] + 1 <= 256
        ksteps = (e["p"] + 1 + 15) // 16
        assert e["config"] != 6 or ksteps <= 12 or ksteps % 4 in (1, 2)
        us = {int(k): v for k, v in e["us"].items()}
        assert e["config"] == min(us, key=us.get)
