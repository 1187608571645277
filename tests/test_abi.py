"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument checks reject malformed input without touching a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mt in re.finditer(r"\b(msat_[a-z0-9_]+)\s*\(", text):
            names.add(mt.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2402_03640_gb300 import build, native
    build.build()
    return native.load()


def test_header_declares_the_entry_points():
    names = _declared_symbols()
    for must in ("msat_create", "msat_step", "msat_evaluate", "msat_best", "msat_destroy",
                 "msat_forward", "msat_backward", "msat_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    so = lib._name
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(msat_[a-z0-9_]+)$", out, flags=re.M))
    missing = [s for s in _declared_symbols() if s not in exported]
    assert not missing, missing
    for s in _declared_symbols():
        assert hasattr(lib, s)


def test_config_default(lib):
    from paper_2402_03640_gb300 import native
    cfg = native.msat_config()
    assert lib.msat_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.lr, cfg.beta1, cfg.beta2, cfg.eps, cfg.restarts, cfg.seed_x) == \
        (1e-4, 0.9, 0.999, 1e-8, 1, 1)


def _create(lib, n, off, lits, w=None, restarts=1, **shape):
    from paper_2402_03640_gb300 import native
    cfg = native.msat_config()
    lib.msat_config_default(ctypes.byref(cfg))
    cfg.restarts = restarts
    for k, v in shape.items():
        setattr(cfg, k, v)
    ctx = ctypes.c_void_p()
    off = np.ascontiguousarray(off, np.int64)
    lits = np.ascontiguousarray(lits, np.int32)
    wp = None if w is None else ctypes.c_void_p(np.ascontiguousarray(w, np.int64).ctypes.data)
    rc = lib.msat_create(ctypes.byref(ctx), n, off.shape[0] - 1, ctypes.c_void_p(off.ctypes.data),
                         ctypes.c_void_p(lits.ctypes.data), wp, ctypes.byref(cfg), None)
    return rc, lib.msat_last_error().decode()


@pytest.mark.parametrize("case,needle", [
    (dict(n=2, off=[0, 2], lits=[1, 3]), "names no variable"),
    (dict(n=2, off=[0, 2], lits=[1, 0]), "is 0"),
    (dict(n=2, off=[0, 2, 1], lits=[1, 2]), "non-decreasing"),
    (dict(n=2, off=[1, 2], lits=[1, 2]), "clause_off[0]"),
    (dict(n=2, off=[0, 2], lits=[1, 2], w=[0]), "weight"),
    (dict(n=2, off=[0, 2], lits=[1, 2], restarts=3), "power of two"),
    (dict(n=0, off=[0], lits=[1]), "n_vars"),
    (dict(n=40000, off=[0, 32768], lits=list(range(1, 32769))), "limit 32767"),
    (dict(n=2, off=[0, 2], lits=[1, 2], restarts=1024, fwd_vw=2), "must not exceed 256"),
    (dict(n=2, off=[0, 2], lits=[1, 2], restarts=512, stage_vw=1), "must not exceed 256"),
    (dict(n=2, off=[0, 2], lits=[1, 2], restarts=4, fwd_vw=8), "powers of two"),
    (dict(n=2, off=[0, 2], lits=[1, 2], loss_norm=7), "unknown loss_norm"),
    (dict(n=2, off=[0, 2], lits=[1, 2], row_order=3), "unknown row_order"),
    (dict(n=2, off=[0, 2], lits=[1, 2], row_order=-1), "unknown row_order"),
])
def test_create_rejects_malformed_input(lib, case, needle):
    from paper_2402_03640_gb300 import native
    rc, msg = _create(lib, **case)
    assert rc == native.MSAT_EINVAL
    assert needle in msg


def test_null_arguments(lib):
    from paper_2402_03640_gb300 import native
    assert lib.msat_step(None, 1, None, None) == native.MSAT_EINVAL
    assert lib.msat_evaluate(None, None, 1, None, 0) == native.MSAT_EINVAL
    assert lib.msat_best(None, None, None) == native.MSAT_EINVAL
    assert lib.msat_solve(None, 1, 1.0, 1, None, None, None, None, 0, None) == native.MSAT_EINVAL
    assert lib.msat_step_ex(None, 1, 0, None, None) == native.MSAT_EINVAL
    assert lib.msat_heuristic_gap(None, None, None) == native.MSAT_EINVAL
    assert lib.msat_selftest_bounded_wait(-1) == native.MSAT_EINVAL
    assert lib.msat_selftest_bounded_wait((1 << 24) + 1) == native.MSAT_EINVAL
    out = ctypes.c_double(0.0)
    assert lib.msat_dense_mma_rate(256, 16, None) == native.MSAT_EINVAL
    for n_assign, iters in ((0, 16), (24, 16), (272, 16), (256, 0), (256, (1 << 20) + 1)):
        assert lib.msat_dense_mma_rate(n_assign, iters, ctypes.byref(out)) == native.MSAT_EINVAL
    assert lib.msat_best_step(None, None) == native.MSAT_EINVAL
    assert lib.msat_autotune(1, 0, None, None, None, None, None, 1, None, None, 0, None) == native.MSAT_EINVAL
    lib.msat_destroy(None)


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2402_03640_gb300 import build, native
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(build, "SO_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        native.load()
