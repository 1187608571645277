"""Launch-shape autotuner (msat_autotune): it times candidate shapes, the
tuned context steps bit for bit like the automatic one, and a second
instance of the same shape reuses the cached winner."""
import ctypes

import numpy as np
import pytest

from synth import uniform_ksat, zipf_weighted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_03640_gb300 as p
    from paper_2402_03640_gb300 import build
    build.build()
    p.load()
    return p


@pytest.mark.parametrize("maker,B", [("ksat", 64), ("zipf", 2)])
def test_tuned_shape_same_bits_and_cached(pkg, maker, B):
    cnf = uniform_ksat(3000, 12900, 3, seed=21) if maker == "ksat" else zipf_weighted(4000, 16000, seed=22)
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=1e-2, tune=True) as t, \
            pkg.Solver.from_cnf(cnf, restarts=B, lr=1e-2) as a:
        info = t.tuning
        assert len(info["timed"]) >= 3
        assert all(ms > 0 for *_, ms in info["timed"])
        best_ms = min(ms for *_, ms in info["timed"])
        assert (info["fwd_vw"], info["stage_vw"], info["light_rows"]) in \
            [(f, s, r) for f, s, r, ms in info["timed"] if ms == best_ms]
        t.step(25)
        a.step(25)
        assert np.array_equal(t.x().view(np.uint32), a.x().view(np.uint32))
        assert np.array_equal(t.best()[1], a.best()[1])
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=1e-2, tune=True) as again:
        assert again.tuning["timed"] == []  # served from the cache
        assert again.tuning["stage_vw"] == info["stage_vw"]


def test_autotune_rejects_malformed_instance(pkg):
    from paper_2402_03640_gb300 import native
    lib = native.load()
    cfg = native.msat_config()
    lib.msat_config_default(ctypes.byref(cfg))
    out = native.msat_config()
    off = np.array([0, 2], np.int64)
    lits = np.array([1, 5], np.int32)  # names variable 5 of 2
    rc = lib.msat_autotune(2, 1, ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(lits.ctypes.data),
                           None, ctypes.byref(cfg), None, 3, ctypes.byref(out), None, 0, None)
    assert rc == native.MSAT_EINVAL
