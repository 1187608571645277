"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes gives up, reports MSAT_ETIMEOUT through the host, and the
device keeps working (the same path every wait of the tensor-core evaluator
takes)."""
import numpy as np
import pytest

from synth import uniform_ksat

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


def test_bounded_wait_times_out_and_device_stays_usable(pkg, oracle):
    from paper_2402_03640_gb300 import native
    lib = native.load()
    for spins in (1, 1000):
        rc = lib.msat_selftest_bounded_wait(spins)
        assert rc == native.MSAT_ETIMEOUT
        assert b"gave up" in lib.msat_last_error()
    # spins = 0: the kernels' own limit, 200 ms of the GPU's global timer
    import time
    t = time.perf_counter()
    rc = lib.msat_selftest_bounded_wait(0)
    dt = time.perf_counter() - t
    assert rc == native.MSAT_ETIMEOUT and b"time limit" in lib.msat_last_error()
    assert 0.15 < dt < 5.0
    # the context and the kernels still work afterwards
    cnf = uniform_ksat(50, 215, 3, seed=0)
    ref = oracle.solve(cnf, 2, 1, 40, mode=oracle.MODE_F32, lr=1e-2, want_hist=False)
    with pkg.Solver.from_cnf(cnf, restarts=2, lr=1e-2) as s:
        s.step(40, want_loss=False, want_cost=False)
        s.check()
        assert np.array_equal(s.best()[1], ref["best_cost"])
