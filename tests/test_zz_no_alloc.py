"""msat_objective_noalloc, the entry point for callers that may not allocate
device memory (a host that gives the library a fixed memory budget, a
latency-bound loop that bans cudaMalloc's device synchronisation, a plugin
that runs where allocation calls are forbidden).  It keeps its scratch in an
array compiled into the library; its results must equal those of the
context path (msat_forward) on the same x, call after call.  This file is
collected last so a failure here does not stop the rest of the suite."""
import ctypes

import numpy as np
import pytest

from synth import Cnf, uniform_ksat, zipf_weighted


def _lib():
    from paper_2402_03640_gb300 import build, native
    build.build()
    return native, native.load()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    native, lib = _lib()
    off = np.zeros(1, np.int64)
    for B in (0, 3, 2048):
        rc = lib.msat_objective_noalloc(4, 0, ctypes.c_void_p(off.ctypes.data), None, None,
                                        ctypes.c_void_p(off.ctypes.data), B,
                                        ctypes.c_void_p(off.ctypes.data),
                                        ctypes.c_void_p(off.ctypes.data), None)
        assert rc == native.MSAT_EINVAL
        assert "restarts" in lib.msat_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("kind,B", [("ksat", 1), ("ksat", 16), ("ksat", 512), ("zipf", 4),
                                    ("long", 2)])
def test_noalloc_matches_context_path(kind, B):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    native, lib = _lib()
    import paper_2402_03640_gb300 as pkg
    if kind == "ksat":
        cnf = uniform_ksat(3000, 12900, 3, seed=3)
    elif kind == "zipf":
        cnf = zipf_weighted(4000, 16000, seed=8)
    else:  # clauses longer than one 32-literal leaf
        rng = np.random.default_rng(5)
        cl = []
        for _ in range(400):
            k = int(rng.integers(1, 90))
            cl.append((rng.choice(300, size=k, replace=False) + 1) * rng.choice([-1, 1], size=k))
        cnf = Cnf.from_clauses(300, [[int(v) for v in c] for c in cl],
                               weights=rng.integers(1, 50, size=400))
    dev = torch.device("cuda", 0)
    off = torch.from_numpy(cnf.off.astype(np.int64)).to(dev)
    lits = torch.from_numpy(cnf.lits.astype(np.int32)).to(dev)
    w = None if cnf.weights is None else torch.from_numpy(cnf.weights.astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(B)
    with pkg.Solver.from_cnf(cnf, restarts=B) as s:
        for call in range(2):  # two calls in a row share the scratch array
            x = torch.from_numpy(rng.uniform(-1, 1, size=(cnf.n, B)).astype(np.float32)).to(dev)
            loss_ref, cost_ref = s.forward(x)
            cost = torch.full((B,), -1, dtype=torch.int64, device=dev)
            loss = torch.full((B,), float("nan"), dtype=torch.float32, device=dev)
            rc = lib.msat_objective_noalloc(cnf.n, cnf.m, _ptr(off), _ptr(lits), _ptr(w), _ptr(x), B,
                                            _ptr(cost), _ptr(loss), ctypes.c_void_p(stream))
            assert rc == 0, lib.msat_last_error().decode()
            torch.cuda.synchronize()
            assert torch.equal(cost.cpu(), cost_ref.cpu()), f"call {call}: cost differs"
            assert np.allclose(loss.cpu().numpy(), loss_ref.cpu().numpy(), rtol=1e-5, atol=0), \
                f"call {call}: loss differs"


def _edge_instance():
    """Weighted clauses of every kind the entry point accepts: long ones
    (several 32-literal leaves), empty ones (always unsat, f = 0), x or not
    x (never unsat), units; no literal repeated inside a clause."""
    rng = np.random.default_rng(17)
    n = 400
    cl = [[], [5, -5], [3], [-3], [], [7, -9, 9]]
    for _ in range(600):
        k = int(rng.choice([1, 2, 3, 33, 64, 97]))
        cl.append([int(v) for v in (rng.choice(n, size=k, replace=False) + 1) * rng.choice([-1, 1], size=k)])
    return Cnf.from_clauses(n, cl, weights=rng.integers(1, 1000, size=len(cl)))


@pytest.mark.gpu
@pytest.mark.parametrize("case,B", [("edge", 1), ("edge", 8), ("edge", 64), ("ksat1e6", 4)])
def test_noalloc_matches_oracle(oracle, case, B):
    """The entry point against the oracle's FP32 objective: exact costs and
    the loss within 1e-5 relative, twice in a row on the shared scratch."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    native, lib = _lib()
    # a million clauses: each thread sums thousands of loss terms
    cnf = _edge_instance() if case == "edge" else uniform_ksat(250000, 1075000, 3, seed=21)
    dev = torch.device("cuda", 0)
    off = torch.from_numpy(cnf.off.astype(np.int64)).to(dev)
    lits = torch.from_numpy(cnf.lits.astype(np.int32)).to(dev)
    w = None if cnf.weights is None else torch.from_numpy(cnf.weights.astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x32 = oracle.init_x(cnf.n, B, 100 + call)
        ref = oracle.objective_f32(cnf, x32, want_grad=False)
        x = torch.from_numpy(x32).to(dev)
        cost = torch.full((B,), -1, dtype=torch.int64, device=dev)
        loss = torch.full((B,), float("nan"), dtype=torch.float32, device=dev)
        rc = lib.msat_objective_noalloc(cnf.n, cnf.m, _ptr(off), _ptr(lits), _ptr(w), _ptr(x), B,
                                        _ptr(cost), _ptr(loss), ctypes.c_void_p(stream))
        assert rc == 0, lib.msat_last_error().decode()
        torch.cuda.synchronize()
        assert np.array_equal(cost.cpu().numpy(), ref["cost"]), f"call {call}: cost differs"
        assert np.allclose(loss.cpu().numpy().astype(np.float64), ref["loss"], rtol=1e-5, atol=0), \
            f"call {call}: loss differs"
