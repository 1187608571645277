"""CUDA-graph replay of the step (MSAT_STEP_GRAPH) and the time-limited
solve (msat_solve, Algorithm 1 with its wall-clock limit): both give bit for
bit the trajectory of plain msat_step launches, which the oracle pins."""
import numpy as np
import pytest

from synth import pigeonhole, planted_ksat, uniform_ksat

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


def _state(s):
    assign, best = s.best()
    return s.x().copy(), best.copy(), assign.copy()


@pytest.mark.parametrize("steps", [1, 31, 32, 70])
def test_graph_steps_equal_plain_steps(pkg, steps):
    cnf = uniform_ksat(700, 3010, 3, seed=4)
    with pkg.Solver.from_cnf(cnf, restarts=8, lr=3e-2, seed_x=3) as a, \
            pkg.Solver.from_cnf(cnf, restarts=8, lr=3e-2, seed_x=3) as b:
        la, ca = a.step(steps)
        lb, cb = b.step(steps, graph=True)
        xa, ba, aa = _state(a)
        xb, bb, ab = _state(b)
    assert np.array_equal(ca, cb) and np.array_equal(la.view(np.uint32), lb.view(np.uint32))
    assert np.array_equal(xa.view(np.uint32), xb.view(np.uint32))
    assert np.array_equal(ba, bb) and np.array_equal(aa, ab)


def test_graph_steps_mixed_lengths_and_repeat(pkg):
    """Generic clause lengths; the captured graphs are reused across calls."""
    from synth import zipf_weighted
    cnf = zipf_weighted(1500, 6000, seed=5)
    with pkg.Solver.from_cnf(cnf, restarts=4, lr=1e-2) as a, \
            pkg.Solver.from_cnf(cnf, restarts=4, lr=1e-2) as b:
        for k in (40, 3, 33):
            a.step(k)
            b.step(k, graph=True)
        assert np.array_equal(a.x().view(np.uint32), b.x().view(np.uint32))
        assert np.array_equal(a.best()[1], b.best()[1])


def test_solve_equals_step_and_oracle(pkg, oracle):
    """Config 1 (3-SAT n=50, m=215): msat_solve for a fixed step count is
    msat_step; both match the FP32-mode oracle's best costs."""
    cnf = uniform_ksat(50, 215, 3, seed=0)
    B, S, lr = 4, 300, 1e-2
    ref = oracle.solve(cnf, B, 1, S, mode=oracle.MODE_F32, lr=lr, want_hist=False)
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=lr) as a, pkg.Solver.from_cnf(cnf, restarts=B, lr=lr) as b:
        a.step(S, want_loss=False, want_cost=False)
        r = b.solve(S, chunk=64)
        assert r["steps"] == S or r["trace_best_cost"][-1] == 0
        if r["steps"] == S:
            assert np.array_equal(a.x().view(np.uint32), b.x().view(np.uint32))
            assert np.array_equal(a.best()[1], b.best()[1])
            assert np.array_equal(b.best()[1], ref["best_cost"])


def test_solve_stops_at_zero_cost(pkg):
    """A planted satisfiable instance: the loop ends once a restart reaches
    cost 0 (Algorithm 1's stop at zero loss), long before max_steps."""
    cnf = planted_ksat(60, 200, 3, seed=2)
    with pkg.Solver.from_cnf(cnf, restarts=16, lr=5e-2) as s:
        r = s.solve(200000, chunk=25)
        _, best = s.best()
    assert best.min() == 0 and r["trace_best_cost"][-1] == 0
    assert r["steps"] < 200000 and r["steps"] % 25 == 0
    assert np.all(np.diff(r["trace_best_cost"]) <= 0)
    assert np.all(np.diff(r["trace_time_s"]) >= 0)


def test_solve_time_limit(pkg):
    """Pigeonhole PHP(9) has optimum 1, so only the limits end the loop: a
    zero time limit stops after the first chunk, max_steps after the rest."""
    cnf = pigeonhole(9)
    with pkg.Solver.from_cnf(cnf, restarts=8, lr=1e-2) as s:
        r0 = s.solve(10 ** 9, time_limit=0.0, chunk=40)
        assert r0["steps"] == 40 and len(r0["trace_best_cost"]) == 2
        r1 = s.solve(130, chunk=40)
        assert r1["steps"] == 130 and len(r1["trace_best_cost"]) == 5
        assert s.best()[1].min() >= 1


def test_captured_step_with_dense_evaluation_replays_the_same_work(pkg):
    """The benchmark times a step captured into a CUDA graph from the library
    calls (step, then the tensor-core evaluation of the new x).  Replaying it
    K times leaves exactly the state and costs of K plain calls."""
    import torch
    cnf = uniform_ksat(2000, 8600, 3, seed=19)
    B, K = 64, 12
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=1e-2) as a, pkg.Solver.from_cnf(cnf, restarts=B, lr=1e-2) as b:
        ca = torch.empty(B, dtype=torch.int64, device="cuda")
        cb = torch.empty(B, dtype=torch.int64, device="cuda")

        def step(s, out):
            s.step_async(1, final_eval=False)
            s.evaluate_x("dense", out=out)

        for _ in range(2):  # warm-up (first use of the dense backend allocates)
            step(a, ca)
            step(b, cb)
        torch.cuda.synchronize()
        main = torch.cuda.current_stream()
        cap = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        b.set_stream(cap)
        try:
            with torch.cuda.graph(g, stream=cap):
                step(b, cb)
        finally:
            b.set_stream(main)
        # capturing records the step without running it: both are at 2 steps
        for _ in range(K):
            step(a, ca)
        for _ in range(K):
            g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ca.cpu().numpy(), cb.cpu().numpy())
        assert np.array_equal(a.x().view(np.uint32), b.x().view(np.uint32))
        assert np.array_equal(a.best()[1], b.best()[1])
