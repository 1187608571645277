"""Partial MaxSAT through the weighted path (Sec. 6 lists weighted and
partial MaxSAT as future work): hard clauses weigh 1 + the total soft
weight.  CPU pins: the encoded optimum, found by enumerating every
assignment with the oracle's exact cost, equals the partial-MaxSAT optimum
computed straight from the definition (hard clauses hold, least soft weight
violated).  GPU: the solver's best assignment keeps every hard clause and
its cost trajectory matches the oracle bit for bit."""
import itertools

import numpy as np
import pytest

from synth import partial_maxsat, random_partial


def _sat(clause, a):
    return any((a[abs(l) - 1] == 1) == (l > 0) for l in clause)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_encoding_optimum_by_enumeration(oracle, seed):
    n = 12
    cnf = random_partial(n, 36, 10, seed=seed)
    top = int(cnf.weights.max())
    clauses = cnf.clauses()
    hard = [c for c, w in zip(clauses, cnf.weights) if w == top]
    soft = [(c, int(w)) for c, w in zip(clauses, cnf.weights) if w != top]
    assert top == 1 + sum(w for _, w in soft)
    grid = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    costs = oracle.cost(cnf, grid)
    best_direct = min(sum(w for c, w in soft if not _sat(c, a))
                      for a in grid if all(_sat(c, a) for c in hard))
    assert costs.min() == best_direct < top  # planted hard clauses are satisfiable
    # any assignment breaking a hard clause costs at least top
    broken = np.array([not all(_sat(c, a) for c in hard) for a in grid])
    assert costs[broken].min() >= top


def test_partial_maxsat_rejects_bad_weights():
    with pytest.raises(ValueError):
        partial_maxsat(3, [[1, 2]], [[3]], [0])
    with pytest.raises(ValueError):
        partial_maxsat(3, [[1, 2]], [[3], [-3]], [1])


@pytest.mark.gpu
def test_gpu_keeps_hard_clauses_and_matches_oracle(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_03640_gb300 as pkg
    from paper_2402_03640_gb300 import build
    build.build()
    cnf = random_partial(300, 900, 150, seed=7)
    top = int(cnf.weights.max())
    B, S, lr = 8, 300, 1e-2
    ref = oracle.solve(cnf, B, 1, S, mode=oracle.MODE_F32, lr=lr, want_hist=False)
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=lr) as s:
        s.step(S, want_loss=False, want_cost=False)
        assign, best = s.best()
    assert np.array_equal(best, ref["best_cost"]) and np.array_equal(assign, ref["best_assign"])
    b = int(np.argmin(best))
    assert best[b] < top
    hard = [c for c, w in zip(cnf.clauses(), cnf.weights) if w == top]
    assert all(_sat(c, assign[b]) for c in hard)
