"""The identity the tensor-core evaluator relies on when it splits a clause
tile along the variables: with W the clause matrix of Sec. 4 and x' a +-1
assignment, every term of S_j = sum_i W_ij x'_i is -1, 0 or +1, so the exact
unsat test S_j = -len_j (no literal true) holds exactly when, for every
piece of a partition of the variables into contiguous ranges, the piece's
partial sum equals minus the number of the clause's literals in that range.
Checked by brute force against the definition (no literal true) on random
instances with mixed lengths, tautologies, empty clauses and arbitrary
piece boundaries.  No GPU, no oracle code."""
import numpy as np
import pytest

from synth import Cnf, uniform_ksat, zipf_weighted


def _canonical(clause):
    out = []
    for l in clause:
        if l not in out:
            out.append(l)
    return out


def _unsat_by_definition(clauses, a01):
    """[b][j]: clause j has no true literal under assignment b."""
    nb = a01.shape[0]
    u = np.zeros((nb, len(clauses)), dtype=bool)
    for j, c in enumerate(clauses):
        true = np.zeros(nb, dtype=bool)
        for l in c:
            v = a01[:, abs(l) - 1].astype(bool)
            true |= v if l > 0 else ~v
        u[:, j] = ~true
    return u


def _pieces_test(clauses, n, a01, bounds):
    """Per piece [lo, hi) of variable indices: partial sums of W^T x' and the
    per-piece targets; a clause with x and not x never counts (its single
    column entry cannot reach the target of two literals)."""
    nb = a01.shape[0]
    xpm = 2 * a01.astype(np.int64) - 1
    ok = np.ones((nb, len(clauses)), dtype=bool)
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        for j, c in enumerate(clauses):
            vars_ = [abs(l) - 1 for l in c]
            taut = len(set(vars_)) < len(vars_)
            col = {}
            for l in c:  # later literals of the same variable overwrite, as in the matrix
                col[abs(l) - 1] = 1 if l > 0 else -1
            s = np.zeros(nb, dtype=np.int64)
            for v, w in col.items():
                if lo <= v < hi:
                    s += w * xpm[:, v]
            cnt = sum(1 for l in c if lo <= abs(l) - 1 < hi)
            ok[:, j] &= (s == -cnt) & (not taut)
    return ok


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_piece_targets_equal_the_unsat_test(seed):
    rng = np.random.default_rng(100 + seed)
    base = zipf_weighted(300, 400, seed=seed) if seed % 2 else uniform_ksat(300, 1200, 3, seed=seed)
    clauses = [_canonical(c) for c in base.clauses()]
    clauses += [[5, -5, 77], [], [299, -300], list(range(1, 301, 3)), list(range(-300, 0, 7)), [1]]
    n = 300
    a01 = rng.integers(0, 2, size=(64, n)).astype(np.uint8)
    want = _unsat_by_definition(clauses, a01)
    for pieces in (1, 2, 3, 4, 7):
        inner = np.sort(rng.choice(np.arange(1, n), size=pieces - 1, replace=False)) if pieces > 1 else []
        bounds = [0] + [int(b) for b in inner] + [n]
        assert np.array_equal(_pieces_test(clauses, n, a01, bounds), want), (seed, bounds)


def test_piece_targets_at_k_step_boundaries():
    """The split the kernel uses: 256-variable k-steps dealt into `split`
    equal ranges of k-steps (piece p covers k-steps [p*kt/split,
    (p+1)*kt/split)); n not a multiple of 256."""
    rng = np.random.default_rng(7)
    n, kt = 1000, (1000 + 255) // 256
    cnf = uniform_ksat(n, 600, 5, seed=3)
    clauses = [_canonical(c) for c in cnf.clauses()] + [list(range(1, n + 1, 9)), []]
    a01 = rng.integers(0, 2, size=(48, n)).astype(np.uint8)
    want = _unsat_by_definition(clauses, a01)
    for split in (2, 3, 4):
        bounds = [min(n, (p * kt // split) * 256) for p in range(split + 1)]
        bounds[-1] = n
        assert np.array_equal(_pieces_test(clauses, n, a01, bounds), want), split


def test_piece_targets_up_to_eight_pieces():
    """Up to eight pieces of whole 256-variable k-steps (the most the
    evaluator splits a tile into), on an instance with 20 k-steps."""
    rng = np.random.default_rng(9)
    n = 5000
    kt = (n + 255) // 256
    cnf = uniform_ksat(n, 400, 3, seed=8)
    clauses = [_canonical(c) for c in cnf.clauses()] + [list(range(1, n + 1, 97)), [], [17, -17, 4000]]
    a01 = rng.integers(0, 2, size=(24, n)).astype(np.uint8)
    want = _unsat_by_definition(clauses, a01)
    for split in (5, 6, 7, 8):
        bounds = [min(n, (p * kt // split) * 256) for p in range(split + 1)]
        bounds[-1] = n
        assert np.array_equal(_pieces_test(clauses, n, a01, bounds), want), split
