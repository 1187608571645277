"""Dense tensor-core evaluation (packed e2m1 W^T times the +-1 batch, exact fp32
accumulation) against the sparse evaluator and the oracle's exact cost:
bit-exact integers for every assignment."""
import numpy as np
import pytest

from synth import Cnf, pigeonhole, uniform_ksat, zipf_weighted

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


def _batch(n, nb, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(nb, n)).astype(np.uint8)


def _check(pkg, oracle, cnf, nbs, seed=0):
    import torch
    with pkg.Solver.from_cnf(cnf, restarts=1) as s:
        for nb in nbs:
            a01 = _batch(cnf.n, nb, seed + nb)
            want = oracle.cost(cnf, a01)
            pm1 = torch.from_numpy((2 * a01.astype(np.int8) - 1).T.copy()).cuda()
            dense = s.evaluate(pm1, backend="dense").cpu().numpy()
            s.check()
            sparse = s.evaluate(pm1, backend="sparse").cpu().numpy()
            assert np.array_equal(sparse, want), f"sparse nb={nb}"
            assert np.array_equal(dense, want), f"dense nb={nb}"


def test_dense_small_batches(pkg, oracle):
    cnf = uniform_ksat(300, 1290, 3, seed=1)
    _check(pkg, oracle, cnf, [1, 7, 16, 33, 100, 256])


def test_dense_multi_tile_batches(pkg, oracle):
    cnf = uniform_ksat(700, 3010, 3, seed=2)
    _check(pkg, oracle, cnf, [257, 300, 513])


def test_dense_weighted_mixed_lengths(pkg, oracle):
    cnf = zipf_weighted(1000, 4000, seed=3)
    _check(pkg, oracle, cnf, [5, 64, 200])


def test_dense_degenerate_and_long_clauses(pkg, oracle):
    cnf = Cnf.from_clauses(140, [[1, -1, 2], [], [3, 3, -4], [5]] +
                           [list(range(6, 140))] + [[-7, -8]] * 3, weights=[4, 9, 2, 1, 3, 5, 6, 7])
    _check(pkg, oracle, cnf, [1, 40])
    _check(pkg, oracle, pigeonhole(30), [24, 130])


def test_dense_config1_full_size(pkg, oracle):
    """Uniform 3-SAT n=5000, m=21500: the 256-assignment batch of the
    batched-restarts configuration."""
    cnf = uniform_ksat(5000, 21500, 3, seed=0)
    _check(pkg, oracle, cnf, [256])


def test_dense_split_tiles(pkg, oracle):
    """More clause tiles than SMs: the leftover tiles are split into k-step
    pieces, each testing its partial sums against per-piece targets, and the
    pieces' bits are ANDed.  Mixed lengths and weights; clauses spanning
    every piece, a tautology, an empty clause and a 1024-literal clause in
    the split tiles; one and two assignment tiles."""
    base = zipf_weighted(5000, 20000, seed=7)
    rng = np.random.default_rng(8)
    extra = [[int(sg) * (1 + 10 * i) for i, sg in enumerate(rng.choice([-1, 1], size=500))] for _ in range(3)]
    extra += [[5, -5, 77], [], [4999, -5000], list(range(1, 1025)), list(range(-5000, 0, 5))]
    w = list(base.weights if base.weights is not None else np.ones(base.m, np.int64)) + [3] * len(extra)
    cnf = Cnf.from_clauses(5000, base.clauses() + extra, weights=w)
    _check(pkg, oracle, cnf, [100, 300])


def test_evaluate_current_x_both_backends(pkg, oracle):
    """The rounded batch of the solver's own x: dense, sparse and the cost the
    step kernels report agree with the oracle after a few steps."""
    cnf = uniform_ksat(2000, 8600, 3, seed=6)
    B, S = 64, 5
    ref = oracle.solve(cnf, B, 1, S, mode=oracle.MODE_F32, lr=3e-2)
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=3e-2) as s:
        _, cost = s.step(S, want_loss=False)
        d = s.evaluate_x("dense").cpu().numpy()
        sp = s.evaluate_x("sparse").cpu().numpy()
        s.check()
    assert np.array_equal(cost, ref["cost_hist"][-1])
    assert np.array_equal(d, cost) and np.array_equal(sp, cost)


@pytest.mark.parametrize("m,nbs", [(19500, [64, 256]), (25000, [16, 200]), (40000, [300]),
                                   (38912, [256, 32]), (32256, [64])])
def test_dense_tile_counts_past_one_wave(pkg, oracle, m, nbs):
    """Clause-tile counts on a persistent grid of one CTA per SM (152 SMs):
    just above one wave (a small leftover split into k-step pieces),
    between one and two waves, above two with two assignment tiles (300
    assignments), exactly two waves (304 tiles, no leftover), and a
    leftover of more than half a wave (252 tiles: 100 CTAs take one more
    whole tile)."""
    cnf = uniform_ksat(3000, m, 3, seed=m)
    _check(pkg, oracle, cnf, nbs, seed=m)


@pytest.mark.gpu
def test_dense_mma_rate_is_a_plausible_peak(pkg):
    """The measured rate of the evaluator's MMA shape: positive, no waits
    given up, and N = 256 at least as fast in flops as N = 64 (the wider
    MMA does more work per instruction); the device stays usable."""
    r256 = pkg.dense_mma_rate(256, 2048)
    r64 = pkg.dense_mma_rate(64, 2048)
    assert r256 > 100.0 and r64 > 10.0
    assert r256 >= 0.9 * r64
    import torch
    assert int(torch.ones(4, device="cuda").sum().item()) == 4
