"""Pins of the CPU oracle against facts fixed outside it: values the paper
prints for its worked example, brute-force enumeration, the dense-matrix
identity of the exact unsat test, known optima of structured instances,
central finite differences, hand-computed Adam steps, published SplitMix64
outputs, libm's tanh, and exact sums.  No GPU."""
import json
import math
import os

import numpy as np
import pytest

from synth import Cnf, ordering, pigeonhole, planted_ksat, uniform_ksat, zipf_weighted

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _all_assignments(n):
    a = (np.arange(2 ** n, dtype=np.int64)[:, None] >> np.arange(n)[None, :]) & 1
    return a.astype(np.uint8)


def _dense_W(cnf):
    """W[i][j] = +1 if x_i in c_j, -1 if not-x_i in c_j (Sec. 4)."""
    W = np.zeros((cnf.n, cnf.m), dtype=np.int64)
    for j, c in enumerate(cnf.clauses()):
        for l in c:
            W[abs(l) - 1, j] = 1 if l > 0 else -1
    return W


def _ulp_dist(a, b):
    ia = np.array([a], dtype=np.float32).view(np.int32)[0].astype(np.int64)
    ib = np.array([b], dtype=np.float32).view(np.int32)[0].astype(np.int64)
    if ia < 0:
        ia = -(ia & 0x7FFFFFFF)
    if ib < 0:
        ib = -(ib & 0x7FFFFFFF)
    return abs(ia - ib)


# ------------------------------------------------------------ generators

def test_splitmix64_published_outputs(oracle):
    # First outputs of the reference splitmix64 generator started from seed 0.
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle.splitmix64(0, c) for c in range(3)] == ref
    from synth import splitmix64
    assert [int(v) for v in splitmix64(0, np.arange(3))] == ref


def test_init_x_grid_and_restart_independence(oracle):
    x = oracle.init_x(1000, 4, seed=1)
    assert x.dtype == np.float32 and x.shape == (1000, 4)
    assert x.min() >= -1.0 and x.max() < 1.0
    k = (x.astype(np.float64) + 1.0) * 2.0 ** 23          # grid points k in [0, 2^24)
    assert np.all(k == np.round(k))
    assert abs(float(x.mean())) < 0.05
    # restart b's start does not depend on how many restarts run
    x1 = oracle.init_x(1000, 1, seed=1)
    assert np.array_equal(x1[:, 0], x[:, 0])
    # counter c = b*n + i of the stream: spot-check one value by hand
    u = oracle.splitmix64(1, 2 * 1000 + 7)
    assert x[7, 2] == np.float32((u >> 40) * 2.0 ** -23 - 1.0)


def test_generators_table2_counts():
    g = _gold("table2_php_gt.json")
    for h, (nv, nc) in g["php"].items():
        c = pigeonhole(int(h))
        assert (c.n, c.m) == (nv, nc), f"PHP {h}"
    for s, (nv, nc) in g["gt"].items():
        c = ordering(int(s))
        assert (c.n, c.m) == (nv, nc), f"GT {s}"


def test_uniform_ksat_shape_and_determinism():
    a = uniform_ksat(50, 215, 3, seed=0)
    b = uniform_ksat(50, 215, 3, seed=0)
    assert np.array_equal(a.lits, b.lits)
    C = np.abs(a.lits.reshape(-1, 3))
    assert C.min() >= 1 and C.max() <= 50
    assert np.all((C[:, 0] != C[:, 1]) & (C[:, 0] != C[:, 2]) & (C[:, 1] != C[:, 2]))
    neg = (a.lits < 0).mean()
    assert 0.4 < neg < 0.6


def test_zipf_weighted_structure():
    z = zipf_weighted(2000, 10000, seed=3)
    lens = np.diff(z.off)
    assert lens.min() >= 2 and lens.max() <= 20
    assert 3.6 < lens.mean() < 4.4                      # 2 + Geom(1/3): mean 4
    assert z.weights.min() >= 1 and z.weights.max() <= 1000
    for j in range(0, z.m, 97):
        v = np.abs(z.lits[z.off[j]:z.off[j + 1]])
        assert len(set(v.tolist())) == len(v)
    deg = np.bincount(np.abs(z.lits) - 1, minlength=z.n)
    assert deg.max() > 20 * deg.mean()                  # heavy head


# ------------------------------------------------------------ tanh / sums

def test_tanh32_against_libm(oracle):
    vals = np.concatenate([
        np.linspace(-9.5, 9.5, 4001),
        np.logspace(-40, 1, 800), -np.logspace(-40, 1, 800),
        np.array([0.3465, 0.3466, 0.5, 0.55, 1.0, 8.6, 8.99, 9.0, 20.0, 1e30, 1e-45]),
    ]).astype(np.float32)
    worst = 0
    for a in vals:
        got = oracle.tanh32(float(a))
        ref = np.float32(math.tanh(float(a)))
        worst = max(worst, _ulp_dist(got, ref))
        assert (got > 0) == (a > 0)
    assert worst <= 2, worst
    assert math.copysign(1.0, oracle.tanh32(-0.0)) == -1.0
    assert oracle.tanh32(float("inf")) == 1.0 and oracle.tanh32(float("-inf")) == -1.0
    assert math.isnan(oracle.tanh32(float("nan")))


def _dyadic(leaves):
    # the leaf tree: split at the largest power of two below the count
    K = len(leaves)
    if K == 1:
        return leaves[0]
    h = 1
    while h * 2 < K:
        h *= 2
    return np.float32(_dyadic(leaves[:h]) + _dyadic(leaves[h:]))


@pytest.mark.parametrize("L", [0, 1, 2, 31, 32, 33, 64, 65, 100, 1000, 4097])
def test_canon_sum_definition(oracle, L):
    rng = np.random.default_rng(L)
    a = rng.standard_normal(L).astype(np.float32) * np.float32(3.0)
    got = oracle.canon_sum(a)
    if L == 0:
        assert got == 0.0
        return
    leaves = []
    for lo in range(0, L, 32):
        s = a[lo]
        for v in a[lo + 1:lo + 32]:
            s = np.float32(s + v)
        leaves.append(s)
    assert np.float32(got) == _dyadic(leaves)
    exact = math.fsum(a.astype(np.float64).tolist())
    bound = (math.log2(L) + 32) * 2.0 ** -24 * float(np.abs(a).astype(np.float64).sum())
    assert abs(got - exact) <= bound
    ints = np.round(a * 100).astype(np.float32)       # small integers: every sum exact
    assert oracle.canon_sum(ints) == float(ints.astype(np.int64).sum())


# ------------------------------------------------------ worked example

def test_worked_example_forward_and_mask(oracle):
    g = _gold("worked_example.json")
    cnf = Cnf.from_clauses(g["n"], g["clauses"])
    x = np.array(g["x"])[:, None]
    r = oracle.objective_f64(cnf, x, want_f=True)
    assert np.array_equal(np.round(r["f"][:, 0], 2), np.array(g["f_printed_2dp"]))
    assert r["unsat"][:, 0].tolist() == g["unsat_printed"]
    assert r["cost"][0] == sum(g["unsat_printed"])
    r32 = oracle.objective_f32(cnf, x.astype(np.float32), want_f=True)
    assert np.array_equal(np.round(r32["f"][:, 0].astype(np.float64), 2), np.array(g["f_printed_2dp"]))
    assert r32["unsat"][:, 0].tolist() == g["unsat_printed"]
    # loss: mean of f^2 over the two unsatisfied clauses
    t1, t2 = math.tanh(0.43), math.tanh(1.27)
    assert r["loss"][0] == pytest.approx((t1 * t1 + t2 * t2) / 2, rel=1e-14)
    # gradient by hand: dL/dx_i = -f_i (1 - t_i^2) with f_i = -t_i
    assert r["grad"][:, 0] == pytest.approx([t1 * (1 - t1 * t1), t2 * (1 - t2 * t2)], rel=1e-13)


def test_worked_example_optimum_by_enumeration(oracle):
    g = _gold("worked_example.json")
    cnf = Cnf.from_clauses(g["n"], g["clauses"])
    costs = oracle.cost(cnf, _all_assignments(2))
    assert costs.min() == g["optimum_cost"]


def test_worked_example_one_adam_step(oracle):
    """Adam's first step has m_hat = g and v_hat = g^2, so each coordinate moves
    by lr * g / (|g| + eps); with lr = 0.1 both values drop by about 0.1
    (the paper prints [0.34, 1.23]; only its direction is reproduced)."""
    g = _gold("worked_example.json")
    cnf = Cnf.from_clauses(g["n"], g["clauses"])
    lr = g["example_lr"]
    x = np.array(g["x"], dtype=np.float32)[:, None].copy()
    mom = np.zeros_like(x)
    vel = np.zeros_like(x)
    best = np.array([3], dtype=np.int64)
    c, loss, grad = oracle.step32(cnf, x, mom, vel, 0, best, lr=lr)
    assert c[0] == 2 and best[0] == 2
    gv = grad[:, 0].astype(np.float64)
    want = np.array(g["x"]) - lr * gv / (np.abs(gv) + 1e-8)
    assert x[:, 0] == pytest.approx(want, abs=2e-7)
    assert np.all(x[:, 0] < np.array(g["x"]))                  # both decrease
    assert x[:, 0] == pytest.approx([0.33, 1.17], abs=1e-6)


# -------------------------------------------------- exact evaluator

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cost_brute_force_and_dense_identity(oracle, seed):
    n = 12
    cnf = uniform_ksat(n, 60, 3, seed=seed)
    w = 1 + (np.arange(cnf.m) * 7919 + seed) % 13
    cw = Cnf(n=cnf.n, off=cnf.off, lits=cnf.lits, weights=w.astype(np.int64))
    A = _all_assignments(n)
    got = oracle.cost(cnf, A)
    gotw = oracle.cost(cw, A)
    # Sec. 4 identity, read with x' mapped to +-1: clause j is unsatisfied
    # iff sum_i W_ij xhat_i equals -len(c_j)
    W = _dense_W(cnf)
    lens = np.diff(cnf.off)
    S = (2 * A.astype(np.int64) - 1) @ W
    unsat = S == -lens[None, :]
    assert np.array_equal(got, unsat.sum(axis=1))
    assert np.array_equal(gotw, unsat.astype(np.int64) @ w)
    # and directly: no literal of the clause is true
    cl = cnf.clauses()
    for r in range(0, len(A), 257):
        a = A[r]
        direct = sum(1 for c in cl if not any((a[abs(l) - 1] == 1) == (l > 0) for l in c))
        assert direct == got[r]


@pytest.mark.parametrize("h", [2, 3, 4])
def test_pigeonhole_optimum_is_one(oracle, h):
    cnf = pigeonhole(h)
    costs = oracle.cost(cnf, _all_assignments(cnf.n))
    assert costs.min() == 1


@pytest.mark.parametrize("s", [1, 2, 3])
def test_ordering_optimum_is_one(oracle, s):
    cnf = ordering(s)
    costs = oracle.cost(cnf, _all_assignments(cnf.n))
    assert costs.min() == 1


def test_planted_has_optimum_zero(oracle):
    cnf = planted_ksat(14, 60, 3, seed=5)
    costs = oracle.cost(cnf, _all_assignments(14))
    assert costs.min() == 0


def test_duplicate_and_tautological_literals(oracle):
    base = Cnf.from_clauses(3, [[1, 2], [-3], [2, 3]])
    dup = Cnf.from_clauses(3, [[1, 1, 2], [-3, -3], [2, 3, 2]])
    taut = Cnf.from_clauses(3, [[1, 2], [-3], [2, 3], [1, -1]])
    A = _all_assignments(3)
    assert np.array_equal(oracle.cost(base, A), oracle.cost(dup, A))
    assert np.array_equal(oracle.cost(base, A), oracle.cost(taut, A))
    x = np.array([[0.3], [-0.2], [0.7]])
    r0 = oracle.objective_f64(base, x, want_f=True)
    r1 = oracle.objective_f64(dup, x, want_f=True)
    assert np.array_equal(r0["f"], r1["f"]) and np.array_equal(r0["grad"], r1["grad"])


def test_empty_clause_always_unsat(oracle):
    cnf = Cnf.from_clauses(2, [[], [1, 2], [-1]], weights=[5, 1, 1])
    A = _all_assignments(2)
    c = oracle.cost(cnf, A)
    assert c.min() >= 5
    r = oracle.objective_f64(cnf, np.array([[0.5], [0.5]]), want_f=True)
    assert r["f"][0, 0] == 0.0 and r["unsat"][0, 0] == 1
    assert r["cost"][0] == 6
    # loss: (5*0^2 + 1*tanh(.5)^2) / 6
    assert r["loss"][0] == pytest.approx(math.tanh(0.5) ** 2 / 6, rel=1e-14)


def test_invalid_cnf_rejected(oracle):
    bad_var = Cnf.from_clauses(2, [[1, 3]])
    with pytest.raises(ValueError):
        oracle.cost(bad_var, np.zeros((1, 2), np.uint8))
    zero_lit = Cnf.from_clauses(2, [[1, 0]])
    with pytest.raises(ValueError):
        oracle.cost(zero_lit, np.zeros((1, 2), np.uint8))
    bad_w = Cnf.from_clauses(2, [[1, 2]], weights=[0])
    with pytest.raises(ValueError):
        oracle.cost(bad_w, np.zeros((1, 2), np.uint8))


# ------------------------------------------------------- gradient / loss

@pytest.mark.parametrize("weighted,loss_norm", [(False, "mean_unsat"), (True, "mean_unsat"),
                                               (True, "sum_unsat"), (True, "mean_all")])
def test_gradient_central_differences(oracle, weighted, loss_norm):
    cnf = uniform_ksat(300, 1290, 3, seed=11)
    if weighted:
        cnf = Cnf(n=cnf.n, off=cnf.off, lits=cnf.lits,
                  weights=(1 + np.arange(cnf.m) % 997).astype(np.int64))
    x = oracle.init_x(cnf.n, 2, seed=4).astype(np.float64)
    base = oracle.objective_f64(cnf, x, want_f=True, loss_norm=loss_norm)
    h = 1e-6
    rng = np.random.default_rng(0)
    idx = [(i, b) for i, b in zip(rng.integers(0, cnf.n, 200), rng.integers(0, 2, 200))
           if abs(x[i, b]) > 10 * h]
    gmax = np.abs(base["grad"]).max()
    for i, b in idx[:60]:
        xp = x.copy(); xp[i, b] += h
        xm = x.copy(); xm[i, b] -= h
        rp = oracle.objective_f64(cnf, xp, want_f=True, want_grad=False, loss_norm=loss_norm)
        rm = oracle.objective_f64(cnf, xm, want_f=True, want_grad=False, loss_norm=loss_norm)
        assert np.array_equal(rp["unsat"], base["unsat"]) and np.array_equal(rm["unsat"], base["unsat"])
        fd = (rp["loss"][b] - rm["loss"][b]) / (2 * h)
        assert abs(fd - base["grad"][i, b]) <= 1e-6 * gmax + 1e-10


def test_loss_normalisers_closed_form(oracle):
    """The three readings of the loss normaliser (Sec. 4 "MSE ... over the
    unsatisfied clauses"): sum_U w f^2 divided by W_U, by 1, by the total
    weight -- computed here from the oracle's f and unsat mask by numpy."""
    cnf = zipf_weighted(400, 1600, seed=8)
    x = oracle.init_x(cnf.n, 3, seed=2).astype(np.float64)
    w = cnf.weights.astype(np.float64)
    r = {ln: oracle.objective_f64(cnf, x, want_f=True, loss_norm=ln)
         for ln in ("mean_unsat", "sum_unsat", "mean_all")}
    f, u = r["mean_unsat"]["f"], r["mean_unsat"]["unsat"].astype(bool)
    S = np.array([(w[u[:, b]] * f[u[:, b], b] ** 2).sum() for b in range(3)])
    WU = np.array([w[u[:, b]].sum() for b in range(3)])
    assert np.array_equal(WU.astype(np.int64), r["mean_unsat"]["cost"])
    assert r["mean_unsat"]["loss"] == pytest.approx(S / WU, rel=1e-13)
    assert r["sum_unsat"]["loss"] == pytest.approx(S, rel=1e-13)
    assert r["mean_all"]["loss"] == pytest.approx(S / w.sum(), rel=1e-13)
    # the gradients differ by the same per-restart factors
    assert r["sum_unsat"]["grad"] == pytest.approx(r["mean_unsat"]["grad"] * WU[None, :], rel=1e-12, abs=1e-14)
    assert r["mean_all"]["grad"] == pytest.approx(r["sum_unsat"]["grad"] / w.sum(), rel=1e-12, abs=1e-18)
    for ln in ("sum_unsat", "mean_all"):  # FP32-canon tracks FP64 in every reading
        b32 = oracle.objective_f32(cnf, x.astype(np.float32), loss_norm=ln)
        g64 = r[ln]["grad"]
        assert np.all(np.abs(b32["grad"] - g64) <= 1e-5 * np.abs(g64).max(axis=0)[None, :])
        assert np.allclose(b32["loss"], r[ln]["loss"], rtol=1e-5, atol=0)
    # the default is restored after each call
    assert oracle.objective_f64(cnf, x)["loss"] == pytest.approx(S / WU, rel=1e-13)


def test_uniform_weights_reduce_to_unweighted(oracle):
    cnf = uniform_ksat(200, 860, 3, seed=2)
    cw = Cnf(n=cnf.n, off=cnf.off, lits=cnf.lits, weights=np.full(cnf.m, 7, np.int64))
    x = oracle.init_x(cnf.n, 3, seed=9).astype(np.float64)
    a = oracle.objective_f64(cnf, x)
    b = oracle.objective_f64(cw, x)
    assert np.array_equal(b["cost"], 7 * a["cost"])
    assert b["loss"] == pytest.approx(a["loss"], rel=1e-14)
    assert b["grad"] == pytest.approx(a["grad"], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("maker", ["ksat", "zipf"])
def test_fp32_canon_within_tolerance_of_fp64(oracle, maker):
    cnf = uniform_ksat(2000, 8600, 3, seed=1) if maker == "ksat" else zipf_weighted(3000, 12000, seed=2)
    x32 = oracle.init_x(cnf.n, 4, seed=1)
    a = oracle.objective_f64(cnf, x32.astype(np.float64), want_f=True)
    b = oracle.objective_f32(cnf, x32, want_f=True)
    assert np.array_equal(a["unsat"], b["unsat"]) and np.array_equal(a["cost"], b["cost"])
    assert np.allclose(b["loss"], a["loss"], rtol=1e-5, atol=0)
    g64 = a["grad"]
    tol = 1e-5 * np.abs(g64).max(axis=0)
    assert np.all(np.abs(b["grad"].astype(np.float64) - g64) <= tol[None, :])
    assert np.all(np.abs(b["f"].astype(np.float64) - a["f"]) <= 1e-5 * np.maximum(1.0, np.abs(a["f"])))


# ----------------------------------------------------------- Adam / loop

@pytest.mark.parametrize("mode", [0, 1])
def test_two_adam_steps_by_hand(oracle, mode):
    """Kingma & Ba's Adam with bias correction, written out for t = 1, 2."""
    cnf = uniform_ksat(60, 258, 3, seed=3)
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    x0 = oracle.init_x(cnf.n, 1, seed=1).astype(np.float64)
    g1 = oracle.objective_f64(cnf, x0)["grad"]
    m1 = (1 - b1) * g1
    v1 = (1 - b2) * g1 * g1
    x1 = x0 - lr * (m1 / (1 - b1)) / (np.sqrt(v1 / (1 - b2)) + eps)
    g2 = oracle.objective_f64(cnf, x1)["grad"]
    m2 = b1 * m1 + (1 - b1) * g2
    v2 = b2 * v1 + (1 - b2) * g2 * g2
    x2 = x1 - lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    r1 = oracle.solve(cnf, 1, 1, 1, mode=mode, lr=lr)
    r2 = oracle.solve(cnf, 1, 1, 2, mode=mode, lr=lr)
    tol = 1e-12 if mode == 0 else 1e-6
    assert np.allclose(r1["x_final"], x1, atol=tol, rtol=0)
    assert np.allclose(r2["x_final"], x2, atol=tol, rtol=0)


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_bookkeeping(oracle, mode):
    cnf = uniform_ksat(50, 215, 3, seed=0)
    r = oracle.solve(cnf, 3, seed_x=1, steps=300, mode=mode, lr=1e-2)
    ch = r["cost_hist"]
    assert ch.shape == (301, 3)
    assert np.array_equal(r["best_cost"], np.minimum(cnf.m, ch.min(axis=0)))
    # the stored best assignment has exactly the best cost
    assert np.array_equal(oracle.cost(cnf, r["best_assign"]), r["best_cost"])
    # a restart that reached cost 0 stays there
    for b in range(3):
        z = np.nonzero(ch[:, b] == 0)[0]
        if z.size:
            assert np.all(ch[z[0]:, b] == 0)


def test_solve_never_beats_enumerated_optimum(oracle):
    for seed in range(3):
        cnf = uniform_ksat(16, 100, 3, seed=seed)
        opt = oracle.cost(cnf, _all_assignments(16)).min()
        r = oracle.solve(cnf, 4, seed_x=seed, steps=400, mode=1, lr=5e-2)
        assert np.all(r["best_cost"] >= opt)
    cnf = pigeonhole(3)
    r = oracle.solve(cnf, 4, seed_x=0, steps=500, mode=1, lr=5e-2)
    assert np.all(r["best_cost"] >= 1)


def test_solved_restart_freezes(oracle):
    cnf = planted_ksat(40, 120, 3, seed=1)
    r = oracle.solve(cnf, 4, seed_x=2, steps=2000, mode=1, lr=5e-2)
    ch = r["cost_hist"]
    solved = [b for b in range(4) if (ch[:, b] == 0).any()]
    assert solved, "planted instance should be solved by some restart"
    for b in solved:
        z = int(np.nonzero(ch[:, b] == 0)[0][0])
        part = oracle.solve(cnf, 4, seed_x=2, steps=z, mode=1, lr=5e-2)
        assert np.array_equal(part["x_final"][:, b], r["x_final"][:, b])


def test_fp32_canon_trajectory_tracks_fp64(oracle):
    """Configuration-0 instance (uniform 3-SAT, n=50, m=215, seed 0; x from
    seed 1; 1000 steps at lr 1e-4).  The float contract follows the double
    definition step for step until variables start to oscillate around 0
    with an amplitude near lr; from there rounding decides the sign pattern
    (chaotic), which is why GPU trajectories are compared bit for bit with
    the float contract and only per step with the double definition."""
    cnf = uniform_ksat(50, 215, 3, seed=0)
    a = oracle.solve(cnf, 1, 1, 1000, mode=0)
    b = oracle.solve(cnf, 1, 1, 1000, mode=1)
    assert np.array_equal(a["cost_hist"][:900], b["cost_hist"][:900])
    assert np.array_equal(a["best_cost"], b["best_cost"])
    assert np.allclose(a["loss_hist"][:900], b["loss_hist"][:900], rtol=1e-5, atol=0)
    assert np.allclose(a["x_final"], b["x_final"], atol=1e-4, rtol=0)


def test_step32_matches_solve(oracle):
    cnf = zipf_weighted(500, 2000, seed=4)
    B, S = 2, 25
    ref = oracle.solve(cnf, B, 1, S, mode=1, lr=1e-3)
    x = oracle.init_x(cnf.n, B, 1)
    mom = np.zeros_like(x)
    vel = np.zeros_like(x)
    best = np.full(B, int(cnf.weights.sum()), np.int64)
    costs = []
    for s in range(S):
        c, _, _ = oracle.step32(cnf, x, mom, vel, s, best, lr=1e-3)
        costs.append(c.copy())
    c, _, _ = oracle.step32(cnf, x, mom, vel, S, best, update=False, lr=1e-3)
    costs.append(c.copy())
    assert np.array_equal(np.array(costs), ref["cost_hist"])
    assert np.array_equal(x.astype(np.float64), ref["x_final"])
    assert np.array_equal(best, ref["best_cost"])


@pytest.mark.parametrize("mode", [0, 1])
def test_restart_split_equals_whole_run(oracle, mode):
    """Restarts never interact: solving groups of restarts side by side
    (each from its own first restart index) gives the arrays of one run."""
    from synth import uniform_ksat, zipf_weighted
    for cnf, B in ((uniform_ksat(60, 258, 3, seed=4), 7), (zipf_weighted(80, 300, seed=2), 5)):
        whole = oracle.solve(cnf, B, 3, 25, mode=mode, lr=5e-2)
        split = oracle.solve(cnf, B, 3, 25, mode=mode, lr=5e-2, threads=3)
        for k in ("cost_hist", "loss_hist", "best_cost", "best_assign", "x_final"):
            assert np.array_equal(whole[k], split[k]), k
