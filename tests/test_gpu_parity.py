"""GPU path against the CPU oracle, through the C ABI.

Unsat counts, weighted costs, rounded (best) assignments and relaxed x are
compared bit for bit with the oracle's FP32-canon mode (same seeds, same
instances); losses and gradients within 1e-5 relative of the FP64 mode.
Sizes span several thread blocks with ragged tails; the full-size
configurations are checked on short trajectories."""
import os

import numpy as np
import pytest

from synth import Cnf, pigeonhole, planted_ksat, uniform_ksat, zipf_weighted

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


def gpu_trajectory(pkg, cnf, B, steps, lr, seed_x=1, chunk=1, per_pass=True, **kw):
    """Cost after each evaluation (x_0 .. x_steps), loss of each update, final
    x.  per_pass: the per-pass kernels even for instances small enough for
    the single-CTA kernel (False: whichever route msat_step takes)."""
    costs, losses = [], []
    with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=seed_x, lr=lr, **kw) as s:
        costs.append(s.step(0, want_loss=False)[1])
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            loss, cost = s.step(k, per_pass=per_pass)
            done += k
            costs.append(cost)
            losses.append(loss)
        x = s.x()
        assign, best = s.best()
        info = s.info()
    return dict(cost_hist=np.array(costs), loss_hist=np.array(losses), x=x, best_assign=assign,
                best_cost=best, info=info)


def check_bit_exact(oracle, cnf, B, steps, lr, chunk=1, seed_x=1, per_pass=True, oracle_threads=1, **kw):
    ref = oracle.solve(cnf, B, seed_x, steps, mode=oracle.MODE_F32, lr=lr,
                       loss_norm=kw.get("loss_norm", "mean_unsat"), threads=oracle_threads)
    got = gpu_trajectory(pkg_module(), cnf, B, steps, lr, seed_x=seed_x, chunk=chunk,
                         per_pass=per_pass, **kw)
    idx = [0] + [min(k, steps) for k in range(chunk, steps + chunk, chunk)] if steps else [0]
    want_costs = ref["cost_hist"][idx]
    assert np.array_equal(got["cost_hist"], want_costs), "unsat cost history differs"
    assert np.array_equal(got["x"].astype(np.float64), ref["x_final"]), "relaxed x differs"
    assert np.array_equal(got["best_cost"], ref["best_cost"])
    assert np.array_equal(got["best_assign"], ref["best_assign"])
    if chunk == 1 and steps:
        # loss of x_s vs the oracle's (reported in double from the same float f)
        assert np.allclose(got["loss_hist"], ref["loss_hist"], rtol=1e-5, atol=1e-7)
    return got, ref


_PKG = {}


def pkg_module():
    return _PKG["p"]


@pytest.fixture(autouse=True)
def _remember(pkg):
    _PKG["p"] = pkg


# ---------------------------------------------------------------- init

@pytest.mark.parametrize("n,B", [(50, 1), (1000, 16), (777, 8), (5000, 256), (33, 2)])
def test_init_matches_oracle(pkg, oracle, n, B):
    cnf = uniform_ksat(max(n, 3), 4 * n, 3, seed=0)
    with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1) as s:
        x = s.x()
    assert np.array_equal(x, oracle.init_x(cnf.n, B, 1))


# --------------------------------------------------------- trajectories

def test_config0_full_trajectory(pkg, oracle):
    """Uniform 3-SAT n=50, m=215 (seed 0), x from seed 1, 1000 Adam steps
    at lr 1e-4: every unsat count, the final x and the best assignment."""
    cnf = uniform_ksat(50, 215, 3, seed=0)
    got, ref = check_bit_exact(oracle, cnf, 1, 1000, 1e-4, chunk=1)
    assert got["cost_hist"][-1, 0] == ref["cost_hist"][-1, 0]


@pytest.mark.parametrize("B", [1, 2, 4, 16, 64, 128, 256, 1024])
def test_restarts_trajectory(pkg, oracle, B):
    cnf = uniform_ksat(300, 1290, 3, seed=5)
    check_bit_exact(oracle, cnf, B, 60, 1e-2)


@pytest.mark.parametrize("f_mode", ["store", "recompute", "expanded"])
@pytest.mark.parametrize("B", [1, 4, 16, 256])
def test_f_modes_identical(pkg, oracle, f_mode, B):
    """Every way of getting f_j to the variable pass gives the same bits."""
    cnf = uniform_ksat(700, 3010, 3, seed=9)
    check_bit_exact(oracle, cnf, B, 12, 2e-2, f_mode=f_mode)


@pytest.mark.parametrize("B", [1, 8, 16, 64])
def test_store_rows_grouped_by_block(pkg, oracle, B):
    """The store's rows grouped by the variable pass's light blocks (the
    occurrence words carry rows, the clause pass reads row-ordered clause
    arrays): the same bits as clause order, on fixed-length clauses with
    several light blocks and on weighted mixed-length clauses with heavy
    variables (clauses whose variables are all heavy come last)."""
    cnf = uniform_ksat(3000, 12900, 3, seed=51)
    got, _ = check_bit_exact(oracle, cnf, B, 12, 5e-2, row_order="block", light_rows=64)
    assert got["info"]["small_kernel"] == 0
    z = zipf_weighted(2500, 9000, seed=52)
    check_bit_exact(oracle, z, B, 8, 2e-2, row_order="block", heavy_deg=16)


@pytest.mark.parametrize("heavy_deg", [1, 8, 40])
@pytest.mark.parametrize("f_mode", ["store", "recompute"])
def test_heavy_split_identical(pkg, oracle, heavy_deg, f_mode):
    """Forcing variables into the chunked heavy path keeps every bit."""
    cnf = zipf_weighted(1500, 6000, seed=2)
    check_bit_exact(oracle, cnf, 2, 8, 2e-2, f_mode=f_mode, heavy_deg=heavy_deg)
    cnf3 = uniform_ksat(400, 1720, 3, seed=4)
    check_bit_exact(oracle, cnf3, 16, 8, 2e-2, f_mode="expanded", heavy_deg=heavy_deg)


@pytest.mark.parametrize("shape", [
    dict(fwd_vw=1, stage_vw=1), dict(fwd_vw=2, stage_vw=16), dict(fwd_vw=8, stage_vw=4),
    dict(fwd_vw=4, stage_vw=8, fwd_blocks=7, light_rows=16), dict(fwd_blocks=1, light_rows=40),
])
def test_launch_shapes_identical(pkg, oracle, shape):
    """Launch shapes the tuner may pick never change a bit of the result."""
    cnf = uniform_ksat(900, 3870, 3, seed=12)
    check_bit_exact(oracle, cnf, 16, 10, 2e-2, **shape)
    z = zipf_weighted(1200, 5000, seed=5)
    clamped = {k: (min(v, 8) if k in ("fwd_vw", "stage_vw") else v) for k, v in shape.items()}
    check_bit_exact(oracle, z, 8, 6, 2e-2, **clamped)


def test_larger_lr_chunked_steps(pkg, oracle):
    cnf = uniform_ksat(1000, 4300, 3, seed=2)
    check_bit_exact(oracle, cnf, 4, 40, 3e-2, chunk=7)


def test_weighted_zipf_with_heavy_variables(pkg, oracle):
    cnf = zipf_weighted(3000, 20000, seed=1)
    deg = np.bincount(np.abs(cnf.lits) - 1, minlength=cnf.n)
    assert deg.max() > 2048                      # several 1024-occurrence chunks
    got, _ = check_bit_exact(oracle, cnf, 1, 25, 1e-2)
    assert got["info"]["n_heavy"] > 0
    check_bit_exact(oracle, cnf, 4, 10, 1e-2)


def test_long_clauses_and_mixed_lengths(pkg, oracle):
    cnf = pigeonhole(40)                         # 40-literal pigeon clauses
    assert np.diff(cnf.off).max() == 40
    check_bit_exact(oracle, cnf, 2, 15, 5e-2)


def test_clauses_of_thousands_of_literals(pkg, oracle):
    """Clauses of 20000 and 5000 literals (hundreds of 32-literal leaves in
    the dyadic counter) among 3-literal clauses: trajectories bit for bit,
    and the tensor-core evaluation of the result."""
    rng = np.random.default_rng(41)
    n = 25000
    long_a = (rng.choice(n, size=20000, replace=False) + 1) * rng.choice([-1, 1], size=20000)
    long_b = (rng.choice(n, size=5000, replace=False) + 1) * rng.choice([-1, 1], size=5000)
    base = uniform_ksat(n, 3000, 3, seed=42)
    cl = base.clauses() + [[int(v) for v in long_a], [int(v) for v in long_b]]
    cnf = Cnf.from_clauses(n, cl, weights=rng.integers(1, 9, size=len(cl)))
    got, _ = check_bit_exact(oracle, cnf, 4, 6, 5e-2)
    with pkg.Solver.from_cnf(cnf, restarts=4, lr=5e-2) as s:
        s.step(6, want_loss=False)
        _, cost = s.step(0, want_loss=False)
        assert np.array_equal(s.evaluate_x("dense").cpu().numpy(), cost)
        s.check()
    assert np.array_equal(cost, got["cost_hist"][-1])


def test_planted_instance_reaches_zero_and_freezes(pkg, oracle):
    cnf = planted_ksat(40, 120, 3, seed=1)
    got, ref = check_bit_exact(oracle, cnf, 4, 400, 5e-2)
    assert (got["best_cost"] == 0).any()


def test_degenerate_clauses(pkg, oracle):
    cnf = Cnf.from_clauses(6, [[1, 1, 2], [-3, 3], [], [4, -5, 6, -4], [2], [-2], [5, 6, 1, 2]],
                           weights=[3, 1, 7, 2, 5, 5, 1])
    check_bit_exact(oracle, cnf, 2, 50, 5e-2)
    empty = Cnf(n=5, off=np.zeros(1, np.int64), lits=np.zeros(0, np.int32))
    got = gpu_trajectory(pkg, empty, 1, 3, 1e-2)
    assert got["cost_hist"].max() == 0


# --------------------------------------------------------- full sizes

def test_config1_batched_restarts(pkg, oracle):
    """Uniform 3-SAT n=5000, m=21500, B=256 restarts: 3 steps bit for bit."""
    cnf = uniform_ksat(5000, 21500, 3, seed=0)
    check_bit_exact(oracle, cnf, 256, 3, 1e-4)


def test_config2_weighted_zipf_full(pkg, oracle):
    """n=200000, m=1000000, Zipf(1.2), weights 1..1000, B=1: 6 steps."""
    cnf = zipf_weighted(200000, 1000000, seed=0)
    check_bit_exact(oracle, cnf, 1, 6, 1e-4)


_CORES = os.cpu_count() or 1


@pytest.mark.slow
def test_config1_batched_restarts_8_steps(pkg, oracle):
    """Uniform 3-SAT n=5000, m=21500, B=256: 8 steps of cost history, x,
    best cost and assignment bit for bit (the oracle's restarts split over
    the host's cores)."""
    cnf = uniform_ksat(5000, 21500, 3, seed=0)
    check_bit_exact(oracle, cnf, 256, 8, 1e-4, oracle_threads=_CORES)


@pytest.mark.slow
def test_config2_weighted_zipf_500_steps(pkg, oracle):
    """The weighted Zipf configuration for its full 500 steps: every int64
    weighted cost of x_0 .. x_500, the final x, best cost and assignment."""
    cnf = zipf_weighted(200000, 1000000, seed=0)
    got, ref = check_bit_exact(oracle, cnf, 1, 500, 1e-4)
    assert got["info"]["n_heavy"] > 0


@pytest.mark.slow
def test_config3_large_scale(pkg, oracle):
    """Uniform 3-SAT n=1e6, m=4.3e6, B=16: 5 steps from the seeded start,
    every cost, x and best assignment bit for bit (the oracle's 16 restarts
    run on the host's cores side by side)."""
    cnf = uniform_ksat(1000000, 4300000, 3, seed=0)
    check_bit_exact(oracle, cnf, 16, 5, 1e-4, oracle_threads=_CORES)


# ------------------------------------------------------------ evaluate

@pytest.mark.parametrize("nb", [1, 7, 33, 256])
def test_evaluate_sparse_exact(pkg, oracle, nb):
    import torch
    cnf = zipf_weighted(2000, 9000, seed=4)
    rng = np.random.default_rng(nb)
    a01 = rng.integers(0, 2, size=(nb, cnf.n)).astype(np.uint8)
    want = oracle.cost(cnf, a01)
    pm1 = torch.from_numpy((2 * a01.astype(np.int8) - 1).T.copy()).cuda()
    with pkg.Solver.from_cnf(cnf, restarts=1) as s:
        got = s.evaluate(pm1, backend="sparse").cpu().numpy()
    assert np.array_equal(got, want)


# ------------------------------------------------------------ autograd

@pytest.mark.parametrize("weighted", [False, True])
def test_autograd_loss_and_gradient(pkg, oracle, weighted):
    """Configuration 3a: 3-SAT n=1000, m=4300; the autograd.Function's loss
    and gradient against the oracle (FP64 within 1e-5, FP32-canon bit for
    bit) and the oracle's central differences."""
    import torch
    cnf = uniform_ksat(1000, 4300, 3, seed=0)
    if weighted:
        cnf = Cnf(n=cnf.n, off=cnf.off, lits=cnf.lits,
                  weights=(1 + np.arange(cnf.m) % 1000).astype(np.int64))
    B = 4
    x32 = oracle.init_x(cnf.n, B, 7)
    r64 = oracle.objective_f64(cnf, x32.astype(np.float64))
    r32 = oracle.objective_f32(cnf, x32)
    with pkg.Solver.from_cnf(cnf, restarts=B) as s:
        x = torch.from_numpy(x32).cuda().requires_grad_(True)
        loss = pkg.msat_loss(x, s)
        loss.sum().backward()
        g = x.grad.cpu().numpy()
        lv = loss.detach().cpu().numpy()
    assert np.allclose(lv, r64["loss"], rtol=1e-5, atol=0)
    tol = 1e-5 * np.abs(r64["grad"]).max(axis=0)
    assert np.all(np.abs(g.astype(np.float64) - r64["grad"]) <= tol[None, :])
    # element-wise relative error where the gradient is not tiny against
    # its restart's largest entry (there the scaled bound above governs)
    sel = np.abs(r64["grad"]) > 1e-3 * np.abs(r64["grad"]).max(axis=0)[None, :]
    assert sel.sum() > cnf.n * B // 2
    rel = np.abs(g.astype(np.float64) - r64["grad"])[sel] / np.abs(r64["grad"])[sel]
    assert rel.max() <= 1e-5
    assert np.array_equal(g, r32["grad"])
    # central differences of the FP64 objective at a few coordinates
    h = 1e-6
    x64 = x32.astype(np.float64)
    for i, b in [(3, 0), (500, 1), (999, 3), (123, 2)]:
        if abs(x64[i, b]) < 10 * h:
            continue
        xp = x64.copy(); xp[i, b] += h
        xm = x64.copy(); xm[i, b] -= h
        fd = (oracle.objective_f64(cnf, xp, want_grad=False)["loss"][b]
              - oracle.objective_f64(cnf, xm, want_grad=False)["loss"][b]) / (2 * h)
        assert abs(fd - g[i, b]) <= 1e-5 * np.abs(r64["grad"][:, b]).max() + 1e-9


def test_autograd_two_forwards_before_backward(pkg, oracle):
    """Two losses of one solver summed before a single backward: each
    input gets the gradient of its own forward, although the context holds
    the state of the latest forward only."""
    import torch
    cnf = uniform_ksat(300, 1290, 3, seed=8)
    B = 4
    xa, xb = oracle.init_x(cnf.n, B, 11), oracle.init_x(cnf.n, B, 12)
    with pkg.Solver.from_cnf(cnf, restarts=B) as s:
        ta = torch.from_numpy(xa).cuda().requires_grad_(True)
        tb = torch.from_numpy(xb).cuda().requires_grad_(True)
        la = pkg.msat_loss(ta, s)
        lb = pkg.msat_loss(tb, s)
        (la.sum() + 2.0 * lb.sum()).backward()
        ga, gb = ta.grad.cpu().numpy(), tb.grad.cpu().numpy()
    assert np.array_equal(ga, oracle.objective_f32(cnf, xa)["grad"])
    assert np.array_equal(gb, oracle.objective_f32(cnf, xb)["grad"] * np.float32(2.0))


def test_autograd_gradient_scaling(pkg, oracle):
    import torch
    cnf = uniform_ksat(200, 860, 3, seed=3)
    with pkg.Solver.from_cnf(cnf, restarts=2) as s:
        x = torch.from_numpy(oracle.init_x(cnf.n, 2, 3)).cuda().requires_grad_(True)
        loss = pkg.msat_loss(x, s)
        (3.0 * loss[0] + 0.5 * loss[1]).backward()
        g = x.grad.cpu().numpy()
    r = oracle.objective_f32(cnf, oracle.init_x(cnf.n, 2, 3))
    assert np.array_equal(g[:, 0], r["grad"][:, 0] * np.float32(3.0))
    assert np.array_equal(g[:, 1], r["grad"][:, 1] * np.float32(0.5))


# ---------------------------------------------------------- checkpoint

def test_checkpoint_resume_is_bit_identical(pkg, oracle):
    cnf = zipf_weighted(2000, 9000, seed=6)
    with pkg.Solver.from_cnf(cnf, restarts=4, lr=1e-2) as a:
        a.step(13, want_loss=False, want_cost=False)
        st = a.get_state()
        a.step(17, want_loss=False, want_cost=False)
        xa = a.x()
        ba = a.best()
    with pkg.Solver.from_cnf(cnf, restarts=4, lr=1e-2, seed_x=99) as b:
        b.set_state(st)
        b.step(17, want_loss=False, want_cost=False)
        xb = b.x()
        bb = b.best()
    assert np.array_equal(xa, xb)
    assert np.array_equal(ba[0], bb[0]) and np.array_equal(ba[1], bb[1])
    ref = oracle.solve(cnf, 4, 1, 30, mode=oracle.MODE_F32, lr=1e-2)
    assert np.array_equal(xb.astype(np.float64), ref["x_final"])


# ------------------------------------------------ loss normaliser ablation

@pytest.mark.parametrize("loss_norm", ["sum_unsat", "mean_all"])
@pytest.mark.parametrize("maker", ["ksat", "zipf"])
def test_loss_normaliser_trajectories(pkg, oracle, loss_norm, maker):
    """The ablation's other readings of the loss normaliser: the same
    bit-exact trajectory against the oracle as the default reading."""
    if maker == "ksat":
        cnf, B = uniform_ksat(300, 1290, 3, seed=12), 8
    else:
        cnf, B = zipf_weighted(900, 3600, seed=13), 4
    check_bit_exact(oracle, cnf, B, 120, 1e-2, loss_norm=loss_norm)


@pytest.mark.parametrize("maker", ["ksat", "php"])
def test_heuristic_gap_matches_oracle(pkg, oracle, maker):
    """The quick f_j > 0 reading of Sec. 4 against the exact test: counts
    of heuristic-unsat clauses and of disagreements per restart equal those
    derived from the oracle's FP32-canon f and unsat mask at the same x
    (PHP(40) has 40-literal clauses: several summation leaves)."""
    cnf = uniform_ksat(400, 1720, 3, seed=14) if maker == "ksat" else pigeonhole(40)
    with pkg.Solver.from_cnf(cnf, restarts=4, lr=1e-2) as s:
        s.step(30)
        x = s.x()
        hu, dg = s.heuristic_gap()
    r = oracle.objective_f32(cnf, x, want_f=True, want_grad=False)
    f, sat = r["f"], r["unsat"] == 0
    assert np.array_equal(hu, (~(f > 0)).sum(axis=0))
    assert np.array_equal(dg, ((f > 0) != sat).sum(axis=0))


# ---------------------------------------------- single-CTA small instances

@pytest.mark.parametrize("case", ["config1", "weighted_zipf", "php40_long", "b64", "planted_stop",
                                  "sum_unsat"])
def test_small_instance_kernel_matches_oracle(pkg, oracle, case):
    """The single-CTA kernel that runs every step of a small instance in one
    launch: bit-exact trajectories against the oracle (chunks of steps, so
    several launches continue one another), and its state continues on the
    per-pass kernels with the same bits."""
    kw = {}
    if case == "config1":
        cnf, B, S, lr, chunk = uniform_ksat(50, 215, 3, seed=0), 1, 300, 1e-2, 37
    elif case == "weighted_zipf":
        cnf, B, S, lr, chunk = zipf_weighted(700, 2800, seed=15), 4, 120, 1e-2, 50
    elif case == "php40_long":
        cnf, B, S, lr, chunk = pigeonhole(40), 1, 40, 1e-2, 13
    elif case == "b64":
        cnf, B, S, lr, chunk = uniform_ksat(80, 344, 3, seed=16), 64, 90, 3e-2, 30
    elif case == "planted_stop":
        cnf, B, S, lr, chunk = planted_ksat(60, 200, 3, seed=2), 16, 400, 5e-2, 100
    else:
        cnf, B, S, lr, chunk = uniform_ksat(200, 860, 3, seed=17), 8, 100, 1e-2, 25
        kw["loss_norm"] = "sum_unsat"
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=lr, **kw) as s:
        assert s.info()["small_kernel"] == 1
    check_bit_exact(oracle, cnf, B, S, lr, chunk=chunk, per_pass=False, **kw)
    # mixing the routes: small-kernel chunks, then per-pass steps
    ref = oracle.solve(cnf, B, 1, S + 7, mode=oracle.MODE_F32, lr=lr,
                       loss_norm=kw.get("loss_norm", "mean_unsat"))
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=lr, **kw) as s:
        s.step(S, want_loss=False, want_cost=False)
        s.step(7, want_loss=False, want_cost=False, per_pass=True)
        x = s.x()
        _, best = s.best()
    assert np.array_equal(x.astype(np.float64), ref["x_final"])
    assert np.array_equal(best, ref["best_cost"])


@pytest.mark.parametrize("per_pass", [True, False])
def test_best_step_is_first_minimum_of_cost_history(pkg, oracle, per_pass):
    """Steps to best: for each restart, the first step index at which the
    oracle's cost history reaches its minimum (strict improvement keeps the
    first), on the per-pass kernels and on the single-CTA route."""
    cnf = uniform_ksat(300, 1290, 3, seed=18)
    B, S, lr = 8, 150, 2e-2
    ref = oracle.solve(cnf, B, 1, S, mode=oracle.MODE_F32, lr=lr)
    want = np.argmin(ref["cost_hist"], axis=0)
    with pkg.Solver.from_cnf(cnf, restarts=B, lr=lr) as s:
        s.step(S, want_loss=False, want_cost=False, per_pass=per_pass)
        assert np.array_equal(s.best_step(), want)
        assert np.array_equal(s.best()[1], ref["best_cost"])
