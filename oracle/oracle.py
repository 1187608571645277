"""Python access to the CPU oracle (msat_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU baseline / reference arm use this module.  The GPU library never imports
it, and it imports nothing from the GPU library.

Every function follows the paper (arXiv 2402.03640): section 4 for the
objective f = tanh(x) . W, the de-relaxation x' = [x > 0], the exact unsat
test and the masked MSE loss; Algorithm 1 for the solving loop; section 5 for
Adam.  The arithmetic modes are described in msat_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msat_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_F64 = 0
MODE_F32 = 1

# PyTorch's Adam defaults; the paper fixes only the learning rate (Sec. 5).
ADAM_DEFAULTS = dict(lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no contraction of a*b+c)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.orc_splitmix64.argtypes = [u64, u64]
        lib.orc_splitmix64.restype = u64
        lib.orc_init_x.argtypes = [i32, i32, u64, P]
        lib.orc_tanh32.argtypes = [ctypes.c_float]
        lib.orc_tanh32.restype = ctypes.c_float
        lib.orc_canon_sum.argtypes = [P, i64]
        lib.orc_canon_sum.restype = ctypes.c_float
        lib.orc_cost.argtypes = [i32, i64, P, P, P, i32, P, P]
        lib.orc_objective_f64.argtypes = [i32, i64, P, P, P, i32, P, P, P, P, P, P]
        lib.orc_objective_f32.argtypes = [i32, i64, P, P, P, i32, P, P, P, P, P, P]
        lib.orc_step32.argtypes = [i32, i64, P, P, P, i32, P, P, P, i64, f64, f64, f64, f64,
                                   i32, P, P, P, P, P]
        lib.orc_solve.argtypes = [i32, i64, P, P, P, i32, u64, f64, f64, f64, f64, i32, i32,
                                  P, P, P, P, P]
        lib.orc_solve_from.argtypes = [i32, i64, P, P, P, i32, i32, u64, f64, f64, f64, f64, i32, i32,
                                       P, P, P, P, P]
        lib.orc_set_loss_norm.argtypes = [i32]
        for name in ("orc_init_x", "orc_cost", "orc_objective_f64", "orc_objective_f32",
                     "orc_step32", "orc_solve", "orc_solve_from", "orc_set_loss_norm"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _cnf_arrays(cnf):
    off = np.ascontiguousarray(cnf.off, dtype=np.int64)
    lits = np.ascontiguousarray(cnf.lits, dtype=np.int32)
    w = None if cnf.weights is None else np.ascontiguousarray(cnf.weights, dtype=np.int64)
    return off, lits, w


LOSS_NORMS = {"mean_unsat": 0, "sum_unsat": 1, "mean_all": 2}


class _loss_norm:
    """Select the loss normaliser of the oracle for one call (Sec. 4 reading:
    mean over the unsat clauses; the sum and the mean over all clauses are the
    ablation's alternatives), restoring the default afterwards."""

    def __init__(self, name):
        self.mode = LOSS_NORMS[name]

    def __enter__(self):
        _check(_load().orc_set_loss_norm(self.mode), "set_loss_norm")

    def __exit__(self, *exc):
        _load().orc_set_loss_norm(0)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def splitmix64(seed: int, c: int) -> int:
    return int(_load().orc_splitmix64(seed, c))


def init_x(n: int, B: int, seed: int) -> np.ndarray:
    """Random start of Algorithm 1: float32 [n][B] on the grid of [-1, 1)."""
    x = np.empty((n, B), dtype=np.float32)
    _check(_load().orc_init_x(n, B, seed, _p(x)), "init_x")
    return x


def tanh32(a: float) -> float:
    return float(_load().orc_tanh32(a))


def tanh32_array(a: np.ndarray) -> np.ndarray:
    f = _load().orc_tanh32
    return np.array([f(float(v)) for v in np.asarray(a, dtype=np.float32).ravel()],
                    dtype=np.float32).reshape(np.shape(a))


def canon_sum(a: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    return float(_load().orc_canon_sum(_p(a), a.size))


def cost(cnf, assign01: np.ndarray) -> np.ndarray:
    """Exact (weighted) number of clauses with no true literal; assign01 is [B][n]."""
    a = np.ascontiguousarray(assign01, dtype=np.uint8)
    if a.ndim == 1:
        a = a[None, :]
    B = a.shape[0]
    out = np.empty(B, dtype=np.int64)
    off, lits, w = _cnf_arrays(cnf)
    _check(_load().orc_cost(cnf.n, cnf.m, _p(off), _p(lits), _p(w), B, _p(a), _p(out)), "cost")
    return out


def objective_f64(cnf, x: np.ndarray, want_f=False, want_grad=True, loss_norm="mean_unsat"):
    """f, unsat mask, cost, loss and gradient at x (double, [n][B]); Sec. 4."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n, B = x.shape
    f = np.empty((cnf.m, B), dtype=np.float64) if want_f else None
    u = np.empty((cnf.m, B), dtype=np.uint8) if want_f else None
    c = np.empty(B, dtype=np.int64)
    loss = np.empty(B, dtype=np.float64)
    g = np.empty((n, B), dtype=np.float64) if want_grad else None
    off, lits, w = _cnf_arrays(cnf)
    with _loss_norm(loss_norm):
        _check(_load().orc_objective_f64(cnf.n, cnf.m, _p(off), _p(lits), _p(w), B, _p(x), _p(f),
                                         _p(u), _p(c), _p(loss), _p(g)), "objective_f64")
    return dict(f=f, unsat=u, cost=c, loss=loss, grad=g)


def objective_f32(cnf, x: np.ndarray, want_f=False, want_grad=True, loss_norm="mean_unsat"):
    """Same as objective_f64 in the FP32-canon arithmetic."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x[:, None]
    n, B = x.shape
    f = np.empty((cnf.m, B), dtype=np.float32) if want_f else None
    u = np.empty((cnf.m, B), dtype=np.uint8) if want_f else None
    c = np.empty(B, dtype=np.int64)
    loss = np.empty(B, dtype=np.float64)
    g = np.empty((n, B), dtype=np.float32) if want_grad else None
    off, lits, w = _cnf_arrays(cnf)
    with _loss_norm(loss_norm):
        _check(_load().orc_objective_f32(cnf.n, cnf.m, _p(off), _p(lits), _p(w), B, _p(x), _p(f),
                                         _p(u), _p(c), _p(loss), _p(g)), "objective_f32")
    return dict(f=f, unsat=u, cost=c, loss=loss, grad=g)


def step32(cnf, x, mom, vel, steps_done, best_cost, best_assign=None, update=True,
           lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8, loss_norm="mean_unsat"):
    """One iteration of Algorithm 1 in FP32-canon arithmetic, in place on
    float32 [n][B] arrays x, mom, vel and on best_cost [B] / best_assign [B][n].
    Returns (cost [B], loss [B], grad [n][B] or None)."""
    n, B = x.shape
    for a in (x, mom, vel):
        assert a.dtype == np.float32 and a.flags.c_contiguous and a.shape == (n, B)
    assert best_cost.dtype == np.int64 and best_cost.shape == (B,)
    if best_assign is not None:
        assert best_assign.dtype == np.uint8 and best_assign.shape == (B, n)
    c = np.empty(B, dtype=np.int64)
    loss = np.empty(B, dtype=np.float64)
    g = np.empty((n, B), dtype=np.float32) if update else None
    off, lits, w = _cnf_arrays(cnf)
    with _loss_norm(loss_norm):
        _check(_load().orc_step32(cnf.n, cnf.m, _p(off), _p(lits), _p(w), B, _p(x), _p(mom),
                                  _p(vel), int(steps_done), lr, beta1, beta2, eps, int(bool(update)),
                                  _p(best_cost), _p(best_assign), _p(c), _p(loss), _p(g)), "step32")
    return c, loss, g


def solve(cnf, B: int, seed_x: int, steps: int, mode: int = MODE_F32, lr=1e-4, beta1=0.9,
          beta2=0.999, eps=1e-8, want_hist=True, want_x=True, loss_norm="mean_unsat", threads=1):
    """Algorithm 1 with `steps` optimizer steps (in place of the time limit T)
    and a final evaluation of x_steps.  Returns a dict of numpy arrays.
    threads > 1 splits the independent restarts into groups solved side by
    side (orc_solve_from on each group; the C code runs without the
    interpreter lock) and joins their columns: the same arrays."""
    if threads > 1 and B > 1:
        return _solve_split(cnf, B, seed_x, steps, mode, lr, beta1, beta2, eps, want_hist, want_x,
                            loss_norm, threads)
    n = cnf.n
    ch = np.empty((steps + 1, B), dtype=np.int64) if want_hist else None
    lh = np.empty((steps, B), dtype=np.float64) if want_hist else None
    best = np.empty(B, dtype=np.int64)
    ba = np.zeros((B, n), dtype=np.uint8)
    xf = np.empty((n, B), dtype=np.float64) if want_x else None
    off, lits, w = _cnf_arrays(cnf)
    with _loss_norm(loss_norm):
        _check(_load().orc_solve(n, cnf.m, _p(off), _p(lits), _p(w), B, seed_x, lr, beta1, beta2,
                                 eps, steps, mode, _p(ch), _p(lh), _p(best), _p(ba), _p(xf)), "solve")
    return dict(cost_hist=ch, loss_hist=lh, best_cost=best, best_assign=ba, x_final=xf)


def _solve_part(cnf, b0, B, seed_x, steps, mode, lr, beta1, beta2, eps, want_hist, want_x):
    n = cnf.n
    ch = np.empty((steps + 1, B), dtype=np.int64) if want_hist else None
    lh = np.empty((steps, B), dtype=np.float64) if want_hist else None
    best = np.empty(B, dtype=np.int64)
    ba = np.zeros((B, n), dtype=np.uint8)
    xf = np.empty((n, B), dtype=np.float64) if want_x else None
    off, lits, w = _cnf_arrays(cnf)
    _check(_load().orc_solve_from(n, cnf.m, _p(off), _p(lits), _p(w), B, b0, seed_x, lr, beta1, beta2,
                                  eps, steps, mode, _p(ch), _p(lh), _p(best), _p(ba), _p(xf)), "solve_from")
    return dict(cost_hist=ch, loss_hist=lh, best_cost=best, best_assign=ba, x_final=xf)


def _solve_split(cnf, B, seed_x, steps, mode, lr, beta1, beta2, eps, want_hist, want_x, loss_norm,
                 threads):
    from concurrent.futures import ThreadPoolExecutor
    groups = min(threads, B)
    bounds = [B * g // groups for g in range(groups + 1)]
    with _loss_norm(loss_norm), ThreadPoolExecutor(max_workers=groups) as ex:
        parts = list(ex.map(lambda g: _solve_part(cnf, bounds[g], bounds[g + 1] - bounds[g], seed_x, steps,
                                                  mode, lr, beta1, beta2, eps, want_hist, want_x),
                            range(groups)))
    def cat(key, axis):
        if parts[0][key] is None:
            return None
        return np.concatenate([p[key] for p in parts], axis=axis)
    return dict(cost_hist=cat("cost_hist", 1), loss_hist=cat("loss_hist", 1), best_cost=cat("best_cost", 0),
                best_assign=cat("best_assign", 0), x_final=cat("x_final", 1))
