"""Python face of the GB300 MaxSAT gradient engine.

Solver wraps one msat_ctx (Algorithm 1 of arXiv 2402.03640 on the GPU with B
restarts); MsatLoss exposes the relaxed objective of Sec. 4 as a
torch.autograd.Function whose forward and backward are the library's
kernels.  Host arrays are numpy; device arrays are torch CUDA tensors.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np

from . import native
from .native import check


def _p(a) -> Optional[ctypes.c_void_p]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _config(restarts=1, seed_x=1, lr=1e-4, beta1=0.9, beta2=0.999, eps=1e-8, f_mode="auto",
            heavy_deg=0, fwd_vw=0, stage_vw=0, fwd_blocks=0, light_rows=0, loss_norm="mean_unsat",
            row_order="auto"):
    lib = native.load()
    cfg = native.msat_config()
    check(lib.msat_config_default(ctypes.byref(cfg)))
    cfg.lr, cfg.beta1, cfg.beta2, cfg.eps = lr, beta1, beta2, eps
    cfg.restarts = int(restarts)
    cfg.seed_x = int(seed_x)
    cfg.f_mode = native.F_MODES[f_mode]
    cfg.heavy_deg = int(heavy_deg)
    cfg.fwd_vw, cfg.stage_vw = int(fwd_vw), int(stage_vw)
    cfg.fwd_blocks, cfg.light_rows = int(fwd_blocks), int(light_rows)
    cfg.loss_norm = native.LOSS_NORMS[loss_norm]
    cfg.row_order = {"auto": 0, "clause": 1, "block": 2}[row_order]
    return cfg


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Solver:
    """One CNF instance with B restarts resident on the GPU.

    n, off, lits, weights follow include/msat.h (DIMACS literals, int64
    offsets, optional int64 weights >= 1).  stream: a torch.cuda.Stream, a
    raw cudaStream_t integer, or None for torch's current stream.
    """

    def __init__(self, n: int, off, lits, weights=None, restarts: int = 1, seed_x: int = 1,
                 lr: float = 1e-4, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 stream=None, f_mode: str = "auto", heavy_deg: int = 0, fwd_vw: int = 0,
                 stage_vw: int = 0, fwd_blocks: int = 0, light_rows: int = 0,
                 loss_norm: str = "mean_unsat", tune: bool = False, row_order: str = "auto"):
        lib = native.load()
        self._lib = lib
        cfg = _config(restarts=restarts, seed_x=seed_x, lr=lr, beta1=beta1, beta2=beta2, eps=eps,
                      f_mode=f_mode, heavy_deg=heavy_deg, fwd_vw=fwd_vw, stage_vw=stage_vw,
                      fwd_blocks=fwd_blocks, light_rows=light_rows, loss_norm=loss_norm,
                      row_order=row_order)
        off = np.ascontiguousarray(off, dtype=np.int64)
        lits = np.ascontiguousarray(lits, dtype=np.int32)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.int64)
        self.n = int(n)
        self.m = int(off.shape[0] - 1)
        self.B = int(restarts)
        self._ctx = ctypes.c_void_p()
        st = _stream_handle(stream)
        sp = ctypes.c_void_p(st) if st else None
        self.tuning = None
        if tune:  # the launch shape from msat_autotune (results are the same bits)
            tuned = native.msat_config()
            ents = (native.msat_tune_entry * 16)()
            cnt = ctypes.c_int32()
            check(lib.msat_autotune(self.n, self.m, _p(off), _p(lits), _p(w), ctypes.byref(cfg), sp,
                                    10, ctypes.byref(tuned), ents, 16, ctypes.byref(cnt)))
            cfg = tuned
            self.tuning = {"fwd_vw": cfg.fwd_vw, "stage_vw": cfg.stage_vw, "light_rows": cfg.light_rows,
                           "timed": [(e.fwd_vw, e.stage_vw, e.light_rows, e.ms_per_step)
                                     for e in ents[:cnt.value]]}
        check(lib.msat_create(ctypes.byref(self._ctx), self.n, self.m, _p(off), _p(lits), _p(w),
                              ctypes.byref(cfg), sp))

    @classmethod
    def from_cnf(cls, cnf, **kw) -> "Solver":
        return cls(cnf.n, cnf.off, cnf.lits, cnf.weights, **kw)

    # -------------------------------------------------------------- life
    def close(self) -> None:
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.msat_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream) -> None:
        st = _stream_handle(stream)
        check(self._lib.msat_set_stream(self._ctx, ctypes.c_void_p(st) if st else None))

    # -------------------------------------------------------------- loop
    def step(self, n_steps: int, want_loss: bool = True, want_cost: bool = True, graph: bool = False,
             per_pass: bool = False) -> Tuple[Optional[np.ndarray], Optional[np.ndarray]]:
        """n_steps iterations of Algorithm 1 plus a final evaluation; returns
        (loss at the last updated x, cost of the final x), each [B] or None.
        graph: replay the steps from captured CUDA graphs; per_pass: keep a
        small instance on the per-pass kernels (both give the same bits)."""
        loss = np.empty(self.B, np.float32) if want_loss else None
        cost = np.empty(self.B, np.int64) if want_cost else None
        flags = (native.STEP_GRAPH if graph else 0) | (native.STEP_PER_PASS if per_pass else 0)
        check(self._lib.msat_step_ex(self._ctx, int(n_steps), flags, _p(loss), _p(cost)))
        return loss, cost

    def step_async(self, n_steps: int, final_eval: bool = True, graph: bool = False,
                   per_pass: bool = False) -> None:
        flags = ((0 if final_eval else native.STEP_NO_FINAL_EVAL) | (native.STEP_GRAPH if graph else 0)
                 | (native.STEP_PER_PASS if per_pass else 0))
        check(self._lib.msat_step_ex(self._ctx, int(n_steps), flags, None, None))

    def solve(self, max_steps: int, time_limit: float = float("inf"), chunk: int = 64,
              trace_cap: int = 4096) -> dict:
        """Algorithm 1 with a wall-clock limit (msat_solve): steps in chunks
        until a restart reaches cost 0, max_steps steps have run or
        time_limit seconds have passed.  Returns the steps taken, the seconds
        spent and the (seconds, best cost) trace after each chunk."""
        steps = ctypes.c_int64()
        elapsed = ctypes.c_double()
        tcost = np.empty(trace_cap, np.int64)
        ttime = np.empty(trace_cap, np.float64)
        tlen = ctypes.c_int32()
        limit = min(float(time_limit), 1e300)
        check(self._lib.msat_solve(self._ctx, int(max_steps), limit, int(chunk), ctypes.byref(steps),
                                   ctypes.byref(elapsed), _p(tcost), _p(ttime), int(trace_cap),
                                   ctypes.byref(tlen)))
        k = tlen.value
        return {"steps": steps.value, "elapsed_s": elapsed.value,
                "trace_time_s": ttime[:k].copy(), "trace_best_cost": tcost[:k].copy()}

    def profile(self, on: bool = True) -> None:
        """Bracket every kernel of this context with CUDA events."""
        check(self._lib.msat_profile_enable(self._ctx, int(bool(on))))

    def profile_read(self, reset: bool = True) -> dict:
        """{kind: (launches, total ms)} for kinds forward, backward, evaluate, other."""
        p = native.msat_profile()
        check(self._lib.msat_profile_read(self._ctx, ctypes.byref(p), int(bool(reset))))
        return {k: (int(p.launches[i]), float(p.ms[i])) for i, k in enumerate(native.PROFILE_KINDS)}

    def best(self) -> Tuple[np.ndarray, np.ndarray]:
        a = np.empty((self.B, self.n), np.uint8)
        c = np.empty(self.B, np.int64)
        check(self._lib.msat_best(self._ctx, _p(a), _p(c)))
        return a, c

    def x(self) -> np.ndarray:
        out = np.empty((self.n, self.B), np.float32)
        check(self._lib.msat_get_x(self._ctx, _p(out)))
        return out

    def info(self) -> dict:
        inf = native.msat_info()
        check(self._lib.msat_get_info(self._ctx, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def get_state(self) -> dict:
        nB = (self.n, self.B)
        st = dict(x=np.empty(nB, np.float32), mom=np.empty(nB, np.float32),
                  vel=np.empty(nB, np.float32), best_cost=np.empty(self.B, np.int64),
                  best_assign=np.empty(nB, np.uint8), steps_done=np.zeros(1, np.int64),
                  adam_pow=np.zeros(2, np.float64))
        check(self._lib.msat_get_state(self._ctx, _p(st["x"]), _p(st["mom"]), _p(st["vel"]),
                                       _p(st["best_cost"]), _p(st["best_assign"]),
                                       _p(st["steps_done"]), _p(st["adam_pow"])))
        return st

    def set_state(self, st: dict) -> None:
        arr = {k: np.ascontiguousarray(v) for k, v in st.items()}
        check(self._lib.msat_set_state(self._ctx, _p(arr["x"].astype(np.float32, copy=False)),
                                       _p(arr["mom"].astype(np.float32, copy=False)),
                                       _p(arr["vel"].astype(np.float32, copy=False)),
                                       _p(arr["best_cost"].astype(np.int64, copy=False)),
                                       _p(arr["best_assign"].astype(np.uint8, copy=False)),
                                       int(arr["steps_done"].reshape(-1)[0]),
                                       _p(arr["adam_pow"].astype(np.float64, copy=False))))

    # -------------------------------------------------------- evaluation
    def evaluate(self, assign_pm1, backend: str = "sparse"):
        """Exact cost of a batch of +-1 assignments (torch int8 CUDA [n][nb]);
        returns a torch int64 CUDA tensor [nb]."""
        import torch
        a = assign_pm1
        if a.dtype != torch.int8 or not a.is_cuda or a.dim() != 2 or a.shape[0] != self.n:
            raise ValueError("assign_pm1 must be a CUDA int8 tensor of shape [n, nb]")
        a = a.contiguous()
        nb = int(a.shape[1])
        out = torch.empty(nb, dtype=torch.int64, device=a.device)
        be = {"sparse": native.BACKEND_SPARSE, "dense": native.BACKEND_DENSE}[backend]
        check(self._lib.msat_evaluate(self._ctx, _p(a), nb, _p(out), be))
        return out

    def best_step(self) -> np.ndarray:
        """Per restart, the optimizer steps taken before the x that gave the
        best cost (0: the random start)."""
        out = np.empty(self.B, np.int64)
        check(self._lib.msat_best_step(self._ctx, _p(out)))
        return out

    def heuristic_gap(self) -> Tuple[np.ndarray, np.ndarray]:
        """(clauses the quick f_j > 0 reading calls unsat, clauses on which it
        disagrees with the exact test), each int64 [B], at the current x."""
        hu = np.empty(self.B, np.int64)
        dg = np.empty(self.B, np.int64)
        check(self._lib.msat_heuristic_gap(self._ctx, _p(hu), _p(dg)))
        return hu, dg

    def evaluate_x(self, backend: str = "sparse", out=None):
        """Exact cost of the current x rounded to +-1, as a torch int64 CUDA
        tensor [B] (written into out when given)."""
        import torch
        if out is None:
            out = torch.empty(self.B, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
        be = {"sparse": native.BACKEND_SPARSE, "dense": native.BACKEND_DENSE}[backend]
        check(self._lib.msat_evaluate_x(self._ctx, be, _p(out)))
        return out

    def check(self) -> None:
        """Raise if a bounded device wait gave up since the last check."""
        check(self._lib.msat_check(self._ctx))

    # ---------------------------------------------------- differentiable
    def forward(self, x):
        import torch
        x = x.contiguous()
        if x.dtype != torch.float32 or not x.is_cuda or tuple(x.shape) != (self.n, self.B):
            raise ValueError("x must be a CUDA float32 tensor of shape [n, B]")
        loss = torch.empty(self.B, dtype=torch.float32, device=x.device)
        cost = torch.empty(self.B, dtype=torch.int64, device=x.device)
        check(self._lib.msat_forward(self._ctx, _p(x), _p(loss), _p(cost)))
        # the context holds the state of one forward (tanh(x), the unsat
        # mask, 2/N): count forwards so a backward can tell whose it is
        self.probe_gen = getattr(self, "probe_gen", 0) + 1
        return loss, cost

    def backward(self, gscale=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        grad = torch.empty((self.n, self.B), dtype=torch.float32, device=dev)
        g = None if gscale is None else gscale.contiguous().to(torch.float32)
        check(self._lib.msat_backward(self._ctx, _p(g), _p(grad)))
        return grad


class Server:
    """Continuous-batching request loop (msat_server_*): submit CNF instances
    at any time, poll or wait for their results."""

    def __init__(self, restarts: int = 8, hbm_budget: int = 0, max_slots: int = 0, chunk: int = 0,
                 lr: float = 1e-4, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 batch_mlits: int = 0):
        lib = native.load()
        self._lib = lib
        cfg = native.msat_server_config()
        check(lib.msat_server_config_default(ctypes.byref(cfg)))
        cfg.restarts = int(restarts)
        cfg.hbm_budget = int(hbm_budget)
        if max_slots:
            cfg.max_slots = int(max_slots)
        if chunk:
            cfg.chunk = int(chunk)
        cfg.batch_mlits = int(batch_mlits)
        cfg.lr, cfg.beta1, cfg.beta2, cfg.eps = lr, beta1, beta2, eps
        self.B = int(restarts)
        self._srv = ctypes.c_void_p()
        check(lib.msat_server_create(ctypes.byref(self._srv), ctypes.byref(cfg)))
        self._n = {}

    def submit(self, cnf, steps: int, seed_x: int = 1) -> int:
        off = np.ascontiguousarray(cnf.off, dtype=np.int64)
        lits = np.ascontiguousarray(cnf.lits, dtype=np.int32)
        w = None if cnf.weights is None else np.ascontiguousarray(cnf.weights, dtype=np.int64)
        req = native.msat_request(n_vars=int(cnf.n), steps=int(steps), n_clauses=int(off.shape[0] - 1),
                                  clause_off=off.ctypes.data, lits=lits.ctypes.data if lits.size else None,
                                  weights=None if w is None else w.ctypes.data, seed_x=int(seed_x))
        t = ctypes.c_uint64()
        check(self._lib.msat_submit(self._srv, ctypes.byref(req), ctypes.byref(t)))
        self._n[t.value] = int(cnf.n)
        return t.value

    def _result(self, rc, res, best, assign, ticket):
        if rc == native.MSAT_EAGAIN:
            return None
        self._n.pop(ticket, None)
        check(rc)
        out = {f: getattr(res, f) for f, _ in res._fields_}
        out["best_costs"] = best
        out["assignment"] = assign
        return out

    def poll(self, ticket: int):
        """The result dict once done, None while queued or running."""
        res = native.msat_result()
        best = np.empty(self.B, np.int64)
        assign = np.empty(self._n.get(ticket, 1), np.uint8)
        rc = self._lib.msat_poll(self._srv, ticket, ctypes.byref(res), _p(best), _p(assign))
        return self._result(rc, res, best, assign, ticket)

    def wait(self, ticket: int, timeout_s: float = 600.0):
        res = native.msat_result()
        best = np.empty(self.B, np.int64)
        assign = np.empty(self._n.get(ticket, 1), np.uint8)
        rc = self._lib.msat_wait(self._srv, ticket, float(timeout_s), ctypes.byref(res), _p(best), _p(assign))
        return self._result(rc, res, best, assign, ticket)

    def cancel(self, ticket: int) -> None:
        check(self._lib.msat_cancel(self._srv, ticket))
        self._n.pop(ticket, None)

    def stats(self) -> dict:
        st = native.msat_server_stats()
        check(self._lib.msat_server_get_stats(self._srv, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self) -> None:
        if getattr(self, "_srv", None) is not None and self._srv.value:
            self._lib.msat_server_destroy(self._srv)
            self._srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _make_autograd():
    import torch

    class MsatLoss(torch.autograd.Function):
        """loss[b] = sum_{unsat j} w_j f_j^2 / sum_{unsat j} w_j for restart b,
        f = tanh(x) . W (Sec. 4); backward through the library's variable-pass
        kernel (the unsat mask is treated as a constant)."""

        @staticmethod
        def forward(ctx, x, solver):
            loss, _ = solver.forward(x)
            ctx.solver = solver
            ctx.gen = solver.probe_gen
            ctx.save_for_backward(x)
            return loss

        @staticmethod
        def backward(ctx, gout):
            solver = ctx.solver
            if solver.probe_gen != ctx.gen:
                # another forward ran on this solver since ours (for example
                # two losses summed before one backward): the context holds
                # its state, so evaluate this call's x again first
                (x,) = ctx.saved_tensors
                solver.forward(x)
            grad = solver.backward(gout)
            return grad, None

    return MsatLoss


_MsatLoss = None


def msat_loss(x, solver: Solver):
    """Differentiable relaxed objective: MsatLoss.apply(x, solver)."""
    global _MsatLoss
    if _MsatLoss is None:
        _MsatLoss = _make_autograd()
    return _MsatLoss.apply(x, solver)


def dense_mma_rate(n_assign: int = 256, iters: int = 4096) -> float:
    """TFLOP/s of the dense backend's MMA instruction shape issued back to
    back on every SM with operands resident in shared memory (msat_dense_mma_rate)."""
    out = ctypes.c_double(0.0)
    native.check(native.load().msat_dense_mma_rate(int(n_assign), int(iters), ctypes.byref(out)))
    return out.value
