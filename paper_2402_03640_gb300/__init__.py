"""GB300-native engine for the torchmSAT objective (arXiv 2402.03640).

The solving loop of Algorithm 1 -- forward over the clause CSR, exact unsat
cost, masked MSE loss, backward over the transposed CSR, Adam -- runs in
hand-written CUDA kernels for sm_103a behind the C ABI in include/msat.h.
This package is the thin binding: build (nvcc), native (ctypes), solver.
"""
from .native import MsatError, library_path, load
from .solver import Server, Solver, dense_mma_rate, msat_loss

__all__ = ["MsatError", "Server", "Solver", "dense_mma_rate", "library_path", "load", "msat_loss"]
