"""Seeded synthetic MaxSAT inputs shared by the oracle tests and the GPU path.
Holds none of the method's arithmetic."""
from .cnf import (ALPHA_K, Cnf, Request, ordering, partial_maxsat, pigeonhole, planted_ksat,
                  random_partial, serving_stream, splitmix64, uniform_ksat, zipf_weighted)

__all__ = ["ALPHA_K", "Cnf", "Request", "ordering", "partial_maxsat", "pigeonhole", "planted_ksat",
           "random_partial", "serving_stream", "splitmix64", "uniform_ksat", "zipf_weighted"]
