"""Seeded synthetic MaxSAT instances.

This module holds the input generators that both the CPU oracle and the GPU
library are fed from.  It contains none of the method's arithmetic: it only
draws clause sets (and request streams) from counter-based SplitMix64
streams, so the same seed gives the same instance on any machine.

Instance families (all clause lists use DIMACS literals: +(i+1) for x_i,
-(i+1) for not x_i):

* uniform_ksat     -- uniform random k-SAT: k distinct variables per clause,
                      drawn uniformly by rejection, each negated with p = 1/2.
* zipf_weighted    -- skewed weighted MaxSAT: clause length 2 + Geom(1/3)
                      truncated to <= 20 by rejection (mean about 4), variables
                      Zipf(s) over ranks mapped through a seeded permutation
                      (distinct within a clause by rejection), signs
                      Bernoulli(1/2), weights uniform on 1..1000.
* planted_ksat     -- random k-SAT conditioned on a hidden assignment
                      satisfying every clause (optimum cost 0).
* pigeonhole       -- PHP with h+1 pigeons and h holes (optimum cost 1).
* ordering         -- the ordering ("greater-than") principle on s+1
                      elements (optimum cost 1).
* serving_stream   -- a stream of random k-SAT requests with Poisson
                      arrivals for the serving loop.
* partial_maxsat   -- hard and soft clauses as one weighted instance: each
                      hard clause weighs 1 + the total soft weight.
* random_partial   -- planted k-SAT hard clauses plus weighted soft unit
                      clauses.

The two structured families follow the principles' mathematical definitions;
their variable and clause counts agree with the paper's Table 2 (PHP and GT
columns).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class Cnf:
    """A clause set in CSR form.

    n        number of variables
    off      int64 [m+1] clause offsets into lits
    lits     int32 [nnz] DIMACS literals
    weights  int64 [m] clause weights >= 1, or None (all 1)
    """

    n: int
    off: np.ndarray
    lits: np.ndarray
    weights: Optional[np.ndarray] = None
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.off[-1])

    def clauses(self) -> List[List[int]]:
        return [self.lits[self.off[j]:self.off[j + 1]].tolist() for j in range(self.m)]

    @staticmethod
    def from_clauses(n: int, clauses, weights=None, name: str = "") -> "Cnf":
        lens = np.array([len(c) for c in clauses], dtype=np.int64)
        off = np.zeros(len(clauses) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        lits = np.array([l for c in clauses for l in c], dtype=np.int32)
        w = None if weights is None else np.asarray(weights, dtype=np.int64)
        return Cnf(n=n, off=off, lits=lits, weights=w, name=name)


# ---------------------------------------------------------------- streams

def splitmix64(seed: int, counters) -> np.ndarray:
    """Output number c (0-based) of the SplitMix64 stream seeded with `seed`
    (Steele, Lea, Flood 2014), vectorised over an array of counters."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _substream(seed: int, stream_id: int) -> int:
    return int(splitmix64(seed, np.array([stream_id], dtype=np.uint64))[0])


def _below(u: np.ndarray, n) -> np.ndarray:
    """Map 64-bit draws to integers in [0, n) with the high 32 bits (multiply-shift)."""
    hi = (u >> np.uint64(32)).astype(np.uint64)
    return ((hi * np.asarray(n, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def _unit(u: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


_MAX_TRIES = 4096


def _distinct_rows(draw, rows: int, k: int) -> np.ndarray:
    """Fill a [rows][k] array column by column; an entry equal to an earlier
    entry of its row is redrawn with the next attempt number (rejection).
    draw(row_idx, pos, attempt) returns int64 candidates."""
    V = np.empty((rows, k), dtype=np.int64)
    all_rows = np.arange(rows, dtype=np.int64)
    for p in range(k):
        todo = all_rows
        attempt = 0
        while todo.size:
            if attempt >= _MAX_TRIES:
                raise RuntimeError("rejection sampling did not converge")
            cand = draw(todo, p, attempt)
            V[todo, p] = cand
            if p == 0:
                break
            clash = np.zeros(todo.size, dtype=bool)
            for q in range(p):
                clash |= V[todo, q] == cand
            todo = todo[clash]
            attempt += 1
    return V


# ---------------------------------------------------------------- families

def uniform_ksat(n: int, m: int, k: int = 3, seed: int = 0, name: str = "") -> Cnf:
    """Uniform random k-SAT: each clause has k distinct variables drawn
    uniformly (rejection), each negated with probability 1/2."""
    if k > n:
        raise ValueError("k distinct variables need k <= n")
    s_var = _substream(seed, 1)
    s_sgn = _substream(seed, 2)

    def draw(rows, p, attempt):
        ctr = ((rows.astype(np.uint64) * np.uint64(k) + np.uint64(p)) << np.uint64(12)) \
            + np.uint64(attempt)
        return _below(splitmix64(s_var, ctr), n)

    V = _distinct_rows(draw, m, k)
    sg = splitmix64(s_sgn, np.arange(m * k, dtype=np.uint64)) & np.uint64(1)
    lits = (V.reshape(-1) + 1) * np.where(sg.astype(bool), -1, 1)
    off = np.arange(m + 1, dtype=np.int64) * k
    return Cnf(n=n, off=off, lits=lits.astype(np.int32), weights=None,
               name=name or f"uniform{k}sat_n{n}_m{m}_s{seed}")


def planted_ksat(n: int, m: int, k: int = 3, seed: int = 0) -> Cnf:
    """Random k-SAT conditioned on a hidden assignment satisfying every clause."""
    s_hide = _substream(seed, 7)
    hidden = (splitmix64(s_hide, np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(bool)
    out = []
    attempt = 0
    need = m
    while need > 0:
        cand = uniform_ksat(n, 2 * need + 16, k, seed=seed * 1000003 + attempt)
        C = cand.lits.reshape(-1, k)
        v = np.abs(C) - 1
        val = hidden[v] ^ (C < 0)          # literal true under the hidden assignment
        ok = val.any(axis=1)
        out.append(C[ok][:need])
        need -= min(need, int(ok.sum()))
        attempt += 1
    L = np.concatenate(out)[:m]
    off = np.arange(m + 1, dtype=np.int64) * k
    return Cnf(n=n, off=off, lits=L.reshape(-1).astype(np.int32), weights=None,
               name=f"planted{k}sat_n{n}_m{m}_s{seed}")


def zipf_weighted(n: int, m: int, s: float = 1.2, seed: int = 0, p_geom: float = 1.0 / 3.0,
                  min_len: int = 2, max_len: int = 20, w_max: int = 1000) -> Cnf:
    """Skewed weighted MaxSAT: clause length min_len + Geom(p) truncated to
    <= max_len by rejection; variables Zipf(s) over ranks 1..n mapped by a
    seeded permutation, distinct within a clause by rejection; signs
    Bernoulli(1/2); weights uniform on 1..w_max."""
    s_len, s_var, s_sgn, s_w, s_perm = (_substream(seed, i) for i in (11, 12, 13, 14, 15))
    gmax = max_len - min_len
    thresh = np.uint64(int(p_geom * 2.0 ** 64) & 0xFFFFFFFFFFFFFFFF)
    # lengths: number of failures before the first success, trials from a counter stream
    G = np.full(m, -1, dtype=np.int64)
    todo = np.arange(m, dtype=np.int64)
    attempt = 0
    while todo.size:
        if attempt >= _MAX_TRIES:
            raise RuntimeError("length rejection did not converge")
        base = (todo.astype(np.uint64) << np.uint64(16)) + np.uint64(attempt * 32)
        trials = splitmix64(s_len, base[:, None] + np.arange(gmax + 1, dtype=np.uint64)[None, :])
        succ = trials < thresh
        has = succ.any(axis=1)
        first = np.argmax(succ, axis=1)
        G[todo[has]] = first[has]
        todo = todo[~has]
        attempt += 1
    lens = (min_len + G).astype(np.int64)
    off = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    nnz = int(off[-1])
    # Zipf ranks via the cumulative distribution
    ranks = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-s))
    cdf /= cdf[-1]
    perm = np.argsort(splitmix64(s_perm, np.arange(n, dtype=np.uint64)), kind="stable")
    clause_of = np.repeat(np.arange(m, dtype=np.int64), lens)
    pos = np.arange(nnz, dtype=np.int64) - off[clause_of]
    V = np.empty(nnz, dtype=np.int64)
    todo = np.arange(nnz, dtype=np.int64)
    # fill position by position so rejection only compares with earlier positions
    for p in range(max_len):
        sel = np.nonzero(pos == p)[0]
        attempt = 0
        cur = sel
        while cur.size:
            if attempt >= _MAX_TRIES:
                raise RuntimeError("variable rejection did not converge")
            ctr = (cur.astype(np.uint64) << np.uint64(12)) + np.uint64(attempt)
            u = _unit(splitmix64(s_var, ctr))
            r = np.searchsorted(cdf, u, side="right")
            r = np.minimum(r, n - 1)
            V[cur] = perm[r]
            clash = np.zeros(cur.size, dtype=bool)
            for q in range(1, p + 1):
                clash |= V[cur - q] == V[cur]
            cur = cur[clash]
            attempt += 1
    sg = splitmix64(s_sgn, np.arange(nnz, dtype=np.uint64)) & np.uint64(1)
    lits = (V + 1) * np.where(sg.astype(bool), -1, 1)
    w = 1 + _below(splitmix64(s_w, np.arange(m, dtype=np.uint64)), w_max)
    return Cnf(n=n, off=off, lits=lits.astype(np.int32), weights=w.astype(np.int64),
               name=f"zipf{s}_n{n}_m{m}_s{seed}")


def pigeonhole(h: int) -> Cnf:
    """h+1 pigeons, h holes.  p(i,k) = pigeon i sits in hole k.  Each pigeon
    sits somewhere; no hole holds two pigeons.  Unsatisfiable; dropping one
    pigeon clause leaves it satisfiable, so the optimum cost is 1."""
    def p(i, k):
        return i * h + k + 1
    clauses = [[p(i, k) for k in range(h)] for i in range(h + 1)]
    for k in range(h):
        for i in range(h + 1):
            for i2 in range(i + 1, h + 1):
                clauses.append([-p(i, k), -p(i2, k)])
    return Cnf.from_clauses(h * (h + 1), clauses, name=f"php{h}")


def ordering(size: int) -> Cnf:
    """Ordering principle on N = size+1 elements.  x(a,b) = "a precedes b"
    for a != b.  Antisymmetry, transitivity, and "every element has a
    predecessor" cannot all hold on a finite set; the optimum cost is 1."""
    N = size + 1
    idx = {}
    for a in range(N):
        for b in range(N):
            if a != b:
                idx[(a, b)] = len(idx) + 1
    clauses = []
    for a in range(N):
        for b in range(a + 1, N):
            clauses.append([-idx[(a, b)], -idx[(b, a)]])
    for a in range(N):
        for b in range(N):
            for c in range(N):
                if len({a, b, c}) == 3:
                    clauses.append([-idx[(a, b)], -idx[(b, c)], idx[(a, c)]])
    for b in range(N):
        clauses.append([idx[(a, b)] for a in range(N) if a != b])
    return Cnf.from_clauses(len(idx), clauses, name=f"gt{size}")


# Satisfiability thresholds of random k-SAT from the cavity method
# (Mertens, Mezard, Zecchina, Random Struct. Algorithms 28, 2006).
ALPHA_K = {3: 4.267, 4: 9.931, 5: 21.117}


@dataclass
class Request:
    rid: int
    arrival_s: float
    k: int
    n: int
    m: int
    seed: int

    def instance(self) -> Cnf:
        return uniform_ksat(self.n, self.m, self.k, seed=self.seed)


def serving_stream(count: int, rate_per_s: float, seed: int = 0, n_lo: int = 100,
                   n_hi: int = 50000, ratio_lo: float = 4.0, ratio_hi: float = 4.6) -> List[Request]:
    """Requests with k uniform in {3,4,5}, n log-uniform in [n_lo, n_hi], the
    clause/variable ratio uniform in [ratio_lo, ratio_hi] for k = 3 and scaled
    by ALPHA_K[k] / ALPHA_K[3] otherwise, and Poisson arrivals at rate_per_s."""
    s = _substream(seed, 21)
    idx = np.arange(count, dtype=np.uint64)
    u_k = splitmix64(s, idx * np.uint64(4) + np.uint64(0))
    u_n = _unit(splitmix64(s, idx * np.uint64(4) + np.uint64(1)))
    u_r = _unit(splitmix64(s, idx * np.uint64(4) + np.uint64(2)))
    u_a = _unit(splitmix64(s, idx * np.uint64(4) + np.uint64(3)))
    ks = 3 + _below(u_k, 3)
    ns = np.floor(np.exp(np.log(n_lo) + u_n * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    ratio = ratio_lo + u_r * (ratio_hi - ratio_lo)
    scale = np.array([ALPHA_K[int(k)] / ALPHA_K[3] for k in ks])
    ms = np.maximum(1, np.rint(ns * ratio * scale)).astype(np.int64)
    gaps = -np.log1p(-u_a) / rate_per_s
    arrivals = np.cumsum(gaps)
    return [Request(rid=i, arrival_s=float(arrivals[i]), k=int(ks[i]), n=int(ns[i]), m=int(ms[i]),
                    seed=int(_substream(seed, 1000 + i) & 0x7FFFFFFF)) for i in range(count)]


def partial_maxsat(n: int, hard, soft, soft_weights) -> Cnf:
    """Partial MaxSAT (hard clauses must hold, soft ones carry weights) as
    one weighted instance: every hard clause weighs top = 1 + sum of the soft
    weights, so violating any hard clause costs more than violating all soft
    ones.  An assignment of cost < top satisfies every hard clause, and its
    cost is then its soft cost."""
    soft_weights = [int(w) for w in soft_weights]
    if len(soft_weights) != len(soft) or any(w < 1 for w in soft_weights):
        raise ValueError("one weight >= 1 per soft clause")
    top = 1 + sum(soft_weights)
    return Cnf.from_clauses(n, list(hard) + list(soft), weights=[top] * len(hard) + soft_weights,
                            name=f"partial_n{n}_h{len(hard)}_s{len(soft)}")


def random_partial(n: int, m_hard: int, m_soft: int, k: int = 3, seed: int = 0) -> Cnf:
    """Hard clauses: planted k-SAT (satisfiable); soft clauses: unit clauses
    on distinct-by-draw variables with random signs, weights uniform 1..9."""
    hard = planted_ksat(n, m_hard, k, seed=seed).clauses()
    s = _substream(seed, 31)
    idx = np.arange(m_soft, dtype=np.uint64)
    var = _below(splitmix64(s, 3 * idx), n)
    sign = (splitmix64(s, 3 * idx + np.uint64(1)) & np.uint64(1)).astype(bool)
    w = 1 + _below(splitmix64(s, 3 * idx + np.uint64(2)), 9)
    soft = [[int(v) + 1 if sg else -(int(v) + 1)] for v, sg in zip(var, sign)]
    return partial_maxsat(n, hard, soft, [int(x) for x in w])
