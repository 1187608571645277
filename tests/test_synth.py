"""The synthetic inputs follow the recipes they stand for: structure (clause
lengths, distinct variables, literal ranges), the stated distributions
(signs, lengths, weights, the Zipf head, the serving stream's k, n, m/n and
arrivals), planted satisfiability, the partial MaxSAT weight encoding, and
determinism by seed.  Distributions are checked against their closed forms
or against an independent sampler of the same recipe (numpy's generator).
No GPU."""
import numpy as np

from synth import ALPHA_K, planted_ksat, random_partial, serving_stream, splitmix64, uniform_ksat, zipf_weighted


def test_uniform_ksat_structure_signs_and_variables():
    n, m, k = 1000, 20000, 3
    a = uniform_ksat(n, m, k, seed=0)
    assert a.n == n and a.m == m and a.nnz == m * k and a.weights is None
    C = a.lits.reshape(m, k)
    V = np.sort(np.abs(C), axis=1)
    assert V.min() >= 1 and V.max() <= n
    assert (V[:, 1:] != V[:, :-1]).all()                 # k distinct variables per clause
    assert abs((C < 0).mean() - 0.5) < 0.01               # Bernoulli(1/2) signs, sd 0.002
    counts = np.bincount(V.ravel(), minlength=n + 1)[1:]  # uniform variables: Binomial(60000, 1/1000)
    assert abs(counts.mean() - 60.0) < 1e-9 and 5.5 < counts.std() < 10.0
    assert np.array_equal(a.lits, uniform_ksat(n, m, k, seed=0).lits)
    assert not np.array_equal(a.lits, uniform_ksat(n, m, k, seed=1).lits)


def _geom_truncated_mean(p, gmax):
    g = np.arange(gmax + 1)
    pg = p * (1 - p) ** g
    return float((g * pg).sum() / pg.sum())


def _zipf_top_share_model(n, s, lens, rng):
    """Share of literal slots taken by rank 1 when each position draws
    Zipf(s) over 1..n and redraws while it equals an earlier variable of its
    clause (the recipe's rejection), sampled with numpy's generator."""
    cdf = np.cumsum(np.arange(1, n + 1, dtype=np.float64) ** (-s))
    cdf /= cdf[-1]
    top = 0
    for L in lens:
        row = []
        for _ in range(L):
            while True:
                r = int(np.searchsorted(cdf, rng.random(), side="right"))
                if r not in row:
                    break
            row.append(r)
        top += row.count(0)
    return top / float(sum(lens))


def test_zipf_weighted_recipe():
    n, m = 200000, 100000
    z = zipf_weighted(n, m, seed=0)
    L = np.diff(z.off)
    assert L.min() >= 2 and L.max() <= 20
    # 2 + Geom(1/3) failures, truncated to <= 18 by rejection: sd of the mean ~0.008
    assert abs(L.mean() - (2 + _geom_truncated_mean(1 / 3, 18))) < 0.035
    rows = [np.abs(z.lits[z.off[j]:z.off[j + 1]]) for j in range(0, m, 50)]
    assert all(len(set(r.tolist())) == len(r) for r in rows)  # distinct within a clause
    assert z.weights.min() >= 1 and z.weights.max() <= 1000 and abs(z.weights.mean() - 500.5) < 5
    assert abs((z.lits < 0).mean() - 0.5) < 0.01
    # the head: rank 1 takes 1/H_{n,1.2} = 0.194 of unconstrained draws; the
    # per-clause rejection lowers it, as an independent sampler of the recipe shows
    counts = np.bincount(np.abs(z.lits))
    share = counts.max() / z.nnz
    rng = np.random.default_rng(5)
    model = _zipf_top_share_model(n, 1.2, L[:6000].tolist(), rng)
    assert abs(share - model) < 0.01, (share, model)
    assert 0.12 < share < 1.0 / np.sum(np.arange(1, n + 1, dtype=np.float64) ** -1.2)


def test_serving_stream_recipe():
    rate = 1000.0
    rs = serving_stream(10000, rate, seed=0)
    ks = np.array([r.k for r in rs])
    ns = np.array([r.n for r in rs])
    ms = np.array([r.m for r in rs])
    arr = np.array([r.arrival_s for r in rs])
    assert set(ks.tolist()) == {3, 4, 5} and np.all(np.abs(np.bincount(ks)[3:] - 10000 / 3) < 200)
    assert ns.min() >= 100 and ns.max() < 50000
    # log-uniform n: log quantiles evenly spaced between log 100 and log 50000
    q = np.quantile(np.log(ns), [0.25, 0.5, 0.75])
    lo, hi = np.log(100), np.log(50000)
    assert np.all(np.abs(q - (lo + np.array([0.25, 0.5, 0.75]) * (hi - lo))) < 0.1)
    for k in (3, 4, 5):
        r = ms[ks == k] / ns[ks == k]
        scale = ALPHA_K[k] / ALPHA_K[3]
        assert r.min() >= 4.0 * scale - 0.01 and r.max() <= 4.6 * scale + 0.01
    gaps = np.diff(arr)
    assert np.all(gaps >= 0) and abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential gaps: coefficient of variation 1
    inst = rs[0].instance()
    assert inst.n == rs[0].n and inst.m == rs[0].m and np.all(np.diff(inst.off) == rs[0].k)


def test_planted_ksat_is_satisfied_by_its_hidden_assignment():
    n, m, seed = 2000, 8000, 0
    c = planted_ksat(n, m, 3, seed=seed)
    hidden = (splitmix64(int(splitmix64(seed, np.array([7], dtype=np.uint64))[0]),
                         np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(bool)
    C = c.lits.reshape(m, 3)
    true = hidden[np.abs(C) - 1] ^ (C < 0)
    assert true.any(axis=1).all()


def test_random_partial_weight_encoding():
    p = random_partial(2000, 6000, 2000, seed=0)
    hard, soft = p.weights[:6000], p.weights[6000:]
    top = int(soft.sum()) + 1
    assert np.all(hard == top) and soft.min() >= 1 and soft.max() <= 9
    assert np.all(np.diff(p.off[6000:]) == 1)  # unit soft clauses
    # any violation of a hard clause costs more than all soft clauses together
    assert top > soft.sum()
