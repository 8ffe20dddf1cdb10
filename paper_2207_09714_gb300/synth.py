"""Seeded synthetic populations, contact graphs and parameter sets.

This module only builds *inputs*: agent ages, a contact graph in
destination-sorted CSR form, the infectiousness-by-day table, the per-age
susceptibility table, per-instance parameters and target curves.  It holds
none of the simulator's arithmetic, so that the FP64 oracle and the CUDA path
can both be fed from it without sharing any code of the method.

The paper's populations come from census and mobility data that are not
available (Sec. 4, App. E); the generators below stand in for them with the
structure the paper describes: agents with one of nine age bins (Sec. 3.1),
households, school/workplace groups and random contacts forming a sparse,
small-world interaction graph (App. A), with per-interaction weights.

CSR convention used everywhere: row ``i`` lists the in-neighbours ``j`` of
agent ``i`` and ``w[p]`` is the weight of the interaction from ``j`` into
``i``.  Self loops are dropped and duplicate pairs are merged by summing their
weights.  All generators here are symmetric (``w_ij == w_ji``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

NUM_AGE_BINS = 9  # 0-10, 11-20, ..., 71-80, 80+ (Sec. 3.1)

# Per-age susceptibility table S_a (Sec. 3.1 names S_a; App. D says it comes from
# clinical sources without printing values).  Project-chosen values.
SUSCEPTIBILITY = np.array([0.4, 0.7, 1.0, 1.0, 1.0, 1.0, 1.2, 1.4, 1.5], dtype=np.float32)

# Interaction-type weight scales: household, school, workplace, random contact.
TYPE_WEIGHT = {"household": 1.0, "school": 0.6, "workplace": 0.4, "random": 0.2}


@dataclasses.dataclass
class Population:
    """One contact graph with agent attributes (destination-sorted CSR)."""

    n: int
    rowptr: np.ndarray  # uint64 [n+1]
    col: np.ndarray  # uint32 [nnz]   in-neighbour j of row i
    w: np.ndarray  # float32 [nnz] weight of the interaction j -> i
    age: np.ndarray  # uint8 [n] in 0..8
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))


def infectiousness_table(tau_EI: int = 4, tau_IR: int = 7, T_E: float = 0.5, T_I: float = 1.0,
                         gamma_shape: float = 3.0, gamma_scale: float = 2.0) -> np.ndarray:
    """Infectiousness by days since exposure, c[k] for k = 0..L-1 (L = tau_EI + tau_IR).

    c[0] = 0 (an agent cannot infect on the day it is exposed, assumption A2 of
    App. A).  For 1 <= k < L, c[k] = T_stage(k) * iota(k): the stage
    transmissibility T_s of Sec. 3.1 (T_E before tau_EI days, T_I after) times
    the mass of a scaled Gamma profile on the day (k-1, k], the form App. D
    names for infectiousness over time (its values are not printed, so the
    shape/scale here are project-chosen).  The table is rescaled to sum to 1.
    """
    from scipy.special import gammainc

    L = tau_EI + tau_IR
    k = np.arange(L, dtype=np.float64)
    cdf = gammainc(gamma_shape, k / gamma_scale)
    mass = np.zeros(L)
    mass[1:] = np.diff(cdf)
    stage = np.where(k < tau_EI, T_E, T_I)
    c = stage * mass
    c[0] = 0.0
    c /= c.sum()
    return c.astype(np.float32)


def _rng(seed) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed))


def _group_pairs(members: np.ndarray, sizes: np.ndarray):
    """All unordered pairs inside consecutive groups of ``members`` with the given sizes."""
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    us, vs = [], []
    for s in np.unique(sizes):
        s = int(s)
        if s < 2:
            continue
        st = starts[sizes == s]
        a, b = np.triu_indices(s, k=1)
        us.append(members[(st[:, None] + a[None, :]).ravel()])
        vs.append(members[(st[:, None] + b[None, :]).ravel()])
    if not us:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(us).astype(np.int64), np.concatenate(vs).astype(np.int64)


def _cut_sizes(rng, total: int, lo: int, hi: int, kind: str = "uniform", p: float = 0.4) -> np.ndarray:
    """Group sizes that add up to exactly ``total`` (the last group is truncated)."""
    if total <= 0:
        return np.zeros(0, np.int64)
    mean = (lo + hi) / 2 if kind == "uniform" else 1.0 / p
    m = int(total / mean * 1.2) + 16
    out = []
    acc = 0
    while acc < total:
        if kind == "uniform":
            s = rng.integers(lo, hi + 1, size=m)
        else:  # geometric on {1,2,...}, resampled until <= hi
            s = rng.geometric(p, size=m)
            bad = s > hi
            while bad.any():
                s[bad] = rng.geometric(p, size=int(bad.sum()))
                bad = s > hi
        out.append(s)
        acc += int(s.sum())
    s = np.concatenate(out).astype(np.int64)
    cs = np.cumsum(s)
    k = int(np.searchsorted(cs, total))
    s = s[: k + 1].copy()
    s[-1] -= int(cs[k] - total)
    return s[s > 0]


def csr_from_undirected(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray,
                        age: np.ndarray, name: str = "") -> Population:
    """Symmetrise an undirected edge list, drop self loops, merge duplicates, build CSR."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    w = np.asarray(w, np.float64)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    dst = np.concatenate([u, v])
    src = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    key = dst * np.int64(n) + src
    order = np.argsort(key, kind="stable")
    key = key[order]
    ww = ww[order]
    if key.size:
        first = np.ones(key.size, bool)
        first[1:] = key[1:] != key[:-1]
        starts = np.flatnonzero(first)
        wsum = np.add.reduceat(ww, starts)
        key = key[starts]
    else:
        wsum = ww
    dst = key // n
    src = key - dst * n
    counts = np.bincount(dst, minlength=n)
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(counts, out=rowptr[1:])
    return Population(n=n, rowptr=rowptr, col=src.astype(np.uint32), w=wsum.astype(np.float32),
                      age=np.asarray(age, np.uint8), name=name)


def population_small(n: int = 10_000, seed: int = 0, er_mean_degree: float = 10.0) -> Population:
    """10k-agent workload: households of size U{1..6} as cliques filled in id order, plus
    Erdos-Renyi contacts of the given mean degree; weights U[0.5, 1.5]; ages U{0..8}."""
    rng = _rng([seed, 100])
    age = rng.integers(0, NUM_AGE_BINS, size=n).astype(np.uint8)
    hs = _cut_sizes(rng, n, 1, 6, "uniform")
    hu, hv = _group_pairs(np.arange(n, dtype=np.int64), hs)
    m = int(round(n * er_mean_degree / 2))
    eu = rng.integers(0, n, size=m)
    ev = rng.integers(0, n, size=m)
    u = np.concatenate([hu, eu])
    v = np.concatenate([hv, ev])
    w = rng.uniform(0.5, 1.5, size=u.size)
    return csr_from_undirected(n, u, v, w, age, name=f"households_er_n{n}")


def population_typed(n: int = 1_000_000, seed: int = 0, er_mean_degree: float = 5.0,
                     powerlaw: bool = False, pl_exponent: float = 2.5, pl_kmax: int = 2000) -> Population:
    """Four-interaction-type population (households, schools, workplaces, random contacts).

    * households: sizes geometric(p=0.4) truncated to <= 6 by resampling, members
      contiguous in id order (census order);
    * groups: age bins 0-1 attend schools, bins 2-6 workplaces, bins 7-8 neither;
      group sizes U{5..30}; members drawn at random (shuffled) from the eligible agents;
    * random contacts: Erdos-Renyi with the given mean degree, or (``powerlaw``)
      Chung-Lu with expected degrees k ~ P(k) proportional to k^-exponent on [1, kmax];
    * weight of an interaction = type scale (1.0 / 0.6 / 0.4 / 0.2) x U[0.5, 1.5].
    """
    rng = _rng([seed, 200])
    age = rng.integers(0, NUM_AGE_BINS, size=n).astype(np.uint8)
    us, vs, ws = [], [], []

    hs = _cut_sizes(rng, n, 1, 6, "geometric", p=0.4)
    u, v = _group_pairs(np.arange(n, dtype=np.int64), hs)
    us.append(u); vs.append(v); ws.append(TYPE_WEIGHT["household"] * rng.uniform(0.5, 1.5, u.size))

    for kind, bins in (("school", (0, 1)), ("workplace", (2, 3, 4, 5, 6))):
        elig = np.flatnonzero(np.isin(age, bins)).astype(np.int64)
        rng.shuffle(elig)
        gs = _cut_sizes(rng, elig.size, 5, 30, "uniform")
        u, v = _group_pairs(elig, gs)
        us.append(u); vs.append(v); ws.append(TYPE_WEIGHT[kind] * rng.uniform(0.5, 1.5, u.size))

    if powerlaw:
        kk = np.arange(1, pl_kmax + 1, dtype=np.float64)
        pk = kk ** (-pl_exponent)
        pk /= pk.sum()
        kexp = rng.choice(kk, size=n, p=pk)
        m = int(round(kexp.sum() / 2))
        cdf = np.cumsum(kexp)
        cdf /= cdf[-1]
        u = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
        v = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
        np.minimum(u, n - 1, out=u); np.minimum(v, n - 1, out=v)
    else:
        m = int(round(n * er_mean_degree / 2))
        u = rng.integers(0, n, size=m)
        v = rng.integers(0, n, size=m)
    us.append(u); vs.append(v); ws.append(TYPE_WEIGHT["random"] * rng.uniform(0.5, 1.5, u.size))

    tag = "powerlaw" if powerlaw else "er"
    return csr_from_undirected(n, np.concatenate(us), np.concatenate(vs), np.concatenate(ws), age,
                               name=f"typed_{tag}_n{n}")


def complete_graph(n: int, age_bin: int = 2) -> Population:
    """Complete graph with unit weights and one age bin (mean-field limit checks)."""
    col = np.empty(n * (n - 1), np.uint32)
    base = np.arange(n, dtype=np.uint32)
    for i in range(n):
        row = np.delete(base, i)
        col[i * (n - 1):(i + 1) * (n - 1)] = row
    rowptr = (np.arange(n + 1, dtype=np.uint64) * np.uint64(n - 1))
    return Population(n=n, rowptr=rowptr, col=col, w=np.ones(col.size, np.float32),
                      age=np.full(n, age_bin, np.uint8), name=f"complete_n{n}")


def random_directed(n: int, nnz_per_row: float, seed: int, w_lo: float = 0.5, w_hi: float = 1.5) -> Population:
    """Small directed (asymmetric) graph, used where edge direction must be visible."""
    rng = _rng([seed, 300])
    m = int(round(n * nnz_per_row))
    dst = rng.integers(0, n, size=m)
    src = rng.integers(0, n, size=m)
    keep = dst != src
    dst, src = dst[keep], src[keep]
    key = np.unique(dst.astype(np.int64) * n + src)
    dst = key // n
    src = key % n
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(dst, minlength=n), out=rowptr[1:])
    w = rng.uniform(w_lo, w_hi, size=key.size).astype(np.float32)
    age = rng.integers(0, NUM_AGE_BINS, size=n).astype(np.uint8)
    return Population(n=n, rowptr=rowptr, col=src.astype(np.uint32), w=w, age=age, name=f"directed_n{n}")


def permute(pop: Population, perm: np.ndarray) -> Population:
    """Relabel agents: new id of old agent ``i`` is ``perm[i]``; rows re-sorted by new ids."""
    n = pop.n
    perm = np.asarray(perm, np.int64)
    deg = pop.degrees()
    dst_old = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = perm[dst_old]
    src = perm[pop.col.astype(np.int64)]
    key = dst * n + src
    order = np.argsort(key, kind="stable")
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(dst, minlength=n), out=rowptr[1:])
    age = np.empty(n, np.uint8)
    age[perm] = pop.age
    return Population(n=n, rowptr=rowptr, col=src[order].astype(np.uint32), w=pop.w[order].copy(),
                      age=age, name=pop.name + "_perm")


@dataclasses.dataclass
class Bipartite:
    """Agents and locations, the heterogeneous contact structure of GradABM-JUNE (Sec. 6):
    agent i attends location l with weight w_il (agent-sorted incidence).  Two agents
    interact through every location they share: the one-hop weight of the pair is
    W_ij = sum_l w_il w_jl (i != j)."""

    n: int               # agents
    n_loc: int           # locations
    rowptr: np.ndarray   # uint64 [n+1]: agent i's locations are loc[rowptr[i]:rowptr[i+1]]
    loc: np.ndarray      # uint32 [nnz]
    w: np.ndarray        # float32 [nnz] attendance weight w_il
    age: np.ndarray      # uint8 [n]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.loc.shape[0])


def population_bipartite(n: int = 20_000, seed: int = 0, school=(100, 400), work=(5, 60),
                         venues_per_agent: float = 1.5, venue_size: float = 40.0) -> Bipartite:
    """Agents attending locations: one household each (sizes geometric(p = 0.4) up to 6), a
    school (age bins 0-1, sizes U{school}) or a workplace (bins 2-6, U{work}), and a
    Poisson(venues_per_agent) number of shared venues (shops, transport) drawn uniformly
    among n / venue_size venues.  Weight = type scale (household 1.0, school 0.6, workplace
    0.4, venue 0.2) x U[0.5, 1.5].  Locations are numbered households, schools,
    workplaces, venues; each agent's list is sorted by location."""
    rng = _rng([seed, 800])
    age = rng.integers(0, NUM_AGE_BINS, size=n).astype(np.uint8)
    agents, locs, ws = [], [], []
    base = 0
    hs = _cut_sizes(rng, n, 1, 6, "geometric", p=0.4)
    agents.append(np.arange(n, dtype=np.int64))
    locs.append(np.repeat(np.arange(hs.size, dtype=np.int64), hs))
    ws.append(TYPE_WEIGHT["household"] * rng.uniform(0.5, 1.5, n))
    base += hs.size
    for kind, bins, (lo, hi) in (("school", (0, 1), school), ("workplace", (2, 3, 4, 5, 6), work)):
        elig = np.flatnonzero(np.isin(age, bins)).astype(np.int64)
        rng.shuffle(elig)
        gs = _cut_sizes(rng, elig.size, lo, hi, "uniform")
        agents.append(elig)
        locs.append(base + np.repeat(np.arange(gs.size, dtype=np.int64), gs))
        ws.append(TYPE_WEIGHT[kind] * rng.uniform(0.5, 1.5, elig.size))
        base += gs.size
    n_venue = max(1, int(n / venue_size))
    k = rng.poisson(venues_per_agent, size=n)
    va = np.repeat(np.arange(n, dtype=np.int64), k)
    vl = base + rng.integers(0, n_venue, size=va.size)
    agents.append(va)
    locs.append(vl)
    ws.append(TYPE_WEIGHT["random"] * rng.uniform(0.5, 1.5, va.size))
    base += n_venue
    a = np.concatenate(agents)
    l = np.concatenate(locs)
    w = np.concatenate(ws)
    key = a * np.int64(base) + l
    order = np.argsort(key, kind="stable")
    key, w = key[order], w[order]
    uniq, start = np.unique(key, return_index=True)          # repeated visits add up
    wsum = np.add.reduceat(w, start)
    a, l = uniq // base, uniq % base
    rowptr = np.zeros(n + 1, np.uint64)
    np.cumsum(np.bincount(a, minlength=n), out=rowptr[1:])
    return Bipartite(n=n, n_loc=int(base), rowptr=rowptr, loc=l.astype(np.uint32), w=wsum.astype(np.float32),
                     age=age, name=f"bipartite_n{n}")


def uneven_county_sizes(num: int = 32, lo: float = 5e4, hi: float = 2e6, seed: int = 0,
                        scale: float = 1.0) -> list:
    """Agent counts of ``uneven_counties``: log-uniform in [lo, hi] (times ``scale``), at least 64."""
    rng = _rng([seed, 400])
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=num)) * scale
    return [max(int(s), 64) for s in sizes]


def county(g: int, n: int, seed: int = 0) -> Population:
    """County g of ``uneven_counties`` (the typed generator with its own seed)."""
    return population_typed(n, seed=seed * 1000 + g)


def uneven_counties(num: int = 32, lo: float = 5e4, hi: float = 2e6, seed: int = 0, scale: float = 1.0):
    """County graphs with agent counts log-uniform in [lo, hi] (times ``scale``)."""
    return [county(g, n, seed) for g, n in enumerate(uneven_county_sizes(num, lo, hi, seed, scale))]


def target_curve(T: int, n: int, seed: int = 1, growth: float = 0.12, level: float = 2e-7) -> np.ndarray:
    """Seeded synthetic daily-deaths target y_t (FP64): an exponential-growth curve with
    multiplicative noise, scaled to the population size."""
    rng = _rng([seed, 500])
    t = np.arange(T, dtype=np.float64)
    base = level * n * np.exp(growth * t)
    return base * (1.0 + 0.1 * rng.standard_normal(T))


def instance_params(num: int, T: int, seed: int = 0, R_range=(1.5, 4.0), m_range=(0.005, 0.05)):
    """Per-instance (R_t, m_t, S_a) with R ~ U[R_range], m ~ U[m_range], constant over days."""
    rng = _rng([seed, 600])
    R = np.repeat(rng.uniform(*R_range, size=(num, 1)), T, axis=1).astype(np.float32)
    m = np.repeat(rng.uniform(*m_range, size=(num, 1)), T, axis=1).astype(np.float32)
    S = np.tile(SUSCEPTIBILITY, (num, 1)).astype(np.float32)
    return R, m, S
