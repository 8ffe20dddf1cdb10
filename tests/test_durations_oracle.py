"""Pins of the stochastic-duration oracle (oracle/durations.py) against things other than
itself.

* A pmf with all its mass on tau_IR is the base model: forward and adjoint equal the C
  oracle's (the adjoint to 1e-10).
* The drawn durations follow the pmf (frequencies within 5 sigma over 200k draws).
* The hand-written adjoint equals torch autograd (CPU, FP64) through a dense restatement
  of the forward whose infection draws are hard + soft - soft.detach() (App. B).
* On a 4-agent graph the sampled E[D_t] over 10k Philox keys matches an exact
  enumeration of the law (within 5 sigma).
"""
import numpy as np
import pytest

import oracle as O
from oracle import durations as DU
from paper_2207_09714_gb300 import synth

NEVER = 32767


def test_point_mass_is_the_base_model():
    pop = synth.population_small(n=3000, seed=4)
    T, n_seed = 36, 20
    rng = np.random.default_rng(3)
    R = rng.uniform(2.2, 3.4, T).astype(np.float32)
    m = rng.uniform(0.01, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    c = synth.infectiousness_table()
    p = np.zeros(7, np.float32); p[6] = 1.0
    for seed in range(20):
        base = O.forward_hard(pop, O.Model(4, 7, c, seed=seed), R, m, S, n_seed=n_seed)
        if base["margin"] > 1e-9:
            break
    md = DU.DurationModel(4, 7, p, c, seed=seed)
    f = DU.forward(pop, md, R, m, S, n_seed=n_seed)
    assert np.array_equal(f["e_final"], base["e_final"])
    assert np.array_equal(f["counts"], base["counts"])
    assert np.array_equal(f["newRM"], base["newRM"])
    assert np.allclose(f["D"], base["D"], rtol=1e-15, atol=0)
    y = rng.uniform(0, 3, T)
    _, gD = O.mse(f["D"], y)
    g = DU.backward(pop, md, R, m, S, f["e_final"], gD)
    h = O.backward_hard(pop, O.Model(4, 7, c, seed=seed), R, m, S, f["e_final"], gD)
    for k in ("dR", "dm", "dS"):
        ref = np.abs(h[k]).max()
        assert ref > 0
        assert np.allclose(g[k], h[k], rtol=1e-10, atol=1e-12 * ref), k


def test_draws_follow_the_pmf():
    p = np.array([0.05, 0.1, 0.3, 0.25, 0.15, 0.1, 0.05], np.float32)
    md = DU.DurationModel(4, 7, p, synth.infectiousness_table(), seed=9)
    n = 200_000
    ids = np.arange(n, dtype=np.uint32)
    for d in (-4, 0, 17):
        j = DU.exit_offsets(md, ids, np.full(n, d)) - md.tau_EI
        freq = np.bincount(j, minlength=8)[1:] / n
        sig = np.sqrt(p * (1 - p) / n)
        assert np.all(np.abs(freq - p) < 5 * sig), (d, freq, p)
    # exposures before day 0 share the day-0 key
    assert np.array_equal(DU.exit_offsets(md, ids[:100], np.full(100, -3)),
                          DU.exit_offsets(md, ids[:100], np.zeros(100, np.int64)))


def _autograd(pop, md, R, m, S, n_seed, y):
    torch = pytest.importorskip("torch")
    n, T, L = pop.n, len(R), md.L
    A = np.zeros((n, n))
    for i in range(n):
        for q in range(int(pop.rowptr[i]), int(pop.rowptr[i + 1])):
            A[i, int(pop.col[q])] += float(pop.w[q])
    W = torch.tensor(A, dtype=torch.float64)
    Dbar = float(np.sum(np.asarray(pop.w, np.float64))) / n
    ids = np.arange(n, dtype=np.uint32)
    Rt = torch.tensor(R.astype(np.float64), requires_grad=True)
    mt = torch.tensor(m.astype(np.float64), requires_grad=True)
    St = torch.tensor(S.astype(np.float64), requires_grad=True)
    age = torch.tensor(np.asarray(pop.age, np.int64))
    seeds = O.select_seeds(n, md.seed, 0, n_seed)
    s = torch.ones(n, dtype=torch.float64)
    s[seeds] = 0.0
    nseed = torch.zeros(n, dtype=torch.float64)
    nseed[seeds] = 1.0
    # cohort d: (exposed mass n(d), each agent's exit offset for an exposure on day d)
    cohorts = {-md.tau_EI: (nseed, DU.exit_offsets(md, ids, np.full(n, -md.tau_EI)))}
    D = []
    E = np.full(n, NEVER, np.int64)
    E[seeds] = -md.tau_EI
    for t in range(T):
        x = torch.zeros(n, dtype=torch.float64)
        exits = torch.zeros(n, dtype=torch.float64)
        for d, (nd, Lx) in cohorts.items():
            k = t - d
            if 1 <= k < L:
                x = x + nd * torch.tensor(np.where(k < Lx, float(md.c[k]), 0.0))
            exits = exits + nd * torch.tensor((k == Lx).astype(np.float64))
        D.append(mt[t] * exits.sum())
        lam = Rt[t] * St[age] * (W @ x) / Dbar
        p = -torch.expm1(-lam)
        u = torch.tensor(O.uniform(md.seed, ids, t, 0, 0))
        ysoft = p * (1 - u) / (p * (1 - u) + (1 - p) * u)
        yhard = ((u < p.detach()) & (s > 0.5)).to(torch.float64)
        E[yhard.numpy() > 0.5] = t
        yh = yhard + ysoft - ysoft.detach()
        cohorts[t] = (s * yh, DU.exit_offsets(md, ids, np.full(n, t)))
        s = s * (1 - yh)
    Dv = torch.stack(D)
    loss = ((Dv - torch.tensor(y)) ** 2).mean()
    loss.backward()
    return Dv.detach().numpy(), E, Rt.grad.numpy(), mt.grad.numpy(), St.grad.numpy()


def test_adjoint_matches_autograd():
    pop = synth.population_small(n=300, seed=5, er_mean_degree=6)
    T, n_seed = 26, 8
    p = np.array([0.1, 0.1, 0.2, 0.3, 0.1, 0.1, 0.1], np.float32)
    md = DU.DurationModel(3, 7, p, np.r_[0.0, np.full(9, 0.1)].astype(np.float32), seed=4)
    rng = np.random.default_rng(7)
    R = rng.uniform(2.5, 4.5, T).astype(np.float32)
    m = rng.uniform(0.2, 0.6, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    f = DU.forward(pop, md, R, m, S, n_seed=n_seed)
    assert f["margin"] > 1e-9 and f["D"].sum() > 0
    y = rng.uniform(0, 3, T)
    _, gD = O.mse(f["D"], y)
    Dg, Eg, dR, dm, dS = _autograd(pop, md, R, m, S, n_seed, y)
    assert np.array_equal(Eg, f["e_final"].astype(np.int64))
    assert np.allclose(Dg, f["D"], rtol=0, atol=1e-12)
    g = DU.backward(pop, md, R, m, S, f["e_final"], gD)
    for name, a, b in (("dR", g["dR"], dR), ("dm", g["dm"], dm), ("dS", g["dS"], dS)):
        ref = np.abs(b).max()
        assert ref > 0, name
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * ref), (name, a, b)


def _exact_duration_law(W, age, S_age, c, tau_EI, p_IR, R, m, e0):
    """E[D_t] by exact enumeration over (exposure days, exit offsets): each exposure
    draws its I-stage duration j from p_IR at once."""
    import itertools
    from collections import defaultdict
    n, T = len(e0), len(R)
    J = len(p_IR)
    Dbar = sum(sum(row) for row in W) / n
    start = defaultdict(float)
    exposed0 = [i for i in range(n) if e0[i] != NEVER]
    for js in itertools.product(range(1, J + 1), repeat=len(exposed0)):
        q = 1.0
        Lx = [0] * n
        for i, j in zip(exposed0, js):
            q *= float(p_IR[j - 1])
            Lx[i] = tau_EI + j
        if q > 0.0:
            start[(tuple(int(v) for v in e0), tuple(Lx))] += q
    states = dict(start)
    ED = [0.0] * T
    for t in range(T):
        nxt = defaultdict(float)
        for (e, Lx), pr in states.items():
            x = [float(c[t - ej]) if ej != NEVER and 1 <= t - ej < Li else 0.0 for ej, Li in zip(e, Lx)]
            ED[t] += pr * float(m[t]) * sum(1 for ej, Li in zip(e, Lx) if ej != NEVER and t - ej == Li)
            sus = [i for i in range(n) if e[i] == NEVER]
            p = {i: 1.0 - np.exp(-float(R[t]) * float(S_age[age[i]]) * sum(W[jj][i] * x[jj] for jj in range(n)) / Dbar)
                 for i in sus}
            for outcome in itertools.product((0, 1), repeat=len(sus)):
                q = pr
                hit_ids = [i for i, h in zip(sus, outcome) if h]
                for i, h in zip(sus, outcome):
                    q *= p[i] if h else 1.0 - p[i]
                if q <= 0.0:
                    continue
                for js in itertools.product(range(1, J + 1), repeat=len(hit_ids)):
                    q2 = q
                    e2, L2 = list(e), list(Lx)
                    for i, j in zip(hit_ids, js):
                        q2 *= float(p_IR[j - 1])
                        e2[i] = t
                        L2[i] = tau_EI + j
                    if q2 > 0.0:
                        nxt[(tuple(e2), tuple(L2))] += q2
        states = nxt
    return ED


def test_monte_carlo_matches_exact_law():
    """4 agents, a 3-point duration pmf: the sampled E[D_t] over 10k Philox keys lies
    within 5 sigma of the exact law."""
    import math
    rowptr = np.array([0, 2, 4, 6, 8], np.uint64)
    col = np.array([1, 2, 0, 3, 0, 3, 1, 2], np.uint32)
    w = np.array([1.0, 0.5, 1.0, 2.0, 0.5, 1.5, 2.0, 1.5], np.float32)
    pop = synth.Population(n=4, rowptr=rowptr, col=col, w=w, age=np.array([0, 3, 5, 8], np.uint8))
    W = [[0.0] * 4 for _ in range(4)]
    for i in range(4):
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            W[int(col[q])][i] += float(w[q])
    p = np.array([0.3, 0.5, 0.2], np.float32)
    c = np.array([0.0, 0.5, 0.5, 0.5], np.float32)
    T = 9
    R = np.full(T, 3.0, np.float32)
    m = np.linspace(0.2, 0.7, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    e0 = np.array([-1, NEVER, NEVER, NEVER], np.int64)
    ED = _exact_duration_law(W, pop.age, S, c, 1, p, R, m, e0)
    runs = 10_000
    Dsum = np.zeros(T); D2 = np.zeros(T)
    for s in range(runs):
        f = DU.forward(pop, DU.DurationModel(1, 3, p, c, seed=s), R, m, S, e0=e0)
        Dsum += f["D"]; D2 += f["D"] ** 2
    assert sum(ED) > 0.3
    for t in range(T):
        var = max(D2[t] / runs - (Dsum[t] / runs) ** 2, 1e-12)
        assert abs(Dsum[t] / runs - ED[t]) <= 5 * math.sqrt(var / runs) + 1e-12, (t, Dsum[t] / runs, ED[t])
