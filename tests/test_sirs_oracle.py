"""Pins of the SIRS-reinfection oracle (oracle/sirs.py) against things other than itself.

* With tau_RS >= T nobody returns within the horizon: the forward and the adjoint are
  the base model's C oracle's (the adjoint to 1e-10).
* The state rules hold on every day: S + E + I + RM = n, an agent's exposures are at
  least L + tau_RS days apart, and reinfections do happen.
* The hand-written adjoint equals torch autograd (CPU, FP64) through a dense restatement
  in which every draw is hard + soft - soft.detach() and returning mass re-enters S
  (App. B's straight-through estimator).
* On a 4-agent graph with fast cycles, the sampled deaths and reinfection frequencies
  over 10k Philox keys match an exact enumeration of the law (within 5 sigma).
"""
import numpy as np
import pytest

import oracle as O
from oracle import sirs as SI
from paper_2207_09714_gb300 import synth

NEVER = 32767


def test_no_return_within_the_horizon_is_the_base_model():
    pop = synth.population_small(n=3000, seed=4)
    T, n_seed = 36, 20
    rng = np.random.default_rng(3)
    R = rng.uniform(2.2, 3.4, T).astype(np.float32)
    m = rng.uniform(0.01, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    c = synth.infectiousness_table()
    for seed in range(20):
        base = O.forward_hard(pop, O.Model(4, 7, c, seed=seed), R, m, S, n_seed=n_seed)
        if base["margin"] > 1e-9:
            break
    md = SI.SirsModel(4, 7, T, c, seed=seed)
    f = SI.forward(pop, md, R, m, S, n_seed=n_seed)
    assert np.array_equal(f["e_final"].astype(np.int16), base["e_final"])
    assert np.array_equal(f["counts"], base["counts"])
    assert np.allclose(f["D"], base["D"], rtol=1e-15, atol=0)
    _, gD = O.mse(f["D"], rng.uniform(0, 3, T))
    g = SI.backward(pop, md, R, m, S, f["e_hist"], gD)
    h = O.backward_hard(pop, O.Model(4, 7, c, seed=seed), R, m, S, base["e_final"], gD)
    for k in ("dR", "dm", "dS"):
        ref = np.abs(h[k]).max()
        assert ref > 0
        assert np.allclose(g[k], h[k], rtol=1e-10, atol=1e-12 * ref), k


def test_state_rules_and_reinfection():
    pop = synth.population_small(n=3000, seed=6)
    T = 60
    md = SI.SirsModel(3, 5, 4, np.r_[0.0, np.full(7, 1 / 7)].astype(np.float32), seed=1)
    f = SI.forward(pop, md, np.full(T, 3.0, np.float32), np.full(T, 0.02, np.float32),
                   synth.SUSCEPTIBILITY.astype(np.float32), n_seed=30)
    assert np.all(f["counts"].sum(axis=1) == pop.n)
    eh = f["e_hist"]
    changed = eh[1:] != eh[:-1]                    # exposures: day t's state -> day t+1's
    t_idx, i_idx = np.nonzero(changed)
    assert np.all(eh[t_idx + 1, i_idx] == t_idx)   # a change is always an exposure on that day
    prev = eh[t_idx, i_idx]
    assert np.all((prev == NEVER) | (t_idx - prev >= md.cycle))
    exposures_per_agent = np.bincount(i_idx, minlength=pop.n)
    assert exposures_per_agent.max() >= 2          # reinfections happen


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
    cohorts = {-md.tau_EI: nseed}
    D = []
    for t in range(T):
        x = torch.zeros(n, dtype=torch.float64)
        for d, nd in cohorts.items():
            if 1 <= t - d < L:
                x = x + nd * float(md.c[t - d])
        D.append(mt[t] * cohorts[t - L].sum() if (t - L) in cohorts else torch.zeros((), dtype=torch.float64))
        lam = Rt[t] * St[age] * (W @ x) / Dbar
        p = -torch.expm1(-lam)
        u = torch.tensor(O.uniform(md.seed, ids, t, 0, 0))
        ysoft = p * (1 - u) / (p * (1 - u) + (1 - p) * u)
        yhard = ((u < p.detach()) & (s > 0.5)).to(torch.float64)
        yh = yhard + ysoft - ysoft.detach()
        cohorts[t] = s * yh
        s = s * (1 - yh)
        back = t + 1 - md.cycle                      # mass exposed then is susceptible again on day t + 1
        if back in cohorts:
            s = s + cohorts[back]
    Dv = torch.stack(D)
    loss = ((Dv - torch.tensor(y)) ** 2).mean()
    loss.backward()
    return Dv.detach().numpy(), Rt.grad.numpy(), mt.grad.numpy(), St.grad.numpy()


def test_adjoint_matches_autograd():
    pop = synth.population_small(n=300, seed=5, er_mean_degree=6)
    T, n_seed = 40, 8
    md = SI.SirsModel(3, 5, 3, np.r_[0.0, np.full(7, 0.15)].astype(np.float32), seed=4)
    rng = np.random.default_rng(7)
    R = rng.uniform(3.0, 5.0, T).astype(np.float32)
    m = rng.uniform(0.2, 0.6, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    f = SI.forward(pop, md, R, m, S, n_seed=n_seed)
    assert f["margin"] > 1e-9
    eh = f["e_hist"]
    assert np.bincount(np.nonzero(eh[1:] != eh[:-1])[1], minlength=pop.n).max() >= 2   # reinfections
    y = rng.uniform(0, 3, T)
    _, gD = O.mse(f["D"], y)
    Dg, dR, dm, dS = _autograd(pop, md, R, m, S, n_seed, y)
    assert np.allclose(Dg, f["D"], rtol=0, atol=1e-12)
    g = SI.backward(pop, md, R, m, S, eh, gD)
    for name, a, b in (("dR", g["dR"], dR), ("dm", g["dm"], dm), ("dS", g["dS"], dS)):
        ref = np.abs(b).max()
        assert ref > 0, name
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * ref), (name, a, b)


def _exact_sirs_law(W, age, S_age, c, tau_EI, tau_IR, tau_RS, R, m, e0):
    """E[D_t] and P(an agent is exposed at least twice) by exact enumeration: every
    reachable state (last exposure days) carried with its probability through the days,
    each susceptible agent infected independently with p_i = 1 - exp(-lambda_i)."""
    import itertools
    from collections import defaultdict
    n, T, L = len(e0), len(R), tau_EI + tau_IR
    cycle = L + tau_RS
    Dbar = sum(sum(row) for row in W) / n
    states = {(tuple(int(v) for v in e0), (0,) * n): 1.0}   # (last exposure days, exposures since day 0)
    ED = [0.0] * T
    for t in range(T):
        nxt = defaultdict(float)
        for (e, cnt), pr in states.items():
            x = [float(c[t - ej]) if ej != NEVER and 1 <= t - ej < L else 0.0 for ej in e]
            ED[t] += pr * float(m[t]) * sum(1 for ej in e if ej != NEVER and t - ej == L)
            sus = [i for i in range(n) if e[i] == NEVER or t - e[i] >= cycle]
            p = {}
            for i in sus:
                lam = float(R[t]) * float(S_age[age[i]]) * sum(W[j][i] * x[j] for j in range(n)) / Dbar
                p[i] = 1.0 - np.exp(-lam)
            for outcome in itertools.product((0, 1), repeat=len(sus)):
                q = pr
                e2, c2 = list(e), list(cnt)
                for i, hit in zip(sus, outcome):
                    q *= p[i] if hit else 1.0 - p[i]
                    if hit:
                        e2[i] = t
                        c2[i] += 1
                if q > 0.0:
                    nxt[(tuple(e2), tuple(c2))] += q
        states = nxt
    P2 = [sum(pr for (e, cnt), pr in states.items() if cnt[i] >= 2) for i in range(n)]
    return ED, P2


def test_monte_carlo_matches_exact_law():
    """A 4-agent weighted graph with fast cycles (L = 3, back to S after 1 more day): the
    oracle's sampled deaths and reinfection frequencies over 10k Philox keys lie within
    5 sigma of the exact law."""
    import math
    rowptr = np.array([0, 2, 4, 6, 8], np.uint64)
    col = np.array([1, 2, 0, 3, 0, 3, 1, 2], np.uint32)
    w = np.array([1.0, 0.5, 1.0, 2.0, 0.5, 1.5, 2.0, 1.5], np.float32)
    pop = synth.Population(n=4, rowptr=rowptr, col=col, w=w, age=np.array([0, 3, 5, 8], np.uint8))
    W = [[0.0] * 4 for _ in range(4)]
    for i in range(4):
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            W[int(col[q])][i] += float(w[q])
    c = np.array([0.0, 0.6, 0.4], np.float32)
    T = 9
    R = np.full(T, 3.5, np.float32)
    m = np.linspace(0.1, 0.5, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    e0 = np.array([-1, NEVER, NEVER, NEVER], np.int64)
    ED, P2 = _exact_sirs_law(W, pop.age, S, c, 1, 2, 1, R, m, e0)
    runs = 10_000
    Dsum = np.zeros(T); D2 = np.zeros(T); twice = np.zeros(4)
    for s in range(runs):
        f = SI.forward(pop, SI.SirsModel(1, 2, 1, c, seed=s), R, m, S, e0=e0)
        Dsum += f["D"]; D2 += f["D"] ** 2
        eh = f["e_hist"]
        twice += np.bincount(np.nonzero(eh[1:] != eh[:-1])[1], minlength=4) >= 2
    assert max(P2) > 0.05                            # reinfection is common here
    for t in range(T):
        var = max(D2[t] / runs - (Dsum[t] / runs) ** 2, 1e-12)
        assert abs(Dsum[t] / runs - ED[t]) <= 5 * math.sqrt(var / runs) + 1e-12, (t, Dsum[t] / runs, ED[t])
    for i in range(4):
        se = math.sqrt(max(P2[i] * (1 - P2[i]), 1e-12) / runs)
        assert abs(twice[i] / runs - P2[i]) <= 5 * se + 1e-12, (i, twice[i] / runs, P2[i])
