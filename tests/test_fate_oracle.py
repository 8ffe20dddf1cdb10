"""Pins of the sampled R/M split oracle (oracle/fate.py) against things other than itself.

* tau_IM = tau_IR: the fate changes no infectiousness, so the trajectory and the stage
  counts are those of the base model's C oracle; deaths are the M-fated share of the RM
  exits (all of them at m = 1, none at m = 0, about m of them otherwise).
* The hand-written straight-through adjoint equals torch autograd (CPU, FP64) through a
  dense restatement of the forward in which every draw is hard + soft - soft.detach()
  (the definition of the straight-through estimator, App. B), for tau_IM below, equal to
  and above tau_IR.
* On a 4-agent graph the sampled E[D_t] over 10k Philox keys matches an exact
  enumeration of the law over exposures and fates (within 5 sigma), for tau_IM below
  and above tau_IR.
"""
import numpy as np
import pytest

import oracle as O
from oracle import fate as F
from paper_2207_09714_gb300 import synth

NEVER = 32767


def _table(L):
    c = np.zeros(L, np.float32)
    k = np.arange(1, L)
    c[1:] = (np.exp(-0.5 * (k - 0.6 * L) ** 2 / (0.3 * L) ** 2)).astype(np.float32)
    return (c / c.sum()).astype(np.float32)


def test_equal_times_reduce_to_base_model():
    pop = synth.population_small(n=4000, seed=3)
    T, n_seed = 40, 25
    rng = np.random.default_rng(1)
    R = rng.uniform(2.2, 3.2, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    c = synth.infectiousness_table()
    for seed in range(20):
        base = O.forward_hard(pop, O.Model(4, 7, c, seed=seed), R, np.full(T, 0.5, np.float32), S, n_seed=n_seed)
        if base["margin"] > 1e-9:
            break
    md = F.FateModel(4, 7, 7, c, seed=seed)
    exits = base["newRM"]
    assert exits.sum() > 500
    for mval in (0.0, 1.0, 0.3):
        m = np.full(T, mval, np.float32)
        f = F.forward(pop, md, R, m, S, n_seed=n_seed)
        assert np.array_equal(f["e_final"], base["e_final"])
        assert np.array_equal(f["counts"], base["counts"])
        E = f["e_final"].astype(np.int64)
        for t in range(T):
            ex = (E != NEVER) & (t - E == md.L_M)
            assert f["D"][t] == np.sum(f["fate"] & ex)
        if mval == 0.0:
            assert f["D"].sum() == 0
        elif mval == 1.0:
            assert np.array_equal(f["D"], exits.astype(np.float64))
        else:
            N = exits.sum()
            assert abs(f["D"].sum() - mval * N) < 4 * np.sqrt(N * mval * (1 - mval))


def _autograd(pop, md, R, m, S, n_seed, y):
    """Loss and its gradients by torch autograd through the straight-through surrogate."""
    torch = pytest.importorskip("torch")
    n, T, L = pop.n, len(R), md.L
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(int(pop.rowptr[i]), int(pop.rowptr[i + 1])):
            A[i, int(pop.col[p])] += float(pop.w[p])
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
    n_seed_vec = torch.zeros(n, dtype=torch.float64)
    n_seed_vec[seeds] = 1.0

    def phi_hat(d):
        tI = max(d + md.tau_EI, 0)
        if tI >= T:
            return torch.zeros(n, dtype=torch.float64)
        v = torch.tensor(O.uniform(md.seed, ids, tI, 0, 1))
        soft = mt[tI] * (1 - v) / (mt[tI] * (1 - v) + (1 - mt[tI]) * v)
        hard = (v < float(m[tI])).to(torch.float64)
        return hard + soft - soft.detach()

    cohorts = {-md.tau_EI: (n_seed_vec, phi_hat(-md.tau_EI))}
    D = []
    E = np.full(n, NEVER, np.int64)
    E[seeds] = -md.tau_EI
    for t in range(T):
        x = torch.zeros(n, dtype=torch.float64)
        for d, (nd, ph) in cohorts.items():
            k = t - d
            if 1 <= k < L:
                cR = float(md.c[k]) if k < md.L_R else 0.0
                cM = float(md.c[k]) if k < md.L_M else 0.0
                x = x + nd * (cR * (1 - ph) + cM * ph)
        if t - md.L_M in cohorts:
            nd, ph = cohorts[t - md.L_M]
            D.append((nd * ph).sum())
        else:
            D.append(torch.zeros((), dtype=torch.float64))
        lam = Rt[t] * St[age] * (W @ x) / Dbar
        p = -torch.expm1(-lam)
        u = torch.tensor(O.uniform(md.seed, ids, t, 0, 0))
        ysoft = p * (1 - u) / (p * (1 - u) + (1 - p) * u)
        yhard = ((u < p.detach()) & (s > 0.5)).to(torch.float64)
        E[yhard.numpy() > 0.5] = t
        yh = yhard + ysoft - ysoft.detach()
        cohorts[t] = (s * yh, phi_hat(t))
        s = s * (1 - yh)
    Dv = torch.stack(D)
    loss = ((Dv - torch.tensor(y)) ** 2).mean()
    loss.backward()
    return (Dv.detach().numpy(), E, float(loss.detach()), Rt.grad.numpy(), mt.grad.numpy(), St.grad.numpy())


@pytest.mark.parametrize("tau_IM", [4, 7, 10])
def test_adjoint_matches_autograd(tau_IM):
    pop = synth.population_small(n=300, seed=5, er_mean_degree=6)
    T, n_seed, tau_EI, tau_IR = 24, 8, 3, 7
    md = F.FateModel(tau_EI, tau_IR, tau_IM, _table(tau_EI + max(tau_IR, tau_IM)), seed=2)
    rng = np.random.default_rng(tau_IM)
    R = rng.uniform(2.5, 4.5, T).astype(np.float32)
    m = rng.uniform(0.2, 0.6, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    f = F.forward(pop, md, R, m, S, n_seed=n_seed)
    assert f["margin"] > 1e-9
    assert f["D"].sum() > 5
    y = rng.uniform(0, 3, T)
    loss, gD = O.mse(f["D"], y)
    Dg, Eg, loss_g, dR, dm, dS = _autograd(pop, md, R, m, S, n_seed, y)
    assert np.array_equal(Eg, f["e_final"].astype(np.int64))
    assert np.allclose(Dg, f["D"], rtol=0, atol=1e-12)   # hard values (+ soft - soft, rounded)
    assert loss_g == pytest.approx(loss, rel=1e-12)
    g = F.backward(pop, md, R, m, S, f["e_final"], gD)
    for name, a, b in (("dR", g["dR"], dR), ("dm", g["dm"], dm), ("dS", g["dS"], dS)):
        ref = np.abs(b).max()
        assert ref > 0, name
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * ref), (name, a, b)


def _tiny_graph():
    rowptr = np.array([0, 2, 4, 6, 8], np.uint64)
    col = np.array([1, 2, 0, 3, 0, 3, 1, 2], np.uint32)
    w = np.array([1.0, 0.5, 1.0, 2.0, 0.5, 1.5, 2.0, 1.5], np.float32)
    pop = synth.Population(n=4, rowptr=rowptr, col=col, w=w, age=np.array([0, 3, 5, 8], np.uint8))
    W = [[0.0] * 4 for _ in range(4)]
    for i in range(4):
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            W[int(col[q])][i] += float(w[q])
    return pop, W


def _exact_fate_law(W, age, S_age, c, tau_EI, tau_IR, tau_IM, R, m, e0):
    """E[D_t] by exact enumeration over (exposure days, fates): each agent's fate is M
    with probability m of its I-entry day (day 0 for earlier exposures), drawn then."""
    import itertools
    from collections import defaultdict
    n, T = len(e0), len(R)
    L_R, L_M = tau_EI + tau_IR, tau_EI + tau_IM
    Dbar = sum(sum(row) for row in W) / n
    states = {(tuple(int(v) for v in e0), (None,) * n): 1.0}
    ED = [0.0] * T
    for t in range(T):
        # fates drawn today
        drawn = defaultdict(float)
        for (e, ph), pr in states.items():
            due = [i for i in range(n) if e[i] != NEVER and ph[i] is None and max(e[i] + tau_EI, 0) == t]
            for outcome in itertools.product((0, 1), repeat=len(due)):
                q = pr
                ph2 = list(ph)
                for i, f in zip(due, outcome):
                    q *= float(m[t]) if f else 1.0 - float(m[t])
                    ph2[i] = f
                if q > 0.0:
                    drawn[(e, tuple(ph2))] += q
        nxt = defaultdict(float)
        for (e, ph), pr in drawn.items():
            x = []
            for ej, fj in zip(e, ph):
                k = t - ej
                Lf = L_M if fj == 1 else L_R
                x.append(float(c[k]) if ej != NEVER and 1 <= k < Lf else 0.0)
            ED[t] += pr * sum(1 for ej, fj in zip(e, ph) if ej != NEVER and fj == 1 and t - ej == L_M)
            sus = [i for i in range(n) if e[i] == NEVER]
            p = {i: 1.0 - np.exp(-float(R[t]) * float(S_age[age[i]]) * sum(W[j][i] * x[j] for j in range(n)) / Dbar)
                 for i in sus}
            for outcome in itertools.product((0, 1), repeat=len(sus)):
                q = pr
                e2 = list(e)
                for i, hit in zip(sus, outcome):
                    q *= p[i] if hit else 1.0 - p[i]
                    if hit:
                        e2[i] = t
                if q > 0.0:
                    nxt[(tuple(e2), ph)] += q
        states = nxt
    return ED


@pytest.mark.parametrize("tau_IM", [2, 5])
def test_monte_carlo_matches_exact_law(tau_IM):
    """4 agents, fates below and above the recovery time: the sampled E[D_t] over 10k
    Philox keys lies within 5 sigma of the exact law."""
    import math
    pop, W = _tiny_graph()
    tau_EI, tau_IR, T = 1, 3, 10
    L = tau_EI + max(tau_IR, tau_IM)
    c = np.r_[0.0, np.full(L - 1, 0.5)].astype(np.float32)
    R = np.full(T, 3.0, np.float32)
    m = np.linspace(0.2, 0.7, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    e0 = np.array([-1, NEVER, NEVER, NEVER], np.int64)
    ED = _exact_fate_law(W, pop.age, S, c, tau_EI, tau_IR, tau_IM, R, m, e0)
    runs = 10_000
    Dsum = np.zeros(T); D2 = np.zeros(T)
    for s in range(runs):
        f = F.forward(pop, F.FateModel(tau_EI, tau_IR, tau_IM, c, seed=s), R, m, S, e0=e0)
        Dsum += f["D"]; D2 += f["D"] ** 2
    assert sum(ED) > 0.5
    for t in range(T):
        var = max(D2[t] / runs - (Dsum[t] / runs) ** 2, 1e-12)
        assert abs(Dsum[t] / runs - ED[t]) <= 5 * math.sqrt(var / runs) + 1e-12, (t, Dsum[t] / runs, ED[t])
