"""Exact enumeration of the hard model on tiny graphs (test infrastructure).

TEST INFRASTRUCTURE ONLY.  An independent restatement of the day update of
Sec. 3.1 (Eq. 1-3) for graphs of a handful of agents: instead of sampling, it
carries the exact probability of every reachable state through the days, by
enumerating every subset of susceptible agents that can be infected on a day
(each with probability p_i or 1 - p_i, independent given the start-of-day
state; App. A, A5/A6).  It uses a dense weight matrix and pure Python, and
shares no code with the C oracle, so the oracle's sampled trajectories can be
checked against the exact law.
"""
from __future__ import annotations

import itertools
import math
from collections import defaultdict

NEVER = 32767


def dense_weights(pop):
    """W[j][i] = weight of the interaction from j into i (row i of the CSR lists j)."""
    n = pop.n
    W = [[0.0] * n for _ in range(n)]
    rp = [int(x) for x in pop.rowptr]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            W[int(pop.col[p])][i] += float(pop.w[p])
    return W


def infection_probs(W, age, S_age, c, L, R_t, t, e):
    """p_i = 1 - exp(-lambda_i) for every susceptible agent of state e on day t."""
    n = len(e)
    total_w = sum(sum(row) for row in W)
    Dbar = total_w / n
    x = []
    for ej in e:
        k = t - ej if ej != NEVER else -1
        x.append(float(c[k]) if 1 <= k < L else 0.0)
    out = {}
    for i in range(n):
        if e[i] != NEVER:
            continue
        lam_sum = sum(W[j][i] * x[j] for j in range(n))
        lam = float(R_t) * float(S_age[age[i]]) * lam_sum / Dbar
        out[i] = 1.0 - math.exp(-lam)
    return out


def exact_law(pop, tau_EI, tau_IR, c, R, m, S_age, e0, T):
    """Exact distribution of the hard trajectory.

    Returns (ED, ED2, P_inf, final) where ED[t] = E[D_t], ED2[t] = E[D_t^2],
    P_inf[i] = P(agent i is ever infected by the end of day T-1) and ``final``
    maps each final state (tuple of exposure days) to its probability.
    """
    L = tau_EI + tau_IR
    W = dense_weights(pop)
    age = [int(a) for a in pop.age]
    n = pop.n
    states = {tuple(int(v) for v in e0): 1.0}
    ED = [0.0] * T
    ED2 = [0.0] * T
    for t in range(T):
        nxt = defaultdict(float)
        for e, pr in states.items():
            nrm = sum(1 for ei in e if ei != NEVER and t - ei == L)
            d = float(m[t]) * nrm
            ED[t] += pr * d
            ED2[t] += pr * d * d
            p = infection_probs(W, age, S_age, c, L, R[t], t, e)
            sus = sorted(p)
            for outcome in itertools.product((0, 1), repeat=len(sus)):
                q = pr
                e_new = list(e)
                for i, hit in zip(sus, outcome):
                    q *= p[i] if hit else (1.0 - p[i])
                    if hit:
                        e_new[i] = t
                if q > 0.0:
                    nxt[tuple(e_new)] += q
        states = nxt
    P_inf = [0.0] * n
    for e, pr in states.items():
        for i in range(n):
            if e[i] != NEVER and e[i] >= 0:
                P_inf[i] += pr
    return ED, ED2, P_inf, dict(states)
