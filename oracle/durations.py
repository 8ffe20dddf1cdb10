"""FP64 oracle of stochastic I-stage durations (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/, the package smoke check and the bench's
CPU baseline, never by the product path.

The base model (Sec. 3.1) gives every agent the same stage times.  Sec. 6 names
stochastic progression as an extension; the variant restated here draws each agent's
infectious period (reading of the variant used here):

* an agent exposed on day d stays in E for tau_EI days and in I for j days, j drawn from
  a given pmf p_IR over 1..tau_IR: j = the first j with u < F_j, F_j = p_IR[0] + ... +
  p_IR[j-1] summed in order in FP64 (tau_IR if none), u the Philox uniform of the agent's
  caller id on day max(d, 0), stream 2;
* it is infectious for 1 <= t - d < L_i = tau_EI + j with the table c[k] (L = tau_EI +
  tau_IR entries), and enters RM at t - d = L_i;
* deaths are the Aggregate's expected ones, D_t = m_t newRM(t).

The draw depends only on the agent and its exposure day, so the final exposure days
still fix the trajectory (no reinfection, A3/A4 of App. A).  The durations carry no
parameter, so the straight-through adjoint (App. B) is the base model's with each row's
own window: G_i(d) = sum_{k < L_i(d)} c[k] gx_i(d + k) + m_{d + L_i(d)} gD_{d + L_i(d)},
L_i(d) the duration an exposure of agent i on day d would draw; dm_t = gD_t newRM(t).
A pmf with all its mass on tau_IR is the base model.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import NUM_AGES, select_seeds, uniform

NEVER = 32767
PAD = -32768


class DurationModel:
    """tau_EI, the longest I stage tau_IR, its pmf p_IR [tau_IR] (entry j-1: P(j days)),
    the table c [tau_EI + tau_IR] and the Philox key."""

    def __init__(self, tau_EI: int, tau_IR: int, p_IR, c, seed: int = 0):
        self.tau_EI, self.tau_IR = int(tau_EI), int(tau_IR)
        self.L = self.tau_EI + self.tau_IR
        self.p_IR = np.asarray(p_IR, np.float32)
        assert self.p_IR.shape == (self.tau_IR,)
        F = np.zeros(self.tau_IR)
        acc = 0.0
        for j in range(self.tau_IR):          # in order, FP64
            acc += float(self.p_IR[j])
            F[j] = acc
        self.F = F
        self.c = np.ascontiguousarray(c, dtype=np.float32)
        assert self.c.shape == (self.L,) and self.c[0] == 0.0
        self.seed = int(seed)


def exit_offsets(md: DurationModel, ids, d, inst: int = 0):
    """L_i = tau_EI + j_i for exposures of agents ``ids`` on days ``d`` (array)."""
    ids = np.asarray(ids, np.uint32)
    d = np.asarray(d, np.int64)
    out = np.zeros(ids.size, np.int64)
    key = np.maximum(d, 0)
    for day in np.unique(key):
        sel = key == day
        u = uniform(md.seed, ids[sel], int(day), inst, 2)
        j = 1 + np.searchsorted(md.F, u, side="right")
        out[sel] = md.tau_EI + np.minimum(j, md.tau_IR)
    return out


def _csr(pop):
    n = pop.n
    return sp.csr_matrix((np.asarray(pop.w, np.float64), np.asarray(pop.col, np.int64),
                          np.asarray(pop.rowptr, np.int64)), shape=(n, n))


def _exits_of_state(md, E, ids, inst):
    """Exit offset of every exposed agent's actual exposure (L for the rest, unused)."""
    E = np.asarray(E, np.int64)
    Lx = np.full(E.size, md.L, np.int64)
    exp_ = (E != NEVER) & (E != PAD)
    if exp_.any():
        Lx[exp_] = exit_offsets(md, ids[exp_], E[exp_], inst)
    return Lx


def forward(pop, md: DurationModel, R, m, S_age, n_seed: int = 0, e0=None, t0: int = 0, inst: int = 0,
            orig_id=None):
    """Hard forward of days t0..T-1; returns e_final, D, counts [T, 4], newRM, margin."""
    R = np.asarray(R, np.float32); m = np.asarray(m, np.float32); S = np.asarray(S_age, np.float32)
    T = R.size
    n = pop.n
    ids = np.arange(n, dtype=np.uint32) if orig_id is None else np.asarray(orig_id, np.uint32)
    if e0 is None:
        e = np.full(n, NEVER, np.int64)
        e[select_seeds(n, md.seed, inst, n_seed, orig_id)] = -md.tau_EI
    else:
        e = np.asarray(e0, np.int64).copy()
    A = _csr(pop)
    Dbar = float(np.sum(np.asarray(pop.w, np.float64))) / n
    age = np.asarray(pop.age, np.int64)
    D = np.zeros(T); newRM = np.zeros(T, np.int64)
    counts = np.zeros((T, 4), np.int64)
    margin = np.inf
    for t in range(t0, T):
        Lx = _exits_of_state(md, e, ids, inst)
        exp_ = e != NEVER
        k = t - e
        counts[t] = [np.sum(~exp_), np.sum(exp_ & (k < md.tau_EI)),
                     np.sum(exp_ & (k >= md.tau_EI) & (k < Lx)), np.sum(exp_ & (k >= Lx))]
        newRM[t] = np.sum(exp_ & (k == Lx))
        D[t] = float(m[t]) * newRM[t]
        on = exp_ & (k >= 1) & (k < Lx)
        x = np.zeros(n)
        x[on] = md.c[k[on]].astype(np.float64)
        Lam = (A @ x) / Dbar
        lam = float(R[t]) * S[age].astype(np.float64) * Lam
        p = -np.expm1(-lam)
        u = uniform(md.seed, ids, t, inst, 0)
        sus = ~exp_
        if sus.any():
            margin = min(margin, float(np.min(np.abs(u[sus] - p[sus]))))
        e[sus & (u < p)] = t
    return dict(e_final=e.astype(np.int16), D=D, newRM=newRM, counts=counts, margin=margin)


def backward(pop, md: DurationModel, R, m, S_age, E, gD, inst: int = 0, orig_id=None):
    """Straight-through adjoint of the trajectory E encodes; returns dR [T], dm [T], dS [9]."""
    R = np.asarray(R, np.float32); m = np.asarray(m, np.float32); S = np.asarray(S_age, np.float32)
    gD = np.asarray(gD, np.float64)
    T = R.size
    n = pop.n
    ids = np.arange(n, dtype=np.uint32) if orig_id is None else np.asarray(orig_id, np.uint32)
    E = np.asarray(E, np.int64)
    A = _csr(pop)
    AT = A.T.tocsr()
    Dbar = float(np.sum(np.asarray(pop.w, np.float64))) / n
    age = np.asarray(pop.age, np.int64)
    Sa = S[age].astype(np.float64)
    agent = E != PAD
    seed_row = agent & (E != NEVER) & (E < 0)
    exp_ = agent & (E != NEVER)
    Lx_E = _exits_of_state(md, E, ids, inst)

    gx = np.zeros((T + 1, n))
    r_next = np.zeros(n)
    Aacc = np.zeros(n)
    dR = np.zeros(T); dS = np.zeros(NUM_AGES)
    newRM = np.zeros(T)
    for t in range(T - 1, -1, -1):
        gx[t + 1] = AT @ r_next if t + 1 < T else 0.0
        newRM[t] = np.sum(exp_ & (t - E == Lx_E))
        sus = agent & ~seed_row & ((E == NEVER) | (E >= t))
        Lt = exit_offsets(md, ids, np.full(n, t), inst)    # the window an exposure today would have
        G = np.zeros(n)
        tail = t + Lt
        has_tail = tail < T
        G[has_tail] = m[tail[has_tail]].astype(np.float64) * gD[tail[has_tail]]
        for k in range(1, md.L):
            if t + k > T:
                break
            G += np.where(k < Lt, float(md.c[k]) * gx[t + k], 0.0)
        on = exp_ & (t - E >= 1) & (t - E < Lx_E)
        x = np.zeros(n)
        x[on] = md.c[(t - E)[on]].astype(np.float64)
        Lam = (A @ x) / Dbar
        lam = float(R[t]) * Sa * Lam
        u = uniform(md.seed, ids, t, inst, 0)
        q = np.exp(-lam); p = -np.expm1(-lam)
        den = p * (1.0 - u) + q * u
        dydl = u * (1.0 - u) * q / (den * den)
        exp_today = sus & (E == t)
        dy = np.where(exp_today | (E == NEVER), G, G - Aacc)
        Aacc = np.where(exp_today, G, Aacc)
        glam = np.where(sus, dy * dydl, 0.0)
        v = glam * Lam
        dR[t] = np.sum(Sa * v)
        for a in range(NUM_AGES):
            dS[a] += float(R[t]) * np.sum(v[age == a])
        r_next = float(R[t]) * Sa * glam / Dbar
    dm = gD * newRM
    return dict(dR=dR, dm=dm, dS=dS, newRM=newRM)
