"""FP64 oracle of SIRS reinfection (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and, once a GPU path exists, the package
smoke check and the bench's CPU baseline), never by the product path.

App. A's A4 (no infection from RM) can be relaxed for diseases such as influenza.
The variant restated here (the reading used for it) returns every agent to S
tau_RS days after it enters RM:

* exposed on day d, an agent is in E for k = t - d < tau_EI, in I for k < L = tau_EI +
  tau_IR (infectious with c[k], k >= 1), in RM for k < L + tau_RS, and susceptible again
  from k = L + tau_RS on, when it can be exposed anew (its last exposure day is the state,
  as in the state vector of Sec. 3.1);
* the infection draw of day t is the Philox uniform of (caller id, t, instance, stream
  0), so an agent draws again on every susceptible day;
* deaths are the Aggregate's expected ones, D_t = m_t newRM(t), newRM counting every
  I -> RM transition.

The final state no longer encodes the trajectory: an agent exposed twice keeps only
its last exposure day.  The forward therefore returns every agent's exposure history,
and the adjoint reads it.

Adjoint (straight-through, App. B).  The mass returning to S on day t + 1 is the mass
exposed on day t + 1 - L - tau_RS, so with B_i(t) = dL/ds_i(t):
  G_i(d) = dL/dn_i(d) = sum_{k=1}^{L-1} c[k] gx_i(d + k) + m_{d+L} gD_{d+L} + B_i(d + L + tau_RS)
  B_i(t) = y_i(t) G_i(t) + (1 - y_i(t)) B_i(t+1),  B_i(T) = 0
  dL/dy_i(t) = s_i(t) (G_i(t) - B_i(t+1))
and the rest is the base model's.  With tau_RS >= T nobody returns within the horizon
and this is the base model.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import NUM_AGES, select_seeds, uniform

NEVER = 32767


class SirsModel:
    """tau_EI, tau_IR, tau_RS (days in RM before S again), the table c [L] and the key."""

    def __init__(self, tau_EI: int, tau_IR: int, tau_RS: int, c, seed: int = 0):
        self.tau_EI, self.tau_IR, self.tau_RS = int(tau_EI), int(tau_IR), int(tau_RS)
        self.L = self.tau_EI + self.tau_IR
        self.cycle = self.L + self.tau_RS
        self.c = np.ascontiguousarray(c, dtype=np.float32)
        assert self.c.shape == (self.L,) and self.c[0] == 0.0
        self.seed = int(seed)


def _csr(pop):
    n = pop.n
    return sp.csr_matrix((np.asarray(pop.w, np.float64), np.asarray(pop.col, np.int64),
                          np.asarray(pop.rowptr, np.int64)), shape=(n, n))


def _susceptible(md, e, t):
    k = t - e
    return (e == NEVER) | (k >= md.cycle)


def _infectiousness(md, e, t):
    k = t - e
    on = (e != NEVER) & (k >= 1) & (k < md.L)
    x = np.zeros(e.size)
    x[on] = md.c[k[on]].astype(np.float64)
    return x


def forward(pop, md: SirsModel, R, m, S_age, n_seed: int = 0, inst: int = 0, e0=None):
    """Hard forward of days 0..T-1 from the seeded state (or the day-0 state e0: exposure
    days before day 0, or NEVER).  Returns e_final (last exposure
    days), exposures (list of (day, agent) in order), e_hist [T+1, n] (the state at the
    start of each day), D, newRM, counts [T, 4] (S, E, I, RM) and margin."""
    R = np.asarray(R, np.float32); m = np.asarray(m, np.float32); S = np.asarray(S_age, np.float32)
    T = R.size
    n = pop.n
    ids = np.arange(n, dtype=np.uint32)
    if e0 is None:
        e = np.full(n, NEVER, np.int64)
        e[select_seeds(n, md.seed, inst, n_seed)] = -md.tau_EI
    else:
        e = np.asarray(e0, np.int64).copy()
    A = _csr(pop)
    Dbar = float(np.sum(np.asarray(pop.w, np.float64))) / n
    age = np.asarray(pop.age, np.int64)
    D = np.zeros(T); newRM = np.zeros(T, np.int64); counts = np.zeros((T, 4), np.int64)
    e_hist = np.zeros((T + 1, n), np.int64)
    margin = np.inf
    for t in range(T):
        e_hist[t] = e
        k = t - e
        sus = _susceptible(md, e, t)
        counts[t] = [np.sum(sus), np.sum(~sus & (k < md.tau_EI)), np.sum(~sus & (k >= md.tau_EI) & (k < md.L)),
                     np.sum(~sus & (k >= md.L))]
        newRM[t] = np.sum((e != NEVER) & (k == md.L))
        D[t] = float(m[t]) * newRM[t]
        Lam = (A @ _infectiousness(md, e, t)) / Dbar
        lam = float(R[t]) * S[age].astype(np.float64) * Lam
        p = -np.expm1(-lam)
        u = uniform(md.seed, ids, t, inst, 0)
        if sus.any():
            margin = min(margin, float(np.min(np.abs(u[sus] - p[sus]))))
        e[sus & (u < p)] = t
    e_hist[T] = e
    return dict(e_final=e, e_hist=e_hist, D=D, newRM=newRM, counts=counts, margin=margin)


def backward(pop, md: SirsModel, R, m, S_age, e_hist, gD, inst: int = 0):
    """Straight-through adjoint of the trajectory whose daily states are e_hist [T+1, n]
    (from ``forward``).  Returns dR [T], dm [T], dS [9]."""
    R = np.asarray(R, np.float32); m = np.asarray(m, np.float32); S = np.asarray(S_age, np.float32)
    gD = np.asarray(gD, np.float64)
    T = R.size
    n = pop.n
    ids = np.arange(n, dtype=np.uint32)
    A = _csr(pop)
    AT = A.T.tocsr()
    Dbar = float(np.sum(np.asarray(pop.w, np.float64))) / n
    age = np.asarray(pop.age, np.int64)
    Sa = S[age].astype(np.float64)
    gx = np.zeros((T + 1, n))
    B = np.zeros((T + 1, n))            # B[t] = dL/ds(t); B[T] = 0
    r_next = np.zeros(n)
    dR = np.zeros(T); dS = np.zeros(NUM_AGES); newRM = np.zeros(T)
    for t in range(T - 1, -1, -1):
        gx[t + 1] = AT @ r_next if t + 1 < T else 0.0
        e = e_hist[t]
        sus = _susceptible(md, e, t)
        y = sus & (e_hist[t + 1] == t)   # exposed today
        newRM[t] = np.sum((e != NEVER) & (t - e == md.L))
        G = np.zeros(n)
        if t + md.L < T:
            G += float(m[t + md.L]) * gD[t + md.L]
        if t + md.cycle <= T:
            G += B[t + md.cycle]
        for k in range(1, md.L):
            if t + k > T:
                break
            G += float(md.c[k]) * gx[t + k]
        dy = np.where(sus, G - B[t + 1], 0.0)
        B[t] = np.where(y, G, B[t + 1])
        Lam = (A @ _infectiousness(md, e, t)) / Dbar
        lam = float(R[t]) * Sa * Lam
        u = uniform(md.seed, ids, t, inst, 0)
        q = np.exp(-lam); p = -np.expm1(-lam)
        den = p * (1.0 - u) + q * u
        glam = dy * (u * (1.0 - u) * q / (den * den))
        v = glam * Lam
        dR[t] = np.sum(Sa * v)
        for a in range(NUM_AGES):
            dS[a] += float(R[t]) * np.sum(v[age == a])
        r_next = float(R[t]) * Sa * glam / Dbar
    return dict(dR=dR, dm=gD * newRM, dS=dS)
