"""FP64 oracle of the sampled R/M split (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/, the package smoke check and the bench's
CPU baseline, never by the product path.

The base model (Sec. 3.1) sends every agent from I to a single RM exit at L = tau_EI +
tau_IR days after exposure and counts expected deaths D_t = m_t newRM(t).  Sec. 3.1 also
names a separate mortality stage with its own I->M time tau_IM.  This module restates the
hard model with that stage sampled per agent (the reading of the variant used here):

* an agent exposed on day d enters I on day t_I = d + tau_EI and draws its fate there:
  M with probability m_{t_I}, else R.  The draw is the Philox uniform v of the agent's
  caller id on day t_I, stream 1 (stream 0 is the infection draw): phi = [v < m_{t_I}].
  Agents exposed before day 0 whose t_I is negative draw on day 0 with m_0;
* an R-fated agent is infectious for k = t - d in [1, L_R), L_R = tau_EI + tau_IR; an
  M-fated one for k in [1, L_M), L_M = tau_EI + tau_IM; both with the table c[k] of
  L_max = max(L_R, L_M) entries (c[0] = 0);
* deaths are counted, not expected: D_t = #{M-fated agents with t - d = L_M}.

The fate of an exposure on day d is a function of the agent's id, d and m, so the final
exposure days still fix the whole trajectory (no reinfection, A3/A4 of App. A).

Adjoint (straight-through, App. B, with the fate draw relaxed like the infection draw,
phi_soft = sigmoid(logit m - logit v), tau = 1).  With gx_i(t) = dL/dx_i(t) and
c_phi[k] = c[k] [k < L_phi]:
  G_i(d) = dL/dn_i(d) = sum_k c_phi[k] gx_i(d + k) + phi gD_{d + L_M}
  H_i(d) = dL/dphi_i(d) = sum_{k in [L_min, L_max)} s c[k] gx_i(d + k) + gD_{d + L_M}
with s = +1 if L_M > L_R else -1; dm_{t_I} += H_i(E_i) dphi_soft/dm for every exposed
agent (seeds included); the infection-draw part is that of the base model with this G.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import NUM_AGES, select_seeds, uniform

NEVER = 32767
PAD = -32768


def _csr(pop):
    """A[i, j] = w of row i's entry for in-neighbour j (so Lam = A x / Dbar)."""
    n = pop.n
    rp = np.asarray(pop.rowptr, np.int64)
    return sp.csr_matrix((np.asarray(pop.w, np.float64), np.asarray(pop.col, np.int64), rp), shape=(n, n))


def _dbar(pop):
    return float(np.sum(np.asarray(pop.w, np.float64))) / pop.n


class FateModel:
    """Stage times tau_EI, tau_IR, tau_IM, the table c [L_max] and the Philox key."""

    def __init__(self, tau_EI: int, tau_IR: int, tau_IM: int, c, seed: int = 0):
        self.tau_EI, self.tau_IR, self.tau_IM = int(tau_EI), int(tau_IR), int(tau_IM)
        self.L_R = self.tau_EI + self.tau_IR
        self.L_M = self.tau_EI + self.tau_IM
        self.L = max(self.L_R, self.L_M)
        self.L_min = min(self.L_R, self.L_M)
        self.c = np.ascontiguousarray(c, dtype=np.float32)
        assert self.c.shape == (self.L,) and self.c[0] == 0.0
        self.seed = int(seed)


def _fate_day(md: FateModel, E):
    """I-entry day of an exposure on day E (day 0 for exposures before -tau_EI)."""
    return np.maximum(E.astype(np.int64) + md.tau_EI, 0)


def fates(md: FateModel, E, m, ids, inst: int = 0):
    """(phi, v, t_I): the fate of each agent's exposure on day E_i, its uniform and its draw
    day; phi = 0 and v = nan where E_i is NEVER or padding or t_I >= T (not drawn)."""
    m = np.asarray(m, np.float32)
    T = m.size
    E = np.asarray(E, np.int64)
    tI = _fate_day(md, E)
    drawn = (E != NEVER) & (E != PAD) & (tI < T)
    phi = np.zeros(E.size, bool)
    v = np.full(E.size, np.nan)
    for day in np.unique(tI[drawn]):
        sel = drawn & (tI == day)
        v[sel] = uniform(md.seed, ids[sel], int(day), inst, 1)
        phi[sel] = v[sel] < float(m[day])
    return phi, v, tI


def infectiousness(md: FateModel, t: int, E, phi):
    """x_i(t) = c[t - E_i] for t - E_i in [1, L_phi), else 0."""
    E = np.asarray(E, np.int64)
    k = t - E
    Lf = np.where(phi, md.L_M, md.L_R)
    on = (E != NEVER) & (E != PAD) & (k >= 1) & (k < Lf)
    x = np.zeros(E.size)
    x[on] = md.c[k[on]].astype(np.float64)
    return x


def forward(pop, md: FateModel, R, m, S_age, n_seed: int = 0, e0=None, t0: int = 0, inst: int = 0,
            orig_id=None):
    """Hard forward of days t0..T-1 (T = len(R)).  Returns e_final, D [T] (deaths counted on
    days t0..T-1), counts [T, 4] (S, E, I, RM at the start of each day), fate of the final
    state, and margin = min |u - p| over the infection draws."""
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
    Dbar = _dbar(pop)
    age = np.asarray(pop.age, np.int64)
    D = np.zeros(T)
    counts = np.zeros((T, 4), np.int64)
    margin = np.inf
    for t in range(t0, T):
        phi, _, _ = fates(md, e, m, ids, inst)
        exp_ = (e != NEVER)
        k = t - e
        Lf = np.where(phi, md.L_M, md.L_R)
        counts[t] = [np.sum(~exp_), np.sum(exp_ & (k < md.tau_EI)),
                     np.sum(exp_ & (k >= md.tau_EI) & (k < Lf)), np.sum(exp_ & (k >= Lf))]
        D[t] = np.sum(exp_ & phi & (k == md.L_M))
        Lam = (A @ infectiousness(md, t, e, phi)) / Dbar
        lam = float(R[t]) * S[age].astype(np.float64) * Lam
        p = -np.expm1(-lam)
        u = uniform(md.seed, ids, t, inst, 0)
        sus = ~exp_
        if sus.any():
            margin = min(margin, float(np.min(np.abs(u[sus] - p[sus]))))
        e[sus & (u < p)] = t
    phi, _, _ = fates(md, e, m, ids, inst)
    return dict(e_final=e.astype(np.int16), D=D, counts=counts, fate=phi, margin=margin)


def dy_dlambda(lam, u):
    """d y_soft / d lambda of y_soft = p (1-u) / (p (1-u) + (1-p) u), p = 1 - exp(-lambda)."""
    q = np.exp(-lam)
    p = -np.expm1(-lam)
    den = p * (1.0 - u) + q * u
    return u * (1.0 - u) * q / (den * den)


def dphi_dm(m, v):
    """d phi_soft / d m of phi_soft = m (1-v) / (m (1-v) + (1-m) v)."""
    den = m * (1.0 - v) + (1.0 - m) * v
    return v * (1.0 - v) / (den * den)


def backward(pop, md: FateModel, R, m, S_age, E, gD, inst: int = 0, orig_id=None):
    """Straight-through adjoint of the trajectory the final state E encodes (days 0..T-1).
    Returns dR [T], dm [T], dS [9]."""
    R = np.asarray(R, np.float32); m = np.asarray(m, np.float32); S = np.asarray(S_age, np.float32)
    gD = np.asarray(gD, np.float64)
    T = R.size
    n = pop.n
    ids = np.arange(n, dtype=np.uint32) if orig_id is None else np.asarray(orig_id, np.uint32)
    E = np.asarray(E, np.int64)
    A = _csr(pop)
    AT = A.T.tocsr()
    Dbar = _dbar(pop)
    age = np.asarray(pop.age, np.int64)
    Sa = S[age].astype(np.float64)
    agent = E != PAD
    seed_row = agent & (E != NEVER) & (E < 0)
    phi_E, v_E, tI_E = fates(md, E, m, ids, inst)   # the exposures that happened
    sgn = 1.0 if md.L_M > md.L_R else -1.0

    def gDat(d):
        return gD[d] if 0 <= d < T else 0.0

    gx = np.zeros((T + 1, n))        # gx[t] = dL/dx(t); gx[T] = 0
    r_next = np.zeros(n)             # r(t+1)
    Aacc = np.zeros(n)               # A_i = G_i(E_i)
    dR = np.zeros(T); dm = np.zeros(T); dS = np.zeros(NUM_AGES)
    for t in range(T - 1, -1, -1):
        gx[t + 1] = AT @ r_next if t + 1 < T else 0.0
        # state on day t and the hypothetical fate of an exposure today
        sus = agent & ~seed_row & ((E == NEVER) | (E >= t))
        phi_t = np.zeros(n, bool)
        if t + md.tau_EI < T:
            v_t = uniform(md.seed, ids, t + md.tau_EI, inst, 1)
            phi_t = v_t < float(m[t + md.tau_EI])
        Lf = np.where(phi_t, md.L_M, md.L_R)
        G = np.where(phi_t, gDat(t + md.L_M), 0.0)
        H = np.full(n, gDat(t + md.L_M))
        for k in range(1, md.L):
            if t + k > T:
                break
            ck = float(md.c[k])
            G += np.where(k < Lf, ck * gx[t + k], 0.0)
            if k >= md.L_min:
                H += sgn * ck * gx[t + k]
        # the draw of today's infections
        x_t = infectiousness(md, t, E, phi_E)
        Lam = (A @ x_t) / Dbar
        lam = float(R[t]) * Sa * Lam
        u = uniform(md.seed, ids, t, inst, 0)
        exp_today = sus & (E == t)
        dy = np.where(exp_today | (E == NEVER), G, G - Aacc)
        Aacc = np.where(exp_today, G, Aacc)
        glam = np.where(sus, dy * dy_dlambda(lam, u), 0.0)
        r_cur = float(R[t]) * Sa * glam / Dbar
        v = glam * Lam
        dR[t] = np.sum(Sa * v)
        for a in range(NUM_AGES):
            dS[a] += float(R[t]) * np.sum(v[age == a])
        # the fate draws of today's exposures (on day t + tau_EI)
        fd = exp_today & (t + md.tau_EI < T)
        if fd.any():
            dm[t + md.tau_EI] += np.sum(H[fd] * dphi_dm(float(m[t + md.tau_EI]), v_E[fd]))
        r_next = r_cur
    gx[0] = AT @ r_next
    # the fate draws of agents exposed before day 0
    for i in np.flatnonzero(seed_row & (tI_E < T)):
        Ei = int(E[i])
        H = gDat(Ei + md.L_M)
        for k in range(md.L_min, md.L):
            if 0 <= Ei + k < T:
                H += sgn * float(md.c[k]) * gx[Ei + k, i]
        dm[tI_E[i]] += H * dphi_dm(float(m[tI_E[i]]), v_E[i])
    return dict(dR=dR, dm=dm, dS=dS)
