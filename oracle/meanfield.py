"""Mean-field limits of the hard model on a complete graph (test infrastructure).

TEST INFRASTRUCTURE ONLY.  On a complete graph with unit weights and a
single susceptibility, every susceptible agent sees the same force of
infection, so the expected dynamics reduce to a compartmental recurrence: the
SEIRM-type model of App. D (the SurrogateODE baseline) with the deterministic
stage delays of Sec. 3.1 in place of exponential ones.  Two consequences are
used to pin the oracle:

* the discrete-time recurrence for the expected number newly exposed per day,
  new_t = S_t (1 - exp(-(R / (n-1)) sum_k c[k] new_{t-k})), seeds at -tau_EI;
* the final-size relation of the Kermack-McKendrick type for that recurrence,
  1 - z = (1 - i0) exp(-R (n z - n_seed kappa) / (n - 1)), where kappa is the
  share of a seed's infectiousness spent before day 0 (sum of c[1..tau_EI-1]).
"""
from __future__ import annotations

import math

import numpy as np


def daily_recurrence(n: int, R: float, c, tau_EI: int, tau_IR: int, n_seed: int, T: int):
    """Expected newly exposed per day and the I-stage occupancy at the start of each day."""
    L = tau_EI + tau_IR
    c = [float(v) for v in c]
    exposed = {-tau_EI: float(n_seed)}
    S = float(n - n_seed)
    new = np.zeros(T)
    I = np.zeros(T)
    E = np.zeros(T)
    for t in range(T):
        I[t] = sum(exposed.get(t - k, 0.0) for k in range(tau_EI, L))
        E[t] = sum(exposed.get(t - k, 0.0) for k in range(1, tau_EI))
        force = sum(c[k] * exposed.get(t - k, 0.0) for k in range(1, L))
        nt = S * (1.0 - math.exp(-(R / (n - 1)) * force))
        exposed[t] = nt
        new[t] = nt
        S -= nt
    return new, E, I


def final_size(n: int, R: float, c, tau_EI: int, n_seed: int) -> float:
    """Solve 1 - z = (1 - i0) exp(-R (n z - n_seed kappa) / (n - 1)) for the attack rate z."""
    from scipy.optimize import brentq

    kappa = float(sum(float(v) for v in c[1:tau_EI]))
    i0 = n_seed / n

    def f(z):
        return 1.0 - z - (1.0 - i0) * math.exp(-R * (n * z - n_seed * kappa) / (n - 1))

    return brentq(f, i0 + 1e-12, 1.0)
