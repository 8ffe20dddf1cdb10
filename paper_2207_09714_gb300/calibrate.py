"""Calibration of the simulator's parameters by gradient descent through the day loop:
C-GradABM (Sec. 3.2, Stages 2-4, and the C-GradABM baseline of Sec. 4.2), and DC- / JDC-
GradABM, where a calibration network (CalibNN, App. C) maps feature time series to the
parameters and is trained through the simulator (one network per county, or one shared by
all the counties of a multi-graph context).

* Parameters are tied within weeks: every day of week w uses R_w and m_w (App. D: one
  parameter set for every 7 days).
* The loss is the mean-squared error of the cumulative deaths (Sec. 3.2, Stage 3).
* Gradients come from the library's straight-through adjoint (App. B): R_t, m_t, S_a,
  and the adjoint of the infectiousness table c[k] (``gabm_backward_table``), which
  reaches the stage factors T_E, T_I and the daily profile iota that define the table
  through c[k] = T_stage(k) iota(k) / sum_j T_stage(j) iota(j), k = 1..L-1, c[0] = 0
  (the form of Sec. 3.1, normalised to sum 1).
* The optimiser is Adam (torch) on unconstrained parameters: log R, logit m, log T,
  log iota.

Every step runs one forward and one backward of the whole horizon on the GPU; the
parameter maps, the cumulative sum and the loss are small torch operations.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import capi


class TableFunction(torch.autograd.Function):
    """``TableFunction.apply(ctx, R, m, S_age, c, n_seed) -> D``.

    Like ``GabmFunction`` but the infectiousness table c [L] is an input too: the forward
    installs it in the ctx (``gabm_set_infectiousness``, skipped when unchanged) and the
    backward returns dL/dc from ``gabm_backward_table``, summed over the ctx's instances
    (they share the table).  R, m: [I, T] float32 CUDA; S_age: [I, 9]; D: [I, T] float64.
    """

    @staticmethod
    def forward(fctx, handle, R, m, S_age, c, n_seed):
        c_host = c.detach().to(torch.float32).cpu().numpy()
        if not np.array_equal(c_host, np.asarray(handle.model.c, np.float32)):
            capi.gabm_set_infectiousness(handle, c_host)
        T = int(R.shape[-1])
        D, _ = capi.gabm_forward(handle, T, R.detach().contiguous(), m.detach().contiguous(),
                                 S_age.detach().contiguous(), n_seed)
        fctx.handle = handle
        fctx.meta = (R.dtype, m.dtype, S_age.dtype, c.dtype, c.device)
        return D

    @staticmethod
    def backward(fctx, gD):
        dR, dm, dS, dc = capi.gabm_backward_table(fctx.handle, gD.detach().to(torch.float64).contiguous())
        tR, tm, tS, tc, dev = fctx.meta
        return None, dR.to(tR), dm.to(tm), dS.to(tS), dc.sum(0).to(device=dev, dtype=tc), None


def gamma_profile(L: int, shape: float = 3.0, scale: float = 2.0) -> np.ndarray:
    """iota(k) for k = 0..L-1: the mass of a Gamma(shape, scale) on (k-1, k], iota(0) = 0."""
    from scipy.special import gammainc

    k = np.arange(L, dtype=np.float64)
    cdf = gammainc(shape, k / scale)
    iota = np.zeros(L)
    iota[1:] = np.diff(cdf)
    return iota


def table_from(log_T: torch.Tensor, log_iota: torch.Tensor, is_E: torch.Tensor) -> torch.Tensor:
    """c = [0, T_stage(k) iota(k) / sum_j T_stage(j) iota(j)] for k = 1..L-1 (is_E[k-1]: day k
    is in the E stage)."""
    T_stage = torch.where(is_E, log_T[0].exp(), log_T[1].exp())
    raw = T_stage * log_iota.exp()
    return torch.cat([raw.new_zeros(1), raw / raw.sum()])


class WeeklyParams(torch.nn.Module):
    """Weekly-tied (R, m) for I instances over T days and the table parameters (T_E, T_I,
    iota) shared by all of them.  ``forward()`` returns (R [I, T], m [I, T], c [L]) as
    float32 tensors on ``device``."""

    def __init__(self, instances: int, T: int, tau_EI: int = 4, tau_IR: int = 7, R0: float = 2.5,
                 m0: float = 0.01, T_E: float = 0.5, T_I: float = 1.0, iota=None, learn_table: bool = True,
                 device="cuda"):
        super().__init__()
        self.T, self.tau_EI, self.L = int(T), int(tau_EI), int(tau_EI + tau_IR)
        W = (self.T + 6) // 7
        iota = gamma_profile(self.L) if iota is None else np.asarray(iota, np.float64)
        if iota.shape != (self.L,) or np.any(iota[1:] <= 0):
            raise ValueError("iota must have L entries, positive for k >= 1")
        f64 = dict(dtype=torch.float64, device=device)
        self.log_R = torch.nn.Parameter(torch.full((instances, W), math.log(R0), **f64))
        self.logit_m = torch.nn.Parameter(torch.full((instances, W), math.log(m0 / (1 - m0)), **f64))
        self.log_T = torch.nn.Parameter(torch.tensor([math.log(T_E), math.log(T_I)], **f64),
                                        requires_grad=learn_table)
        self.log_iota = torch.nn.Parameter(torch.tensor(np.log(iota[1:]), **f64), requires_grad=learn_table)
        self.register_buffer("week", torch.arange(self.T, device=device) // 7)
        self.register_buffer("is_E", torch.arange(1, self.L, device=device) < self.tau_EI)

    def table(self) -> torch.Tensor:
        return table_from(self.log_T, self.log_iota, self.is_E)

    def forward(self):
        R = self.log_R.exp()[:, self.week]
        m = torch.sigmoid(self.logit_m)[:, self.week]
        return R.float(), m.float(), self.table().float()


class CalibNN(torch.nn.Module):
    """The calibration network of App. C: a GRU encodes the feature series x^t (t0..tN)
    into h^t; scaled dot-product self-attention over the h^t, summed over t, gives the
    context u; a GRU decoder started from u reads the positional codes tau_k = k/K
    (k = 1..K) and a feed-forward head maps each output o^k to parameters bounded as
    theta = theta_L + (theta_U - theta_L) * sigmoid(FFN(o^k)).

    forward(x [I, t_N, F]) -> theta [I, K, P]."""

    def __init__(self, in_features: int, steps: int, lower, upper, hidden: int = 32):
        super().__init__()
        self.steps = int(steps)
        self.register_buffer("lower", torch.as_tensor(lower, dtype=torch.float32))
        self.register_buffer("upper", torch.as_tensor(upper, dtype=torch.float32))
        n_out = int(self.lower.numel())
        self.encoder = torch.nn.GRU(in_features, hidden, batch_first=True)
        self.q = torch.nn.Linear(hidden, hidden)
        self.k = torch.nn.Linear(hidden, hidden)
        self.v = torch.nn.Linear(hidden, hidden)
        self.decoder = torch.nn.GRU(1, hidden, batch_first=True)
        self.head = torch.nn.Sequential(torch.nn.Linear(hidden, hidden), torch.nn.ReLU(),
                                        torch.nn.Linear(hidden, n_out))

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        h, _ = self.encoder(x)                                           # [I, tN, H]
        att = torch.softmax(self.q(h) @ self.k(h).transpose(1, 2) / math.sqrt(h.shape[-1]), dim=-1)
        u = (att @ self.v(h)).sum(dim=1)                                 # context [I, H]
        tau = torch.arange(1, self.steps + 1, dtype=x.dtype, device=x.device) / self.steps
        o, _ = self.decoder(tau.expand(x.shape[0], -1).unsqueeze(-1), u.unsqueeze(0).contiguous())
        return self.lower + (self.upper - self.lower) * torch.sigmoid(self.head(o))


class DeepCalibration(torch.nn.Module):
    """DC-GradABM (one instance) or JDC-GradABM (several instances, one shared network):
    CalibNN maps each instance's features to weekly (R_w, m_w); the infectiousness table
    (T_E, T_I, iota) is shared and learned directly.  forward(x [I, t_N, F]) -> (R [I, T],
    m [I, T], c [L]) float32."""

    def __init__(self, in_features: int, T: int, tau_EI: int = 4, tau_IR: int = 7, R_bounds=(0.5, 6.0),
                 m_bounds=(0.001, 0.1), hidden: int = 32, T_E: float = 0.5, T_I: float = 1.0, iota=None,
                 learn_table: bool = True):
        super().__init__()
        self.T, self.L = int(T), int(tau_EI + tau_IR)
        W = (self.T + 6) // 7
        self.net = CalibNN(in_features, W, [R_bounds[0], m_bounds[0]], [R_bounds[1], m_bounds[1]], hidden)
        iota = gamma_profile(self.L) if iota is None else np.asarray(iota, np.float64)
        self.log_T = torch.nn.Parameter(torch.tensor([math.log(T_E), math.log(T_I)], dtype=torch.float64),
                                        requires_grad=learn_table)
        self.log_iota = torch.nn.Parameter(torch.tensor(np.log(iota[1:]), dtype=torch.float64),
                                           requires_grad=learn_table)
        self.register_buffer("week", torch.arange(self.T) // 7)
        self.register_buffer("is_E", torch.arange(1, self.L) < int(tau_EI))

    def forward(self, x: torch.Tensor):
        theta = self.net(x)                                              # [I, W, 2]
        R = theta[:, self.week, 0]
        m = theta[:, self.week, 1]
        return R.float(), m.float(), table_from(self.log_T, self.log_iota, self.is_E).float()


def synthetic_features(R_t: np.ndarray, t_N: int, F: int = 5, seed: int = 0) -> np.ndarray:
    """Seeded synthetic feature series [I, t_N, F] standing in for the CalibNN inputs of
    Sec. 4.1 (claims, surveys, line lists): noisy, lagged and scaled views of each
    instance's reproduction-number curve R_t [I, T] plus pure-noise channels."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 700]))
    I, T = R_t.shape
    out = np.empty((I, t_N, F), np.float32)
    for f in range(F):
        if f < F - 1:
            lag = f
            idx = np.clip(np.arange(t_N) - lag, 0, T - 1)
            out[:, :, f] = (R_t[:, idx] * rng.uniform(0.5, 1.5) + rng.normal(0, 0.1, (I, t_N)))
        else:
            out[:, :, f] = rng.normal(0, 1, (I, t_N))
    return out


def cumulative_mse(D: torch.Tensor, y_cum: torch.Tensor) -> torch.Tensor:
    """Mean over instances and days of (sum_{s<=t} D_s - y_cum_t)^2 (Sec. 3.2, Stage 3)."""
    return ((torch.cumsum(D, dim=-1) - y_cum) ** 2).mean()


def calibrate(ctx: capi.GabmCtx, params: torch.nn.Module, y_cum, S_age, n_seed, steps: int = 50,
              lr: float = 0.05, callback=None, inputs=()):
    """Adam on ``params`` (a module returning (R, m, c) from ``inputs``: ``WeeklyParams``
    with none, ``DeepCalibration`` with the features) against the cumulative deaths
    ``y_cum`` [I, T], averaged over instances (JDC: one loss for all counties); returns the
    loss of every step (the loss of the parameters before that step's update)."""
    opt = torch.optim.Adam([p for p in params.parameters() if p.requires_grad], lr=lr)
    y_cum = torch.as_tensor(y_cum, dtype=torch.float64, device=S_age.device)
    losses = []
    for step in range(steps):
        opt.zero_grad()
        R, m, c = params(*inputs)
        D = TableFunction.apply(ctx, R, m, S_age, c, n_seed)
        loss = cumulative_mse(D, y_cum)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        if callback is not None:
            callback(step, losses[-1], params)
    return losses
