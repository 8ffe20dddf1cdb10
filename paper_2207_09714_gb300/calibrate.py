"""Calibration of the simulator's parameters by gradient descent through the day loop
(C-GradABM: Sec. 3.2, Stages 2-4, and the C-GradABM baseline of Sec. 4.2).

* Parameters are tied within weeks: every day of week w uses R_w and m_w (App. C: one
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
        T_stage = torch.where(self.is_E, self.log_T[0].exp(), self.log_T[1].exp())
        raw = T_stage * self.log_iota.exp()
        return torch.cat([raw.new_zeros(1), raw / raw.sum()])

    def forward(self):
        R = self.log_R.exp()[:, self.week]
        m = torch.sigmoid(self.logit_m)[:, self.week]
        return R.float(), m.float(), self.table().float()


def cumulative_mse(D: torch.Tensor, y_cum: torch.Tensor) -> torch.Tensor:
    """Mean over instances and days of (sum_{s<=t} D_s - y_cum_t)^2 (Sec. 3.2, Stage 3)."""
    return ((torch.cumsum(D, dim=-1) - y_cum) ** 2).mean()


def calibrate(ctx: capi.GabmCtx, params: WeeklyParams, y_cum, S_age, n_seed, steps: int = 50,
              lr: float = 0.05, callback=None):
    """Adam on ``params`` against the cumulative deaths ``y_cum`` [I, T]; returns the loss
    of every step (the loss of the parameters before that step's update)."""
    opt = torch.optim.Adam([p for p in params.parameters() if p.requires_grad], lr=lr)
    y_cum = torch.as_tensor(y_cum, dtype=torch.float64, device=params.log_R.device)
    losses = []
    for step in range(steps):
        opt.zero_grad()
        R, m, c = params()
        D = TableFunction.apply(ctx, R, m, S_age, c, n_seed)
        loss = cumulative_mse(D, y_cum)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        if callback is not None:
            callback(step, losses[-1], params)
    return losses
