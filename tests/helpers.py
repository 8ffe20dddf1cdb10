"""Shared helpers of the GPU parity tests: build the CUDA library once, make
contexts and run the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2207_09714_gb300 import capi, synth

NEVER = capi.GABM_NEVER

# lambda relative tolerance and flip rule of the forward parity bar
LAM_RTOL = 1e-5
FLIP_MARGIN = 1e-6
FLIP_FRACTION = 1e-5
# an oracle run whose every draw has |u - p| above this is reproduced exactly by the GPU
# (fp32 lambda error ~1e-6 relative moves p by far less)
EXACT_MARGIN = 1e-6
# adjoint bar (spec: 1e-3 relative), element by element: |gpu - oracle| <= ADJ_RTOL * |oracle|
# for every element, and an oracle zero must be a GPU zero.  For a quantity that is a linear map
# W = J^T g of the simulator's adjoint g (network weights, chain-rule parameter maps), the bar
# that the elementwise 1e-3 on g implies is ADJ_RTOL * (|J|^T |g|) elementwise: pass it as `bound`.
ADJ_RTOL = 1e-3

_built = False


def ensure_built():
    global _built
    if not _built:
        from paper_2207_09714_gb300 import build
        build.build()
        _built = True
    return capi.load_library()


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def model(c=None, tau_EI=4, tau_IR=7, seed=0, policy=capi.GABM_STORE_LAMBDA, order=capi.GABM_ORDER_COMMUNITY):
    if c is None:
        c = synth.infectiousness_table(tau_EI, tau_IR)
    return capi.ModelDesc(tau_EI=tau_EI, tau_IR=tau_IR, c=np.asarray(c, np.float32), seed=seed,
                          lambda_policy=policy, agent_order=order)


def to_dev(*arrays):
    torch = torch_cuda()
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def check_adjoint(gpu, orc, what="", bound=None):
    """Elementwise adjoint bar; returns the largest |gpu - orc| / (ADJ_RTOL-scaled bound)."""
    gpu = np.asarray(gpu, np.float64)
    orc = np.asarray(orc, np.float64)
    assert gpu.shape == orc.shape, what
    assert np.all(np.isfinite(gpu)), what
    ref = np.abs(orc) if bound is None else np.asarray(bound, np.float64)
    assert np.all(ref >= np.abs(orc) * (1 - 1e-12)), (what, "bound below |oracle|")
    err = np.abs(gpu - orc)
    bad = err > ADJ_RTOL * ref
    assert not bad.any(), (what, np.flatnonzero(bad)[:10], gpu[bad][:5], orc[bad][:5])
    nz = ref > 0
    return float(np.max(err[nz] / ref[nz])) if nz.any() else 0.0


def oracle_day(pop, md_o, t, R_t, S, e_in, inst=0):
    return O.day_hard(pop, md_o, t, R_t, S, e_in, inst=inst)


def compare_day(pop, md_o, ctx, t, R, S, e_start, inst_slice=slice(None), inst=0):
    """One lockstep day: GPU from the oracle's start-of-day state vs the oracle's day.

    Returns (max lambda relative error, flips, S agents)."""
    ref = O.day_hard(pop, md_o, t, float(R[t]), S, e_start, inst=inst)
    lam_gpu = capi.gabm_get_lambda(ctx, t)[0][inst_slice].astype(np.float64)
    e_gpu = capi.gabm_get_state(ctx)[0][inst_slice]
    sus = e_start == NEVER
    lam_ref = float(R[t]) * S[pop.age].astype(np.float64) * ref["Lam"]
    rel = np.abs(lam_gpu[sus] - lam_ref[sus]) / np.maximum(np.abs(lam_ref[sus]), 1e-30)
    rel[lam_ref[sus] == 0] = np.abs(lam_gpu[sus][lam_ref[sus] == 0])
    assert np.all(lam_gpu[~sus] == 0.0)
    diff = e_gpu != ref["e_out"]
    if diff.any():
        assert np.all(np.abs(ref["u"][diff] - ref["p"][diff]) < FLIP_MARGIN), "flip away from a near-tie"
        assert np.all(sus[diff])
    return float(rel.max() if rel.size else 0.0), int(diff.sum()), int(sus.sum())
