"""The calibration workload (weekly-tied R and m, MSE on cumulative deaths, stage factors
and infectiousness profile of the table) on the GPU.

* Gradient parity: torch autograd through ``TableFunction`` against the FP64 oracle's
  adjoint of the same trajectory, mapped to the unconstrained parameters by the chain
  rule written out here in numpy (bar: the adjoint bar, 1e-3).
* The Adam loop lowers the loss on a target simulated from known parameters.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import calibrate, capi, synth

from helpers import EXACT_MARGIN, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _table_chain(c, raw, dc, tau_EI):
    """dL/dlog_T [2] and dL/dlog_iota [L-1] from dL/dc, for c = [0, raw / sum(raw)]."""
    s = raw.sum()
    d_raw = (dc[1:] - np.dot(dc[1:], c[1:])) / s
    g_raw = d_raw * raw                  # d/dlog of each raw entry
    k = np.arange(1, len(c))
    return np.array([g_raw[k < tau_EI].sum(), g_raw[k >= tau_EI].sum()]), g_raw


def test_calibration_gradient_matches_oracle():
    torch = torch_cuda()
    pop = synth.population_small(n=6000, seed=2)
    T, n_seed = 28, 20
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    y_cum = np.cumsum(synth.target_curve(T, pop.n, seed=3, level=5e-5))
    p = calibrate.WeeklyParams(1, T, R0=2.6, m0=0.02, T_E=0.6, T_I=1.1)
    with torch.no_grad():
        p.log_R[0] += torch.tensor([0.0, 0.1, -0.05, 0.15], dtype=torch.float64, device="cuda")
        p.logit_m[0] += torch.tensor([0.0, 0.2, -0.1, 0.1], dtype=torch.float64, device="cuda")
    R, m, c = p()
    R_np, m_np, c_np = (x.detach().cpu().numpy()[0] if x.dim() == 2 else x.detach().cpu().numpy()
                        for x in (R, m, c))
    # a Philox key whose trajectory has no near-tie draw, so the GPU reproduces it exactly
    for seed in range(30):
        md_o = O.Model(4, 7, c_np, seed=seed)
        f = O.forward_hard(pop, md_o, R_np, m_np, S, n_seed=n_seed)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN

    # oracle: loss on cumulative deaths, gD_t = sum_{s >= t} dL/dC_s, adjoint, chain rule
    C = np.cumsum(f["D"])
    dC = 2.0 * (C - y_cum) / T
    gD = np.cumsum(dC[::-1])[::-1]
    g = O.backward_hard(pop, md_o, R_np, m_np, S, f["e_final"], gD)
    week = np.arange(T) // 7
    R64 = np.exp(p.log_R.detach().cpu().numpy()[0])[week]
    m64 = 1.0 / (1.0 + np.exp(-p.logit_m.detach().cpu().numpy()[0]))[week]
    ref_R = np.bincount(week, g["dR"] * R64)
    ref_m = np.bincount(week, g["dm"] * m64 * (1.0 - m64))
    T_stage = np.where(np.arange(1, 11) < 4, np.exp(p.log_T[0].item()), np.exp(p.log_T[1].item()))
    raw = T_stage * np.exp(p.log_iota.detach().cpu().numpy())
    c64 = np.concatenate([[0.0], raw / raw.sum()])
    ref_T, ref_iota = _table_chain(c64, raw, g["dc"], 4)

    ctx = capi.gabm_create([pop], model(seed=seed))
    (Sd,) = to_dev(S[None, :])
    D = calibrate.TableFunction.apply(ctx, R, m, Sd, c, [n_seed])
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    loss = calibrate.cumulative_mse(D, torch.as_tensor(y_cum[None, :], device="cuda"))
    assert float(loss.detach()) == pytest.approx(np.mean((C - y_cum) ** 2), rel=1e-12)
    loss.backward()
    check_adjoint(p.log_R.grad.cpu().numpy()[0], ref_R, "log_R")
    check_adjoint(p.logit_m.grad.cpu().numpy()[0], ref_m, "logit_m")
    check_adjoint(p.log_T.grad.cpu().numpy(), ref_T, "log_T")
    check_adjoint(p.log_iota.grad.cpu().numpy(), ref_iota, "log_iota")
    assert np.abs(ref_T).min() > 0 and np.abs(ref_iota).max() > 0


def test_adam_calibration_lowers_the_loss():
    torch = torch_cuda()
    pop = synth.population_small(n=20000, seed=5)
    T, n_seed = 42, 30
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    (Sd,) = to_dev(S[None, :])
    ctx = capi.gabm_create([pop], model(seed=7))
    # target: a run at known weekly parameters
    truth = calibrate.WeeklyParams(1, T, R0=3.0, m0=0.03, T_E=0.4, T_I=1.2)
    with torch.no_grad():
        truth.log_R[0] += torch.linspace(0.2, -0.3, truth.log_R.shape[1], dtype=torch.float64, device="cuda")
        R, m, c = truth()
        y_cum = torch.cumsum(calibrate.TableFunction.apply(ctx, R, m, Sd, c, [n_seed]), dim=-1)
    p = calibrate.WeeklyParams(1, T, R0=2.0, m0=0.01)
    losses = calibrate.calibrate(ctx, p, y_cum, Sd, [n_seed], steps=40, lr=0.08)
    assert all(np.isfinite(losses))
    assert min(losses[-5:]) < 0.2 * losses[0], losses[::5]


def _outputs64(net, x):
    """DeepCalibration's outputs before its float32 cast: R [1, T], m [1, T], c [L] in FP64."""
    theta = net.net(x)
    return theta[:, net.week, 0], theta[:, net.week, 1], calibrate.table_from(net.log_T, net.log_iota, net.is_E)


def test_deep_calibration_gradient_matches_oracle():
    """DC-GradABM: the CalibNN weights' gradients through the simulator equal the network's
    vector-Jacobian product J^T g with the oracle's g = (dL/dR_t, dL/dm_t, dL/dc).

    The network runs in FP64 (on the host), so the only fp32 arithmetic between the two
    sides is the simulator's.  Each weight gradient is a sum over the entries of g; with
    every entry of g held to 1e-3 relative, the bar that follows for the sum is
    1e-3 * (|J|^T |g|) elementwise, which is 1e-3 relative wherever the sum does not cancel.
    The two sides run the network's FP64 backward in different orders (one pass over the
    graph against rows of J): a weight whose gradient is zero in exact arithmetic (the
    attention keys' bias, which the softmax cancels) carries FP64 rounding of the other
    terms, below 1e-12 of the largest gradient; that is added to the bar."""
    torch = torch_cuda()
    torch.manual_seed(0)
    pop = synth.population_small(n=6000, seed=4)
    T, n_seed = 21, 20
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    x = torch.as_tensor(calibrate.synthetic_features(np.full((1, T), 2.5), t_N=14, F=5, seed=1),
                        dtype=torch.float64)
    net = calibrate.DeepCalibration(5, T, R_bounds=(2.0, 3.5), m_bounds=(0.005, 0.05), hidden=16).double()
    R, m, c = net(x)
    R_np, m_np, c_np = R.detach().numpy()[0], m.detach().numpy()[0], c.detach().numpy()
    for seed in range(30):
        md_o = O.Model(4, 7, c_np, seed=seed)
        f = O.forward_hard(pop, md_o, R_np, m_np, S, n_seed=n_seed)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    y_cum = np.cumsum(synth.target_curve(T, pop.n, seed=5, level=5e-5))
    C = np.cumsum(f["D"])
    gD = np.cumsum((2.0 * (C - y_cum) / T)[::-1])[::-1]
    g = O.backward_hard(pop, md_o, R_np, m_np, S, f["e_final"], gD)
    params = [p for p in net.parameters() if p.requires_grad]
    # the Jacobian J [outputs, weights] of the network's FP64 outputs, one row per output
    outs = torch.cat([o.reshape(-1) for o in _outputs64(net, x)])
    g_vec = np.concatenate([g["dR"], g["dm"], g["dc"]])
    assert outs.numel() == g_vec.size
    J = np.stack([np.concatenate([(gr if gr is not None else torch.zeros_like(p)).numpy().ravel()
                                  for gr, p in zip(torch.autograd.grad(outs[k], params, retain_graph=True,
                                                                       allow_unused=True), params)])
                  for k in range(outs.numel())])
    flat_ref = J.T @ g_vec
    bound = np.abs(J).T @ np.abs(g_vec) + 1e-9 * np.abs(flat_ref).max()   # 1e-3 x this: see above
    ctx = capi.gabm_create([pop], model(seed=seed))
    (Sd,) = to_dev(S[None, :])
    D = calibrate.TableFunction.apply(ctx, R.cuda(), m.cuda(), Sd, c.cuda(), [n_seed])
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    calibrate.cumulative_mse(D, torch.as_tensor(y_cum[None, :], device="cuda")).backward()
    flat_gpu = np.concatenate([p.grad.detach().numpy().ravel() for p in params])
    assert np.abs(flat_ref).max() > 0
    check_adjoint(flat_gpu, flat_ref, "CalibNN weights", bound=bound)
    # most weights are not cancellation-dominated: there the bar is the plain relative one
    assert np.mean(np.abs(flat_ref) >= 0.1 * bound) > 0.5


def test_joint_deep_calibration_lowers_the_loss():
    """JDC-GradABM: one CalibNN shared by three counties of a multi-graph context."""
    torch = torch_cuda()
    torch.manual_seed(2)
    pops = [synth.population_small(n=n, seed=60 + i) for i, n in enumerate((12000, 8000, 15000))]
    G, T, n_seed = len(pops), 35, 25
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    (Sd,) = to_dev(S)
    ctx = capi.gabm_create(pops, model(seed=3))
    # each county's true weekly R curve, its deaths, and features derived from the curve
    weeks = np.arange(T) // 7
    R_true = np.stack([np.array([3.2, 2.8, 2.2, 1.8, 1.5])[weeks] * f for f in (1.0, 1.15, 0.9)])
    m_true = np.full((G, T), 0.03)
    with torch.no_grad():
        y_cum = torch.cumsum(calibrate.TableFunction.apply(
            ctx, torch.as_tensor(R_true, dtype=torch.float32, device="cuda"),
            torch.as_tensor(m_true, dtype=torch.float32, device="cuda"), Sd,
            torch.as_tensor(synth.infectiousness_table(), device="cuda"), [n_seed] * G), dim=-1)
    x = torch.as_tensor(calibrate.synthetic_features(R_true, t_N=T, F=5, seed=4), device="cuda")
    # (at lr = 0.02 the bounded outputs saturate within ten steps; the oracle, driven by the
    # same loop on the CPU, gives this configuration's curve: 143 -> 7.8 over 80 steps)
    net = calibrate.DeepCalibration(5, T, R_bounds=(1.0, 4.0), m_bounds=(0.005, 0.06), hidden=16,
                                    learn_table=False).cuda()
    losses = calibrate.calibrate(ctx, net, y_cum, Sd, [n_seed] * G, steps=80, lr=0.004, inputs=(x,))
    assert all(np.isfinite(losses))
    assert min(losses[-5:]) < 0.2 * losses[0], losses[::10]
