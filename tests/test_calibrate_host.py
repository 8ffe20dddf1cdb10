"""Host-side pieces of the calibration workload: the weekly tying and the table
parameterisation (no GPU)."""
import numpy as np
import torch

from paper_2207_09714_gb300 import calibrate, synth


def test_default_table_is_the_model_table():
    p = calibrate.WeeklyParams(2, 30, device="cpu")
    c = p.table().detach().numpy()
    ref = synth.infectiousness_table(4, 7, T_E=0.5, T_I=1.0)
    assert c[0] == 0.0
    assert np.allclose(c, ref, rtol=2e-7, atol=1e-9)
    assert abs(c.sum() - 1.0) < 1e-12


def test_weekly_tying_and_parameter_maps():
    p = calibrate.WeeklyParams(3, 23, R0=2.0, m0=0.02, device="cpu")
    with torch.no_grad():
        p.log_R[1, 2] = np.log(3.0)
        p.logit_m[2, 3] = np.log(0.05 / 0.95)
    R, m, c = p()
    assert R.shape == (3, 23) and m.shape == (3, 23) and c.shape == (11,)
    assert R.dtype == torch.float32
    assert torch.all(R[1, 14:21] == 3.0) and torch.all(R[1, :14] == 2.0) and torch.all(R[1, 21:] == 2.0)
    assert torch.allclose(m[2, 21:], torch.tensor(0.05)) and torch.allclose(m[2, :21], torch.tensor(0.02))


def test_stage_factors_change_only_their_stage():
    p = calibrate.WeeklyParams(1, 7, device="cpu")
    c0 = p.table().detach().numpy()
    with torch.no_grad():
        p.log_T[0] += np.log(2.0)          # T_E doubled
    c1 = p.table().detach().numpy()
    raw = c0.copy()
    raw[1:4] *= 2.0                        # k < tau_EI = 4 are the E days
    assert np.allclose(c1, raw / raw.sum(), rtol=1e-12)


def test_cumulative_mse():
    D = torch.tensor([[1.0, 2.0, 0.0]], dtype=torch.float64)
    y = torch.tensor([[1.0, 2.0, 4.0]], dtype=torch.float64)
    # cumulative D = 1, 3, 3 against 1, 2, 4
    assert float(calibrate.cumulative_mse(D, y)) == (0 + 1 + 1) / 3


def test_calibnn_bounds_and_shapes():
    torch.manual_seed(0)
    net = calibrate.CalibNN(in_features=5, steps=6, lower=[0.5, 0.001], upper=[6.0, 0.1], hidden=16)
    x = torch.randn(3, 20, 5) * 10.0
    theta = net(x)
    assert theta.shape == (3, 6, 2)
    assert torch.all(theta[..., 0] >= 0.5) and torch.all(theta[..., 0] <= 6.0)
    assert torch.all(theta[..., 1] >= 0.001) and torch.all(theta[..., 1] <= 0.1)
    # instances are independent: one instance's output does not depend on another's features
    x2 = x.clone()
    x2[1] += 1.0
    t2 = net(x2)
    assert torch.equal(t2[0], theta[0]) and torch.equal(t2[2], theta[2]) and not torch.equal(t2[1], theta[1])


def test_deep_calibration_weekly_parameters():
    torch.manual_seed(1)
    T = 30
    dc = calibrate.DeepCalibration(in_features=4, T=T, hidden=8)
    x = torch.randn(2, 12, 4)
    R, m, c = dc(x)
    assert R.shape == (2, T) and m.shape == (2, T) and c.shape == (11,)
    for w in range(5):
        days = slice(7 * w, min(T, 7 * w + 7))
        assert torch.all(R[:, days] == R[:, days][:, :1]) and torch.all(m[:, days] == m[:, days][:, :1])
    assert np.allclose(c.detach().numpy(), synth.infectiousness_table(), rtol=2e-7, atol=1e-9)


def test_synthetic_features_follow_the_curve():
    R_t = np.stack([np.linspace(3.0, 1.0, 40), np.full(40, 2.0)])
    x = calibrate.synthetic_features(R_t, t_N=30, F=5, seed=3)
    assert x.shape == (2, 30, 5) and x.dtype == np.float32
    assert np.array_equal(x, calibrate.synthetic_features(R_t, t_N=30, F=5, seed=3))
    # the unlagged channel tracks R_t: falling for instance 0, flat for instance 1
    assert np.polyfit(np.arange(30), x[0, :, 0], 1)[0] < -0.02
    assert abs(np.polyfit(np.arange(30), x[1, :, 0], 1)[0]) < 0.02
