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
