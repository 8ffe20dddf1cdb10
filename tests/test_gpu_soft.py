"""GPU fixed-noise soft relaxation against the FP64 oracle.

The soft model (every draw relaxed, y = sigmoid(logit p - logit u), mass flow
s -> n -> x) is smooth in the parameters, so its adjoint can be checked against
finite differences.  Bars: D and lambda within 1e-4 of the oracle (fp32
arithmetic over the horizon), the adjoint within 1e-3 of the oracle's soft
adjoint, and within 1e-2 of central differences of the oracle's soft loss.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import check_adjoint, ensure_built, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _soft_model(seed):
    return capi.ModelDesc(tau_EI=4, tau_IR=7, c=synth.infectiousness_table(), seed=seed,
                          relax_mode=capi.GABM_SOFT)


def _case(n=3000, T=25, seed=4, graph_seed=7):
    pop = synth.population_small(n=n, seed=graph_seed)
    rng = np.random.default_rng(seed)
    R = rng.uniform(2.0, 3.5, T).astype(np.float32)
    m = rng.uniform(0.005, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    y = synth.target_curve(T, pop.n, seed=seed, level=5e-5)
    return pop, R, m, S, y


def _gpu(pop, R, m, S, y, seed, n_seed):
    ctx = capi.gabm_create([pop], _soft_model(seed))
    Rd, md_, Sd, yd = to_dev(R[None], m[None], S[None], y[None])
    D, _ = capi.gabm_forward(ctx, R.size, Rd, md_, Sd, [n_seed])
    loss, gD = capi.gabm_mse_loss(ctx, yd)
    dR, dm, dS = capi.gabm_backward(ctx, gD)
    return ctx, D.cpu().numpy()[0], float(loss.cpu().numpy()[0]), dR.cpu().numpy()[0], dm.cpu().numpy()[0], \
        dS.cpu().numpy()[0]


def test_soft_forward_and_adjoint_match_oracle():
    pop, R, m, S, y = _case()
    md = O.Model(4, 7, synth.infectiousness_table(), seed=3)
    f = O.forward_soft(pop, md, R, m, S, n_seed=6)
    loss, gD = O.mse(f["D"], y)
    g = O.backward_soft(pop, md, R, m, S, gD, f["s_hist"], f["y_hist"], f["dydl_hist"], f["Lam_hist"], f["newRM"])
    ctx, D, loss_g, dR, dm, dS = _gpu(pop, R, m, S, y, 3, 6)
    assert np.allclose(D, f["D"], rtol=1e-4, atol=1e-6 * np.abs(f["D"]).max())
    assert loss_g == pytest.approx(loss, rel=1e-3)
    seeds = np.zeros(pop.n, bool)
    seeds[O.select_seeds(pop.n, 3, 0, 6)] = True
    for t in (0, 7, 24):
        lam = capi.gabm_get_lambda(ctx, t)[0].astype(np.float64)
        ref = float(R[t]) * S[pop.age].astype(np.float64) * f["Lam_hist"][t]
        # the seeds hold no susceptible mass: their lambda is reported as 0
        assert np.all(lam[seeds] == 0.0)
        nz = (ref > 0) & ~seeds
        assert nz.sum() > 10
        assert np.max(np.abs(lam[nz] - ref[nz]) / ref[nz]) < 1e-4
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    assert np.abs(g["dR"]).max() > 0
    # the soft state is masses: no exposure days to read or set, no integer counts
    with pytest.raises(capi.GabmError):
        capi.gabm_get_state(ctx)
    Rd, md_, Sd = to_dev(R[None], m[None], S[None])
    with pytest.raises(capi.GabmError):
        capi.gabm_forward(ctx, R.size, Rd, md_, Sd, [6], want_counts=True)


def test_soft_adjoint_matches_central_differences():
    """GPU adjoint of the soft loss vs central differences (Richardson-extrapolated) of the
    oracle's FP64 soft loss, for every R_t, every m_t and every S_a: within 1e-2."""
    pop, R, m, S, y = _case(n=2500, T=20, seed=5, graph_seed=8)
    md = O.Model(4, 7, synth.infectiousness_table(), seed=11)
    _, _, _, dR, dm, dS = _gpu(pop, R, m, S, y, 11, 5)

    def loss_at(name, idx, delta, base_vec):
        v = base_vec.copy()
        v[idx] = np.float32(float(base_vec[idx]) + delta)
        args = dict(R=R, m=m, S=S)
        args[name] = v
        f = O.forward_soft(pop, md, args["R"], args["m"], args["S"], n_seed=5)
        return O.mse(f["D"], y)[0]

    scale = max(np.abs(dR).max(), 1e-30)
    worst = 0.0
    for name, vec, an in (("R", R, dR), ("m", m, dm), ("S", S, dS)):
        for idx in range(vec.size):
            base = float(vec[idx])
            h = 2.0 ** (math.floor(math.log2(max(1.0, abs(base)))) - 12)   # exact in fp32
            d1 = (loss_at(name, idx, h, vec) - loss_at(name, idx, -h, vec)) / (2 * h)
            d2 = (loss_at(name, idx, 2 * h, vec) - loss_at(name, idx, -2 * h, vec)) / (4 * h)
            fd = (4 * d1 - d2) / 3
            ref = max(abs(fd), 1e-3 * (scale if name != "m" else max(np.abs(dm).max(), 1e-30)))
            err = abs(float(an[idx]) - fd) / ref
            worst = max(worst, err)
            assert err <= 1e-2, (name, idx, float(an[idx]), fd)
    assert worst < 1e-2


def test_soft_multi_graph_and_schedule_calls():
    """Uneven graphs in one soft ctx: each graph's D matches its own oracle run; the
    autotuner has one schedule here and keeps the results."""
    pops = [synth.population_small(n=n, seed=70 + i) for i, n in enumerate((1200, 2100))]
    T = 18
    rng = np.random.default_rng(3)
    R = rng.uniform(2.0, 3.5, (2, T)).astype(np.float32)
    m = rng.uniform(0.005, 0.05, (2, T)).astype(np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (2, 1)).astype(np.float32)
    ctx = capi.gabm_create(pops, _soft_model(2))
    Rd, md_, Sd = to_dev(R, m, S)
    D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [4, 7])
    D = D.cpu().numpy()
    md = O.Model(4, 7, synth.infectiousness_table(), seed=2)
    for g, pop in enumerate(pops):
        f = O.forward_soft(pop, md, R[g], m[g], S[g], n_seed=[4, 7][g], inst=g)
        assert np.allclose(D[g], f["D"], rtol=1e-4, atol=1e-6 * np.abs(f["D"]).max())
    capi.gabm_autotune(ctx, 1)
    D2, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [4, 7])
    assert np.array_equal(D2.cpu().numpy(), D)


def test_soft_table_adjoint():
    """dL/dc[k] of the soft relaxation: against the oracle's soft adjoint (1e-3) and
    against Richardson central differences of the oracle's soft loss in c[k] (1e-2)."""
    pop, R, m, S, y = _case(n=2500, T=22, seed=6, graph_seed=9)
    md = O.Model(4, 7, synth.infectiousness_table(), seed=13)
    f = O.forward_soft(pop, md, R, m, S, n_seed=5)
    _, gD = O.mse(f["D"], y)
    e0 = np.full(pop.n, capi.GABM_NEVER, np.int16)
    e0[O.select_seeds(pop.n, 13, 0, 5)] = -4
    g = O.backward_soft(pop, md, R, m, S, gD, f["s_hist"], f["y_hist"], f["dydl_hist"], f["Lam_hist"],
                        f["newRM"], e0=e0)
    ctx = capi.gabm_create([pop], _soft_model(13))
    Rd, md_, Sd, yd = to_dev(R[None], m[None], S[None], y[None])
    capi.gabm_forward(ctx, R.size, Rd, md_, Sd, [5])
    _, gDd = capi.gabm_mse_loss(ctx, yd)
    dc = capi.gabm_backward_table(ctx, gDd)[3].cpu().numpy()[0]
    assert dc[0] == 0.0 and np.abs(g["dc"][1:]).min() > 0
    check_adjoint(dc[1:], g["dc"][1:], "dc")
    for k in range(1, 11):
        base = float(md.c[k])
        h = 2.0 ** (math.floor(math.log2(max(1.0, abs(base)))) - 12)

        def L_at(delta):
            c = md.c.copy()
            c[k] = np.float32(base + delta)
            return O.mse(O.forward_soft(pop, O.Model(4, 7, c, seed=13), R, m, S, n_seed=5)["D"], y)[0]
        d1 = (L_at(h) - L_at(-h)) / (2 * h)
        d2 = (L_at(2 * h) - L_at(-2 * h)) / (4 * h)
        fd = (4 * d1 - d2) / 3
        assert abs(dc[k] - fd) <= 1e-2 * max(abs(fd), 1e-3 * np.abs(dc).max()), (k, dc[k], fd)
