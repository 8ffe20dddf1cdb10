"""GPU parity of the straight-through adjoint against the FP64 oracle adjoint.

Bar: |gpu - oracle| <= 1e-3 * max(|oracle|, 1e-3 * max|oracle|) element by element
for dR_t, dm_t and dS_a.  The GPU replays the oracle's own trajectory (its final
exposure days) with GABM_RECOMPUTE, so no input of the oracle comes from the GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import EXACT_MARGIN, NEVER, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _setup(pop, T, seed, n_seed, R=2.5, m=0.02, rng_seed=0, inst=0):
    rng = np.random.default_rng(rng_seed)
    Rv = rng.uniform(0.8 * R, 1.2 * R, T).astype(np.float32)
    mv = rng.uniform(0.5 * m, 1.5 * m, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=seed)
    ref = O.forward_hard(pop, md_o, Rv, mv, S, n_seed=n_seed, inst=inst)
    y = synth.target_curve(T, pop.n, seed=rng_seed + 1, level=5e-5)
    loss, gD = O.mse(ref["D"], y)
    g = O.backward_hard(pop, md_o, Rv, mv, S, ref["e_final"], gD, inst=inst)
    return Rv, mv, S, md_o, ref, y, loss, gD, g


def _replay(pop, T, Rv, mv, S, seed, E, gD, order=capi.GABM_ORDER_COMMUNITY):
    ctx = capi.gabm_create([pop], model(seed=seed, policy=capi.GABM_RECOMPUTE, order=order))
    capi.gabm_set_state(ctx, T, E[None, :])
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    capi.gabm_forward(ctx, T, Rd, md_, Sd)
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS = capi.gabm_backward(ctx, gDd)
    return dR.cpu().numpy()[0], dm.cpu().numpy()[0], dS.cpu().numpy()[0]


def test_replay_adjoint_10k():
    pop = synth.population_small()
    T = 30
    Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=0, n_seed=20)
    dR, dm, dS = _replay(pop, T, Rv, mv, S, 0, ref["e_final"], gD)
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    assert np.abs(g["dR"]).max() > 0 and np.abs(g["dS"]).max() > 0


@pytest.mark.parametrize("order", [capi.GABM_ORDER_INPUT, capi.GABM_ORDER_BFS, capi.GABM_ORDER_COMMUNITY])
def test_replay_adjoint_agent_orders(order):
    pop = synth.population_small(n=4099, seed=3)
    T = 28
    Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=5, n_seed=10, R=2.8, rng_seed=2)
    dR, dm, dS = _replay(pop, T, Rv, mv, S, 5, ref["e_final"], gD, order=order)
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")


def test_replay_adjoint_directed_graph():
    """Asymmetric weights: the transpose gather runs over a separate source-sorted CSR."""
    pop = synth.random_directed(3000, 15.0, seed=8)
    T = 26
    Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=2, n_seed=25, R=3.0, rng_seed=4)
    dR, dm, dS = _replay(pop, T, Rv, mv, S, 2, ref["e_final"], gD)
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")


def test_store_and_recompute_are_bitwise_equal_and_match_oracle():
    """Free-running forward + loss + backward entirely on the GPU, for both lambda policies."""
    pop = synth.population_small(n=8000, seed=6)
    T = 30
    for seed in range(20):
        Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=seed, n_seed=20, R=2.6, rng_seed=seed)
        if ref["margin"] > EXACT_MARGIN:
            break
    assert ref["margin"] > EXACT_MARGIN
    outs = []
    for policy in (capi.GABM_STORE_LAMBDA, capi.GABM_RECOMPUTE):
        ctx = capi.gabm_create([pop], model(seed=seed, policy=policy))
        Rd, md_, Sd, yd = to_dev(Rv[None, :], mv[None, :], S[None, :], y[None, :])
        D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [20])
        lossd, gDd = capi.gabm_mse_loss(ctx, yd)
        assert np.allclose(D.cpu().numpy()[0], ref["D"], rtol=1e-15, atol=0)
        assert lossd.cpu().numpy()[0] == pytest.approx(loss, rel=1e-13)
        assert np.allclose(gDd.cpu().numpy()[0], gD, rtol=1e-13, atol=0)
        dR, dm, dS = capi.gabm_backward(ctx, gDd)
        outs.append([x.cpu().numpy()[0] for x in (dR, dm, dS)])
        check_adjoint(outs[-1][0], g["dR"], "dR")
        check_adjoint(outs[-1][1], g["dm"], "dm")
        check_adjoint(outs[-1][2], g["dS"], "dS")
        # a second backward of the same forward is bitwise identical
        dR2, _, dS2 = capi.gabm_backward(ctx, gDd)
        assert np.array_equal(dR2.cpu().numpy()[0], outs[-1][0])
        assert np.array_equal(dS2.cpu().numpy()[0], outs[-1][2])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_host_buffers_match_device_buffers():
    pop = synth.population_small(n=5000, seed=12)
    T = 25
    Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=1, n_seed=10)
    ctx = capi.gabm_create([pop], model(seed=1))
    Rd, md_, Sd, yd = to_dev(Rv[None, :], mv[None, :], S[None, :], y[None, :])
    D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    l1, g1 = capi.gabm_mse_loss(ctx, yd)
    d1 = [x.cpu().numpy() for x in capi.gabm_backward(ctx, g1)]
    Dh, _ = capi.gabm_forward(ctx, T, Rv[None, :], mv[None, :], S[None, :], [10])
    l2, g2 = capi.gabm_mse_loss(ctx, y[None, :])
    d2 = capi.gabm_backward(ctx, g2)
    assert np.array_equal(Dh, D.cpu().numpy()) and np.array_equal(l2, l1.cpu().numpy())
    for a, b in zip(d1, d2):
        assert np.array_equal(a, b)


def test_multi_graph_adjoint():
    pops = [synth.population_small(n=n, seed=20 + i) for i, n in enumerate((3000, 1234, 5001))]
    T = 24
    I = len(pops)
    rng = np.random.default_rng(9)
    R = rng.uniform(2.2, 3.2, (I, T)).astype(np.float32)
    m = rng.uniform(0.01, 0.04, (I, T)).astype(np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (I, 1)).astype(np.float32)
    refs, gDs, gs = [], [], []
    for gi, pop in enumerate(pops):
        md_o = O.Model(4, 7, synth.infectiousness_table(), seed=7)
        ref = O.forward_hard(pop, md_o, R[gi], m[gi], S[gi], n_seed=8, inst=gi)
        y = synth.target_curve(T, pop.n, seed=gi, level=5e-5)
        _, gD = O.mse(ref["D"], y)
        refs.append(ref); gDs.append(gD)
        gs.append(O.backward_hard(pop, md_o, R[gi], m[gi], S[gi], ref["e_final"], gD, inst=gi))
    ctx = capi.gabm_create(pops, model(seed=7, policy=capi.GABM_RECOMPUTE))
    E = np.concatenate([r["e_final"] for r in refs])
    capi.gabm_set_state(ctx, T, E[None, :])
    Rd, md_, Sd, gDd = to_dev(R, m, S, np.stack(gDs))
    capi.gabm_forward(ctx, T, Rd, md_, Sd)
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    for gi in range(I):
        check_adjoint(dR[gi], gs[gi]["dR"], f"dR[{gi}]")
        check_adjoint(dm[gi], gs[gi]["dm"], f"dm[{gi}]")
        check_adjoint(dS[gi], gs[gi]["dS"], f"dS[{gi}]")


def test_autograd_function():
    torch = torch_cuda()
    from paper_2207_09714_gb300.autograd import GabmFunction
    pop = synth.population_small(n=6000, seed=13)
    T = 30
    Rv, mv, S, md_o, ref, y, loss, gD, g = _setup(pop, T, seed=3, n_seed=15)
    ctx = capi.gabm_create([pop], model(seed=3))
    R = torch.tensor(Rv[None, :], device="cuda", requires_grad=True)
    m = torch.tensor(mv[None, :], device="cuda", requires_grad=True)
    Sa = torch.tensor(S[None, :], device="cuda", requires_grad=True)
    D = GabmFunction.apply(ctx, R, m, Sa, [15])
    yt = torch.tensor(y[None, :], device="cuda")
    L = ((D - yt) ** 2).mean()
    L.backward()
    if ref["margin"] > EXACT_MARGIN:
        assert L.item() == pytest.approx(loss, rel=1e-12)
        check_adjoint(R.grad.double().cpu().numpy()[0], g["dR"], "dR")
        check_adjoint(Sa.grad.double().cpu().numpy()[0], g["dS"], "dS")
    assert R.grad.dtype == torch.float32 and torch.isfinite(R.grad).all()


def test_state_errors_and_injected_allocation_failure(monkeypatch):
    pop = synth.population_small(n=500, seed=1)
    ctx = capi.gabm_create([pop], model())
    gD = np.zeros((1, 5))
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward(ctx, *to_dev(gD))
    assert ei.value.status == capi.GABM_ESTATE
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_mse_loss(ctx, *to_dev(gD))
    assert ei.value.status == capi.GABM_ESTATE
    # store policy cannot replay a state it did not simulate
    capi.gabm_set_state(ctx, 5, np.full((1, pop.n), capi.GABM_NEVER, np.int16))
    capi.gabm_forward(ctx, 5, *to_dev(np.ones((1, 5), np.float32), np.ones((1, 5), np.float32),
                                      np.ones((1, 9), np.float32)))
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward(ctx, *to_dev(gD))
    assert ei.value.status == capi.GABM_ESTATE
    # an allocation refused part-way through create leaves nothing behind
    torch = torch_cuda()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for after in (0, 3, 12):
        monkeypatch.setenv("GABM_FAIL_ALLOC_AFTER", str(after))
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_create([pop], model())
        assert ei.value.status == capi.GABM_ENOMEM
    monkeypatch.delenv("GABM_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    ok = capi.gabm_create([pop], model())
    cur, peak = capi.gabm_mem_stats(ok)
    assert 0 < cur <= peak


@pytest.fixture(scope="module")
def full_size_adjoint():
    pop = synth.population_typed(1_000_000, seed=0)
    T = 60
    R = np.full(T, 2.5, np.float32)
    m = np.full(T, 0.01, np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=0)
    ref = O.forward_hard(pop, md_o, R, m, S, n_seed=20)
    y = synth.target_curve(T, pop.n)
    loss, gD = O.mse(ref["D"], y)
    g = O.backward_hard(pop, md_o, R, m, S, ref["e_final"], gD)
    return pop, T, R, m, S, ref, y, loss, gD, g


def test_full_size_replay_adjoint(full_size_adjoint):
    pop, T, R, m, S, ref, y, loss, gD, g = full_size_adjoint
    dR, dm, dS = _replay(pop, T, R, m, S, 0, ref["e_final"], gD)
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")


def test_full_size_store_policy_pipeline(full_size_adjoint):
    """The benchmark's own call sequence (store policy, device buffers) at full size.

    At 1M agents x 60 days some draw lies within the kernel's fp32 error of its
    threshold on most seeds, so the GPU may take another trajectory than the oracle's
    run after such a near-tie (the lockstep tests hold each day's decisions to the
    flip rule).  The check is therefore made on the GPU's own trajectory, whatever it
    is: its deaths equal m_t times the exits that its final state implies, its loss
    gradient equals the oracle's MSE gradient of those deaths, and its adjoint equals
    the oracle's adjoint of that trajectory."""
    pop, T, R, m, S, ref, y, loss, gD, g = full_size_adjoint
    L = 11
    ctx = capi.gabm_create([pop], model(seed=0))
    Rd, md_, Sd, yd = to_dev(R[None, :], m[None, :], S[None, :], y[None, :])
    D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [20])
    E = capi.gabm_get_state(ctx)[0].astype(np.int64)
    exits = np.bincount(E[(E != NEVER) & (E + L >= 0) & (E + L < T)] + L, minlength=T)
    D_ref = m.astype(np.float64) * exits
    assert np.array_equal(D.cpu().numpy()[0], D_ref)
    loss_gpu, gDd = capi.gabm_mse_loss(ctx, yd)
    loss_ref, gD_ref = O.mse(D_ref, y)
    assert abs(float(loss_gpu.cpu().numpy().ravel()[0]) - loss_ref) <= 1e-12 * abs(loss_ref)
    assert np.allclose(gDd.cpu().numpy()[0], gD_ref, rtol=1e-12, atol=0)
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=0)
    g_own = O.backward_hard(pop, md_o, R, m, S, E.astype(np.int16), gDd.cpu().numpy()[0])
    check_adjoint(dR, g_own["dR"], "dR")
    check_adjoint(dm, g_own["dm"], "dm")
    check_adjoint(dS, g_own["dS"], "dS")
    assert np.abs(g_own["dR"]).max() > 0


def test_long_horizon_adjoint_beyond_fp32_range():
    """200 days at R = 1.3: the exact adjoint reaches ~1e42, beyond fp32.  The reverse sweep
    keeps each day's values at a power-of-two scale, so the GPU still matches the FP64 oracle."""
    pop = synth.population_small(n=3000, seed=3)
    T = 200
    Rv = np.full(T, 1.3, np.float32)
    mv = np.full(T, 0.02, np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=1)
    ref = O.forward_hard(pop, md_o, Rv, mv, S, n_seed=10)
    _, gD = O.mse(ref["D"], synth.target_curve(T, pop.n, seed=2, level=5e-5))
    g = O.backward_hard(pop, md_o, Rv, mv, S, ref["e_final"], gD)
    assert np.abs(g["dR"]).max() > 3.4e38          # the case the scaling exists for
    dR, dm, dS = _replay(pop, T, Rv, mv, S, 1, ref["e_final"], gD)
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
