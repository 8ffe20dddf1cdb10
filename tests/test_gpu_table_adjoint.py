"""GPU parity of the infectiousness-table adjoint dL/dc[k] (gabm_backward_table)
against the FP64 oracle, on the oracle's own trajectories.

Bar: the adjoint bar of the other parameters, |gpu - oracle| <= 1e-3 * max(|oracle|,
1e-3 * max|oracle|) for k = 1..L-1, and dc[0] = 0 exactly.  dR, dm and dS from the same
call are bitwise those of gabm_backward.  Contexts with several sets per graph are
checked by the batched adjoint tests (test_gpu_batched.py), per instance.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import EXACT_MARGIN, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _oracle(pop, T, seed, n_seed, R=2.5, m=0.02, rng_seed=0, inst=0):
    rng = np.random.default_rng(rng_seed)
    Rv = rng.uniform(0.8 * R, 1.2 * R, T).astype(np.float32)
    mv = rng.uniform(0.5 * m, 1.5 * m, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=seed)
    ref = O.forward_hard(pop, md_o, Rv, mv, S, n_seed=n_seed, inst=inst)
    y = synth.target_curve(T, pop.n, seed=rng_seed + 1, level=5e-5)
    loss, gD = O.mse(ref["D"], y)
    g = O.backward_hard(pop, md_o, Rv, mv, S, ref["e_final"], gD, inst=inst)
    return Rv, mv, S, ref, gD, g


def _replay_table(pop, T, Rv, mv, S, seed, E, gD):
    ctx = capi.gabm_create([pop], model(seed=seed, policy=capi.GABM_RECOMPUTE))
    capi.gabm_set_state(ctx, T, E[None, :])
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    capi.gabm_forward(ctx, T, Rd, md_, Sd)
    (gDd,) = to_dev(gD[None, :])
    out = [x.cpu().numpy()[0] for x in capi.gabm_backward_table(ctx, gDd)]
    base = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    return out, base


def _check_table(dc, ref):
    assert dc[0] == 0.0 and ref[0] == 0.0
    assert np.abs(ref[1:]).max() > 0
    check_adjoint(dc[1:], ref[1:], "dc")


@pytest.mark.parametrize("directed", [False, True])
def test_table_adjoint_matches_oracle(directed):
    """Symmetric weights (the gather shares the forward's edges) and directed ones (a
    separate source-sorted copy)."""
    pop = synth.random_directed(3000, 15.0, seed=8) if directed else synth.population_small(n=6000, seed=2)
    T = 30
    Rv, mv, S, ref, gD, g = _oracle(pop, T, seed=3, n_seed=20, R=2.8, rng_seed=5)
    (dR, dm, dS, dc), base = _replay_table(pop, T, Rv, mv, S, 3, ref["e_final"], gD)
    _check_table(dc, g["dc"])
    for a, b in zip((dR, dm, dS), base):
        assert np.array_equal(a, b)


def test_table_adjoint_store_policy_and_host_buffers():
    """Free-running forward with stored lambdas; device and host outputs agree bitwise."""
    pop = synth.population_small(n=8000, seed=6)
    T = 28
    for seed in range(20):
        Rv, mv, S, ref, gD, g = _oracle(pop, T, seed=seed, n_seed=20, R=2.6, rng_seed=seed)
        if ref["margin"] > EXACT_MARGIN:
            break
    assert ref["margin"] > EXACT_MARGIN
    ctx = capi.gabm_create([pop], model(seed=seed, policy=capi.GABM_STORE_LAMBDA))
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [20])
    assert np.array_equal(capi.gabm_get_state(ctx)[0], ref["e_final"])
    (gDd,) = to_dev(gD[None, :])
    dev = [x.cpu().numpy()[0] for x in capi.gabm_backward_table(ctx, gDd)]
    _check_table(dev[3], g["dc"])
    host = [x[0] for x in capi.gabm_backward_table(ctx, gD[None, :])]
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)
    # the plain backward afterwards is unchanged (the table accumulation is off again)
    dR, _, _ = capi.gabm_backward(ctx, gDd)
    assert np.array_equal(dR.cpu().numpy()[0], dev[0])


def test_table_adjoint_multi_graph():
    pops = [synth.population_small(n=n, seed=40 + i) for i, n in enumerate((2500, 777, 4100))]
    T = 22
    rng = np.random.default_rng(9)
    G = len(pops)
    R = rng.uniform(2.2, 3.2, (G, T)).astype(np.float32)
    m = rng.uniform(0.01, 0.03, (G, T)).astype(np.float32)
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=4)
    E, gD, refs = [], np.zeros((G, T)), []
    for gi, pop in enumerate(pops):
        f = O.forward_hard(pop, md_o, R[gi], m[gi], S[gi], n_seed=8, inst=gi)
        _, gD[gi] = O.mse(f["D"], synth.target_curve(T, pop.n, seed=gi, level=5e-5))
        refs.append(O.backward_hard(pop, md_o, R[gi], m[gi], S[gi], f["e_final"], gD[gi], inst=gi))
        E.append(f["e_final"])
    ctx = capi.gabm_create(pops, model(seed=4, policy=capi.GABM_RECOMPUTE))
    capi.gabm_set_state(ctx, T, np.concatenate(E)[None, :])
    Rd, md_, Sd, gDd = to_dev(R, m, S, gD)
    capi.gabm_forward(ctx, T, Rd, md_, Sd)
    dc = capi.gabm_backward_table(ctx, gDd)[3].cpu().numpy()
    for gi in range(G):
        _check_table(dc[gi], refs[gi]["dc"])


def test_table_adjoint_long_horizon_and_short_horizon():
    """200 days (the adjoint beyond the fp32 range: per-day scales) and T = L + 1 = 12, the
    shortest horizon whose deaths depend on day-0 infections (there the seeds' day-0
    infectiousness, gathered after the sweep, is a large share of dc[tau_EI])."""
    pop = synth.population_small(n=3000, seed=3)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=1)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    for T, R in ((200, 1.3), (12, 3.0)):
        Rv = np.full(T, R, np.float32)
        mv = np.full(T, 0.02, np.float32)
        ref = O.forward_hard(pop, md_o, Rv, mv, S, n_seed=10)
        _, gD = O.mse(ref["D"], synth.target_curve(T, pop.n, seed=2, level=5e-5) + 1e-3)
        g = O.backward_hard(pop, md_o, Rv, mv, S, ref["e_final"], gD)
        (dR, dm, dS, dc), _ = _replay_table(pop, T, Rv, mv, S, 1, ref["e_final"], gD)
        _check_table(dc, g["dc"])


def test_set_infectiousness_validation_and_state():
    """An invalid table is refused and leaves the ctx as it was; a valid one invalidates the
    last trajectory until the next forward, which then uses the new table (it equals a
    ctx created with that table, bitwise)."""
    pop = synth.population_small(n=2000, seed=9)
    T = 15
    Rd, md_, Sd = to_dev(np.full((1, T), 2.8, np.float32), np.full((1, T), 0.02, np.float32),
                         synth.SUSCEPTIBILITY[None, :].astype(np.float32))
    ctx = capi.gabm_create([pop], model(seed=2))
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    e0 = capi.gabm_get_state(ctx)
    (gDd,) = to_dev(np.ones((1, T)))
    c = synth.infectiousness_table().copy()
    for bad in (np.r_[0.1, c[1:]], np.r_[c[:3], -0.5, c[4:]], np.r_[c[:5], np.nan, c[6:]]):
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_set_infectiousness(ctx, bad.astype(np.float32))
        assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(ValueError):
        capi.gabm_set_infectiousness(ctx, c[:5])
    capi.gabm_backward(ctx, gDd)                          # the refused tables changed nothing
    c2 = synth.infectiousness_table(T_E=0.2, T_I=1.3)
    capi.gabm_set_infectiousness(ctx, c2)
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward(ctx, gDd)
    assert ei.value.status == capi.GABM_ESTATE
    D1, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    ref = capi.gabm_create([pop], model(c=c2, seed=2))
    D2, _ = capi.gabm_forward(ref, T, Rd, md_, Sd, [10])
    assert np.array_equal(D1.cpu().numpy(), D2.cpu().numpy())
    assert np.array_equal(capi.gabm_get_state(ctx), capi.gabm_get_state(ref))
    assert not np.array_equal(capi.gabm_get_state(ctx), e0)
    a = [x.cpu().numpy() for x in capi.gabm_backward_table(ctx, gDd)]
    b = [x.cpu().numpy() for x in capi.gabm_backward_table(ref, gDd)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
