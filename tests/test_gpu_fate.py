"""The sampled R/M split (a mortality stage with its own I->M time tau_IM, the fate drawn
at I entry) on the GPU against the FP64 oracle (oracle/fate.py).

Bars: the base model's.  On an oracle trajectory with no near-tie infection draw the GPU
reproduces the final state, the stage counts and the counted deaths exactly (the fate
draws compare the same fp32 uniform with the same fp32 m on both sides); the adjoint
(dR, dm, dS) is within 1e-3 of the oracle's elementwise (relative to max(|oracle|,
1e-3 max|oracle|)).
"""
import numpy as np
import pytest

import oracle as O
from oracle import fate as F
from paper_2207_09714_gb300 import capi, synth

from helpers import EXACT_MARGIN, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TAU_EI, TAU_IR = 4, 7


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _fate_model(tau_IM, seed, policy=capi.GABM_STORE_LAMBDA):
    c = synth.infectiousness_table(TAU_EI, max(TAU_IR, tau_IM))
    return (capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, tau_IM=tau_IM, c=c, seed=seed, lambda_policy=policy),
            F.FateModel(TAU_EI, TAU_IR, tau_IM, c, seed=seed))


def _params(T, rng_seed, R=2.6):
    rng = np.random.default_rng(rng_seed)
    return (rng.uniform(0.8 * R, 1.2 * R, T).astype(np.float32), rng.uniform(0.1, 0.4, T).astype(np.float32),
            synth.SUSCEPTIBILITY.astype(np.float32))


@pytest.mark.parametrize("tau_IM,T", [(4, 30), (10, 30), (4, 9), (10, 12), (7, 26)])
def test_trajectory_deaths_and_adjoint_match_oracle(tau_IM, T):
    """tau_IM below, above and equal to tau_IR; the short horizons end inside the seeds'
    windows (the days between their two possible exits)."""
    pop = synth.population_small(n=6000, seed=7)
    n_seed = 30
    Rv, mv, S = _params(T, 11 + tau_IM)
    for seed in range(30):
        md, mo = _fate_model(tau_IM, seed)
        f = F.forward(pop, mo, Rv, mv, S, n_seed=n_seed)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    assert f["D"].sum() > 0
    y = synth.target_curve(T, pop.n, seed=3, level=2e-4)
    _, gD = O.mse(f["D"], y)
    g = F.backward(pop, mo, Rv, mv, S, f["e_final"], gD)

    ctx = capi.gabm_create([pop], md)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    assert np.array_equal(D.cpu().numpy()[0], f["D"])
    assert np.array_equal(counts.cpu().numpy()[0], f["counts"])
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    assert np.abs(g["dm"]).max() > 0
    # when no exposure of day 0 or later can die within the horizon (T <= L_M), only the
    # seeds' deaths count and R cannot move them: dR = 0 on both sides
    assert (np.abs(g["dR"]).max() > 0) == (T > mo.L_M)
    # host buffers give the same numbers; a second sweep too
    host = capi.gabm_backward(ctx, gD[None, :])
    for a, b in zip((dR, dm, dS), host):
        assert np.array_equal(a, b[0])


def test_equal_times_all_fatal_is_the_base_model():
    """tau_IM = tau_IR and m = 1: every exit is a death, so the trajectory and D equal the
    base model's (D = 1 * newRM) bitwise."""
    pop = synth.population_small(n=8000, seed=2)
    T = 40
    Rv, _, S = _params(T, 4)
    mv = np.ones(T, np.float32)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    out = []
    for tau_IM in (0, TAU_IR):
        md = model(seed=5) if tau_IM == 0 else _fate_model(TAU_IR, 5)[0]
        ctx = capi.gabm_create([pop], md)
        D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [25], want_counts=True)
        out.append((capi.gabm_get_state(ctx), D.cpu().numpy(), counts.cpu().numpy()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert out[0][1].sum() > 100


def test_forward_from_a_set_state():
    """A mid-epidemic state set at day 15 (exposures of every age, some past their
    fate draw): the bitmap of day 15 and the days after follow the oracle's forward from
    the same state."""
    pop = synth.population_small(n=6000, seed=9)
    T, t0, tau_IM = 32, 15, 10
    Rv, mv, S = _params(T, 8, R=2.8)
    for seed in range(30):
        md, mo = _fate_model(tau_IM, seed)
        pre = F.forward(pop, mo, Rv[:t0], mv[:t0], S, n_seed=30)
        f = F.forward(pop, mo, Rv, mv, S, e0=pre["e_final"], t0=t0)
        if min(pre["margin"], f["margin"]) > EXACT_MARGIN:
            break
    assert min(pre["margin"], f["margin"]) > EXACT_MARGIN
    ctx = capi.gabm_create([pop], md)
    capi.gabm_set_state(ctx, t0, pre["e_final"][None, :])
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    assert np.array_equal(D.cpu().numpy()[0][t0:], f["D"][t0:])
    assert np.array_equal(counts.cpu().numpy()[0][t0:], f["counts"][t0:])
    assert f["D"][t0:].sum() > 0
    # the stored lambdas cover days t0..T-1 only
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward(ctx, to_dev(np.ones((1, T)))[0])
    assert ei.value.status == capi.GABM_ESTATE


def test_unsupported_and_invalid():
    pop = synth.population_small(n=500, seed=1)
    for policy, sets in ((capi.GABM_RECOMPUTE, 1), (capi.GABM_STORE_LAMBDA, 4)):
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_create([pop], _fate_model(9, 0, policy)[0], sets_per_graph=sets)
        assert ei.value.status == capi.GABM_EUNSUPPORTED
    md = _fate_model(9, 0)[0]
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create_bipartite(synth.population_bipartite(800, seed=1), md)
    assert ei.value.status == capi.GABM_EUNSUPPORTED
    bad = capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, tau_IM=-1, c=synth.infectiousness_table(), seed=0)
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create([pop], bad)
    assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(ValueError):   # the table must cover the longer window
        capi.gabm_create([pop], capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, tau_IM=9,
                                               c=synth.infectiousness_table(), seed=0))
    ctx = capi.gabm_create([pop], md)
    T = 12
    Rd, md_, Sd = to_dev(np.full((1, T), 2.5, np.float32), np.full((1, T), 0.2, np.float32),
                         synth.SUSCEPTIBILITY[None, :].astype(np.float32))
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward_table(ctx, to_dev(np.ones((1, T)))[0])
    assert ei.value.status == capi.GABM_EUNSUPPORTED


def test_several_graphs_and_graph_replay(monkeypatch):
    """Three graphs in one ctx, each following the oracle's run of its own instance (its own
    Dbar, seeds and Philox instance, dm from its own fate draws); CUDA-graph replay of the
    day loops equals eager launches bitwise."""
    pops = [synth.population_small(n=n, seed=30 + i) for i, n in enumerate((3000, 777, 4500))]
    G, T, n_seed, tau_IM = len(pops), 26, 12, 10
    rng = np.random.default_rng(31)
    R = rng.uniform(2.2, 3.2, (G, T)).astype(np.float32)
    m = rng.uniform(0.1, 0.4, (G, T)).astype(np.float32)
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    md, mo = _fate_model(tau_IM, 3)
    refs = [F.forward(pops[g], mo, R[g], m[g], S[g], n_seed=n_seed, inst=g) for g in range(G)]
    gD = np.stack([O.mse(refs[g]["D"], synth.target_curve(T, pops[g].n, seed=g, level=2e-4))[1] for g in range(G)])
    Rd, md_, Sd, gDd = to_dev(R, m, S, gD)
    out = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("GABM_CUDA_GRAPHS", graphs)
        ctx = capi.gabm_create(pops, md)
        D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed] * G)
        out.append([capi.gabm_get_state(ctx)[0], D.cpu().numpy()] +
                   [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    e, D, dR, dm, dS = out[0]
    off = np.concatenate([[0], np.cumsum([p.n for p in pops])])
    checked = 0
    for g in range(G):
        if refs[g]["margin"] <= EXACT_MARGIN:
            continue
        assert np.array_equal(e[off[g]:off[g + 1]], refs[g]["e_final"]), g
        assert np.array_equal(D[g], refs[g]["D"]), g
        ref = F.backward(pops[g], mo, R[g], m[g], S[g], refs[g]["e_final"], gD[g], inst=g)
        check_adjoint(dR[g], ref["dR"], f"dR[{g}]")
        check_adjoint(dm[g], ref["dm"], f"dm[{g}]")
        check_adjoint(dS[g], ref["dS"], f"dS[{g}]")
        checked += 1
    assert checked >= 2
