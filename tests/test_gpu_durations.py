"""Stochastic I-stage durations (a per-agent infectious period drawn from a pmf) on the
GPU against the FP64 oracle (oracle/durations.py).

Bars: the base model's.  On an oracle trajectory with no near-tie infection draw the GPU
reproduces the final state, the stage counts and D = m newRM exactly (the duration draws
compare the same fp32 uniform with the same FP64 running sums on both sides); the adjoint
(dR, dm, dS) is within 1e-3 of the oracle's elementwise.  A pmf with all its mass on
tau_IR gives bitwise the base model's forward and adjoint.
"""
import numpy as np
import pytest

import oracle as O
from oracle import durations as DU
from paper_2207_09714_gb300 import capi, synth

from helpers import EXACT_MARGIN, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TAU_EI, TAU_IR = 4, 9
PMF = np.array([0.02, 0.05, 0.13, 0.2, 0.2, 0.15, 0.12, 0.08, 0.05], np.float32)


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _models(p, seed, policy=capi.GABM_STORE_LAMBDA):
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    return (capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, seed=seed, lambda_policy=policy, p_IR=p),
            DU.DurationModel(TAU_EI, TAU_IR, p, c, seed=seed))


def _params(T, rng_seed, R=2.6):
    rng = np.random.default_rng(rng_seed)
    return (rng.uniform(0.8 * R, 1.2 * R, T).astype(np.float32), rng.uniform(0.01, 0.05, T).astype(np.float32),
            synth.SUSCEPTIBILITY.astype(np.float32))


@pytest.mark.parametrize("T", [30, 11])
def test_trajectory_and_adjoint_match_oracle(T):
    pop = synth.population_small(n=6000, seed=8)
    Rv, mv, S = _params(T, 20 + T)
    for seed in range(30):
        md, mo = _models(PMF, seed)
        f = DU.forward(pop, mo, Rv, mv, S, n_seed=30)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    assert f["newRM"].sum() > 0
    _, gD = O.mse(f["D"], synth.target_curve(T, pop.n, seed=2, level=5e-5))
    g = DU.backward(pop, mo, Rv, mv, S, f["e_final"], gD)
    ctx = capi.gabm_create([pop], md)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [30], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    assert np.array_equal(counts.cpu().numpy()[0], f["counts"])
    assert np.array_equal(D.cpu().numpy()[0], f["D"])
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    assert np.abs(g["dR"]).max() > 0 and np.abs(g["dm"]).max() > 0


def test_point_mass_is_bitwise_the_base_model():
    pop = synth.population_small(n=8000, seed=3)
    T = 40
    Rv, mv, S = _params(T, 5)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    (gDd,) = to_dev(np.linspace(-1, 1, T)[None, :])
    p = np.zeros(TAU_IR, np.float32)
    p[-1] = 1.0
    out = []
    for mdl in (model(tau_IR=TAU_IR, seed=6), _models(p, 6)[0]):
        ctx = capi.gabm_create([pop], mdl)
        D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [25], want_counts=True)
        out.append([capi.gabm_get_state(ctx), D.cpu().numpy(), counts.cpu().numpy()] +
                   [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert out[0][1].sum() > 0


def test_forward_from_a_set_state():
    pop = synth.population_small(n=6000, seed=10)
    T, t0 = 34, 16
    Rv, mv, S = _params(T, 9, R=2.8)
    for seed in range(30):
        md, mo = _models(PMF, seed)
        pre = DU.forward(pop, mo, Rv[:t0], mv[:t0], S, n_seed=30)
        f = DU.forward(pop, mo, Rv, mv, S, e0=pre["e_final"], t0=t0)
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
    assert f["newRM"][t0:].sum() > 0


def test_unsupported_and_invalid():
    pop = synth.population_small(n=500, seed=1)
    for policy, sets in ((capi.GABM_RECOMPUTE, 1), (capi.GABM_STORE_LAMBDA, 4)):
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_create([pop], _models(PMF, 0, policy)[0], sets_per_graph=sets)
        assert ei.value.status == capi.GABM_EUNSUPPORTED
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    with pytest.raises(capi.GabmError) as ei:   # not together with the R/M split
        capi.gabm_create([pop], capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, tau_IM=5, p_IR=PMF))
    assert ei.value.status == capi.GABM_EUNSUPPORTED
    for bad in (np.r_[PMF[:3], -0.1, PMF[4:]], np.zeros(TAU_IR), np.r_[PMF[:5], np.nan, PMF[6:]]):
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_create([pop], capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, p_IR=bad.astype(np.float32)))
        assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(ValueError):
        capi.gabm_create([pop], capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, p_IR=PMF[:5]))
    ctx = capi.gabm_create([pop], _models(PMF, 0)[0])
    T = 12
    Rd, md_, Sd = to_dev(np.full((1, T), 2.5, np.float32), np.full((1, T), 0.02, np.float32),
                         synth.SUSCEPTIBILITY[None, :].astype(np.float32))
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward_table(ctx, to_dev(np.ones((1, T)))[0])
    assert ei.value.status == capi.GABM_EUNSUPPORTED


def test_several_graphs_and_graph_replay(monkeypatch):
    """Three graphs in one ctx, each following the oracle's run of its own instance; CUDA-
    graph replay of the day loops equals eager launches bitwise."""
    pops = [synth.population_small(n=n, seed=40 + i) for i, n in enumerate((3000, 777, 4500))]
    G, T, n_seed = len(pops), 26, 12
    rng = np.random.default_rng(41)
    R = rng.uniform(2.2, 3.2, (G, T)).astype(np.float32)
    m = rng.uniform(0.01, 0.05, (G, T)).astype(np.float32)
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    md, mo = _models(PMF, 3)
    refs = [DU.forward(pops[g], mo, R[g], m[g], S[g], n_seed=n_seed, inst=g) for g in range(G)]
    gD = np.stack([O.mse(refs[g]["D"], synth.target_curve(T, pops[g].n, seed=g, level=5e-5))[1] for g in range(G)])
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
        ref = DU.backward(pops[g], mo, R[g], m[g], S[g], refs[g]["e_final"], gD[g], inst=g)
        check_adjoint(dR[g], ref["dR"], f"dR[{g}]")
        check_adjoint(dm[g], ref["dm"], f"dm[{g}]")
        check_adjoint(dS[g], ref["dS"], f"dS[{g}]")
        checked += 1
    assert checked >= 2
