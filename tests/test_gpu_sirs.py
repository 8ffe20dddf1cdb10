"""SIRS reinfection (return to S tau_RS days after entering RM) on the GPU against the
FP64 oracle (oracle/sirs.py).

Bars: the base model's.  On an oracle trajectory with no near-tie infection draw the GPU
reproduces the final state (last exposure days), the stage counts and D exactly; the
adjoint (dR, dm, dS) is within 1e-3 of the oracle's elementwise.  With nobody returning
within the horizon the results are bitwise the base model's kernels'.
"""
import numpy as np
import pytest

import oracle as O
from oracle import sirs as SI
from paper_2207_09714_gb300 import capi, synth

from helpers import EXACT_MARGIN, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TAU_EI, TAU_IR = 4, 7


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _models(tau_RS, seed):
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    return (capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, seed=seed, tau_RS=tau_RS),
            SI.SirsModel(TAU_EI, TAU_IR, tau_RS, c, seed=seed))


def _reinfected(e_hist):
    t_idx, i_idx = np.nonzero(e_hist[1:] != e_hist[:-1])
    return int((np.bincount(i_idx, minlength=e_hist.shape[1]) >= 2).sum())


@pytest.mark.parametrize("tau_RS,T", [(6, 50), (2, 36)])
def test_trajectory_and_adjoint_match_oracle(tau_RS, T):
    pop = synth.population_small(n=6000, seed=12)
    rng = np.random.default_rng(tau_RS)
    Rv = rng.uniform(2.6, 3.4, T).astype(np.float32)
    mv = rng.uniform(0.01, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    for seed in range(30):
        md, mo = _models(tau_RS, seed)
        f = SI.forward(pop, mo, Rv, mv, S, n_seed=30)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    assert _reinfected(f["e_hist"]) > 50
    _, gD = O.mse(f["D"], synth.target_curve(T, pop.n, seed=5, level=5e-5))
    g = SI.backward(pop, mo, Rv, mv, S, f["e_hist"], gD)
    ctx = capi.gabm_create([pop], md)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [30], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0].astype(np.int64), f["e_final"])
    assert np.array_equal(counts.cpu().numpy()[0], f["counts"])
    assert np.array_equal(D.cpu().numpy()[0], f["D"])
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    assert np.abs(g["dR"]).max() > 0


def test_no_return_within_the_horizon_is_bitwise_the_base_model():
    pop = synth.population_small(n=8000, seed=3)
    T = 40
    rng = np.random.default_rng(2)
    Rv = rng.uniform(2.2, 3.0, T).astype(np.float32)
    mv = rng.uniform(0.01, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    (gDd,) = to_dev(np.linspace(-1, 1, T)[None, :])
    out = []
    for mdl in (model(seed=6), _models(T, 6)[0]):
        ctx = capi.gabm_create([pop], mdl)
        D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [25], want_counts=True)
        out.append([capi.gabm_get_state(ctx), D.cpu().numpy(), counts.cpu().numpy()] +
                   [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)])
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert out[0][1].sum() > 0


def test_several_graphs_and_graph_replay(monkeypatch):
    pops = [synth.population_small(n=n, seed=50 + i) for i, n in enumerate((3000, 777, 4500))]
    G, T, n_seed, tau_RS = len(pops), 40, 12, 4
    rng = np.random.default_rng(51)
    R = rng.uniform(2.6, 3.4, (G, T)).astype(np.float32)
    m = rng.uniform(0.01, 0.05, (G, T)).astype(np.float32)
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    md, mo = _models(tau_RS, 3)
    refs = [SI.forward(pops[g], mo, R[g], m[g], S[g], n_seed=n_seed, inst=g) for g in range(G)]
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
        assert np.array_equal(e[off[g]:off[g + 1]].astype(np.int64), refs[g]["e_final"]), g
        assert np.array_equal(D[g], refs[g]["D"]), g
        ref = SI.backward(pops[g], mo, R[g], m[g], S[g], refs[g]["e_hist"], gD[g], inst=g)
        check_adjoint(dR[g], ref["dR"], f"dR[{g}]")
        check_adjoint(dm[g], ref["dm"], f"dm[{g}]")
        check_adjoint(dS[g], ref["dS"], f"dS[{g}]")
        checked += 1
    assert checked >= 2


def test_unsupported():
    pop = synth.population_small(n=500, seed=1)
    c = synth.infectiousness_table(TAU_EI, TAU_IR)
    for kw, sets in ((dict(lambda_policy=capi.GABM_RECOMPUTE), 1), (dict(), 4),
                     (dict(p_IR=np.full(TAU_IR, 1 / TAU_IR, np.float32)), 1)):
        with pytest.raises(capi.GabmError) as ei:
            capi.gabm_create([pop], capi.ModelDesc(tau_EI=TAU_EI, tau_IR=TAU_IR, c=c, tau_RS=5, **kw), sets_per_graph=sets)
        assert ei.value.status == capi.GABM_EUNSUPPORTED
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create_bipartite(synth.population_bipartite(800, seed=1), _models(5, 0)[0])
    assert ei.value.status == capi.GABM_EUNSUPPORTED
    ctx = capi.gabm_create([pop], _models(5, 0)[0])
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_set_state(ctx, 3, np.full((1, pop.n), capi.GABM_NEVER, np.int16))
    assert ei.value.status == capi.GABM_EUNSUPPORTED
    T = 12
    Rd, md_, Sd = to_dev(np.full((1, T), 2.5, np.float32), np.full((1, T), 0.02, np.float32),
                         synth.SUSCEPTIBILITY[None, :].astype(np.float32))
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [10])
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_backward_table(ctx, to_dev(np.ones((1, T)))[0])
    assert ei.value.status == capi.GABM_EUNSUPPORTED


def test_more_than_255_exposures_per_agent():
    """A 3-day cycle (tau_EI = tau_IR = tau_RS = 1) over 900 days: agents are exposed up
    to ~300 times, so each row's history holds more entries than an 8-bit count can
    number.  State, counts, D and the adjoint follow the oracle.  Each susceptible day's
    dL/dy is a difference of two adjoints that share the return term of every later
    exposure; the sweep cancels that term exactly (in fp32 it would swamp the
    difference on a cycle this short)."""
    pop = synth.population_small(n=300, seed=3)
    T, n_seed = 900, 30
    c = np.array([0.0, 1.0], np.float32)
    Rv = np.full(T, 5.0, np.float32)
    mv = np.full(T, 0.02, np.float32)
    S = synth.SUSCEPTIBILITY.astype(np.float32)
    for seed in range(40):
        mo = SI.SirsModel(1, 1, 1, c, seed=seed)
        f = SI.forward(pop, mo, Rv, mv, S, n_seed=n_seed)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    assert (f["e_hist"][1:] != f["e_hist"][:-1]).sum(0).max() > 255
    _, gD = O.mse(f["D"], synth.target_curve(T, pop.n, seed=5, growth=0.0, level=5e-3))
    g = SI.backward(pop, mo, Rv, mv, S, f["e_hist"], gD)
    assert np.abs(g["dR"]).max() > 0
    ctx = capi.gabm_create([pop], capi.ModelDesc(tau_EI=1, tau_IR=1, c=c, seed=seed, tau_RS=1))
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0].astype(np.int64), f["e_final"])
    assert np.array_equal(counts.cpu().numpy()[0], f["counts"])
    assert np.array_equal(D.cpu().numpy()[0], f["D"])
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
