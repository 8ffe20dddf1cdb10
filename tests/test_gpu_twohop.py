"""Agent-location graphs (GradABM-JUNE, Sec. 6) on the GPU against the oracle.

The GPU computes every day in two hops over the attendance entries (location
pressures, then the agents' pull over their locations; the adjoint likewise).  The
oracle runs the one-hop model on the written-out pair weights W_ij = sum_l w_il w_jl
(``oracle.bipartite.expand``).  Bars: the forward's (lambda within 1e-5 relative,
decisions equal away from near-ties) and the adjoint's (1e-3), as for one-hop graphs.
"""
import numpy as np
import pytest

import oracle as O
from oracle import bipartite as OB
from paper_2207_09714_gb300 import capi, synth

from helpers import (EXACT_MARGIN, FLIP_MARGIN, LAM_RTOL, NEVER, check_adjoint, ensure_built, model, to_dev,
                     torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


@pytest.fixture(scope="module")
def bip():
    b = synth.population_bipartite(6000, seed=1)
    return b, OB.expand(b)


def _params(T, rng_seed, R=2.2):
    rng = np.random.default_rng(rng_seed)
    Rv = rng.uniform(0.8 * R, 1.2 * R, T).astype(np.float32)
    mv = rng.uniform(0.01, 0.03, T).astype(np.float32)
    return Rv, mv, synth.SUSCEPTIBILITY.astype(np.float32)


def test_expansion_is_large(bip):
    b, W = bip
    assert W.nnz > 20 * b.nnz          # the pair graph the two hops avoid forming


def test_forward_trajectory_and_adjoint_match_oracle(bip):
    b, W = bip
    T, n_seed = 30, 15
    Rv, mv, S = _params(T, 3)
    for seed in range(30):
        md_o = O.Model(4, 7, synth.infectiousness_table(), seed=seed)
        f = O.forward_hard(W, md_o, Rv, mv, S, n_seed=n_seed)
        if f["margin"] > EXACT_MARGIN:
            break
    assert f["margin"] > EXACT_MARGIN
    assert f["counts"][-1, 0] < b.n - 200          # the epidemic spread
    y = synth.target_curve(T, b.n, seed=4, level=5e-5)
    _, gD = O.mse(f["D"], y)
    g = O.backward_hard(W, md_o, Rv, mv, S, f["e_final"], gD)

    ctx = capi.gabm_create_bipartite(b, model(seed=seed))
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0], f["e_final"])
    assert np.allclose(D.cpu().numpy()[0], f["D"], rtol=1e-15, atol=0)
    assert np.array_equal(counts.cpu().numpy()[0], f["counts"])
    (gDd,) = to_dev(gD[None, :])
    dR, dm, dS, dc = [x.cpu().numpy()[0] for x in capi.gabm_backward_table(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")
    check_adjoint(dc[1:], g["dc"][1:], "dc")
    assert np.abs(g["dR"]).max() > 0


def test_lockstep_lambda(bip):
    """One day from the oracle's own mid-epidemic state: lambda within 1e-5 relative."""
    b, W = bip
    T, n_seed, t = 26, 15, 18
    Rv, mv, S = _params(T, 5, R=2.6)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=2)
    e_start = O.forward_hard(W, md_o, Rv[:t], mv[:t], S, n_seed=n_seed)["e_final"]
    ref = O.day_hard(W, md_o, t, float(Rv[t]), S, e_start)
    ctx = capi.gabm_create_bipartite(b, model(seed=2))
    capi.gabm_set_state(ctx, t, e_start[None, :])
    Rd, md_, Sd = to_dev(Rv[None, :t + 1], mv[None, :t + 1], S[None, :])
    capi.gabm_forward(ctx, t + 1, Rd, md_, Sd)
    lam = capi.gabm_get_lambda(ctx, t)[0].astype(np.float64)
    sus = e_start == NEVER
    lam_ref = float(Rv[t]) * S[b.age].astype(np.float64) * ref["Lam"]
    pos = sus & (lam_ref > 0)
    assert pos.sum() > 100
    assert np.max(np.abs(lam[pos] - lam_ref[pos]) / lam_ref[pos]) <= LAM_RTOL
    assert np.all(lam[sus & (lam_ref == 0)] == 0.0)
    e_gpu = capi.gabm_get_state(ctx)[0]
    diff = e_gpu != ref["e_out"]
    if diff.any():
        assert np.all(np.abs(ref["u"][diff] - ref["p"][diff]) < FLIP_MARGIN)


def test_graph_replay_equals_eager(bip, monkeypatch):
    b, _ = bip
    T = 20
    Rv, mv, S = _params(T, 7)
    Rd, md_, Sd = to_dev(Rv[None, :], mv[None, :], S[None, :])
    out = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("GABM_CUDA_GRAPHS", graphs)
        ctx = capi.gabm_create_bipartite(b, model(seed=4))
        D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [12])
        (gDd,) = to_dev(np.linspace(-1, 1, T)[None, :])
        out.append([D.cpu().numpy()] + [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)])
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_invalid_and_unsupported(bip):
    b, _ = bip
    bad = synth.Bipartite(n=b.n, n_loc=b.n_loc, rowptr=b.rowptr, loc=b.loc.copy(), w=b.w, age=b.age)
    bad.loc[5] = b.n_loc
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create_bipartite(bad, model(seed=0))
    assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create_bipartite(b, model(seed=0, policy=capi.GABM_RECOMPUTE))
    assert ei.value.status == capi.GABM_EUNSUPPORTED


def test_several_agent_location_graphs():
    """Three counties as agent-location graphs in one ctx: each follows the oracle's run of
    its own expanded graph (its own Dbar and Philox instance)."""
    bips = [synth.population_bipartite(n, seed=10 + i) for i, n in enumerate((3000, 777, 4500))]
    Ws = [OB.expand(b) for b in bips]
    G, T, n_seed = len(bips), 24, 10
    rng = np.random.default_rng(12)
    R = rng.uniform(1.8, 2.6, (G, T)).astype(np.float32)
    m = rng.uniform(0.01, 0.03, (G, T)).astype(np.float32)
    S = np.repeat(synth.SUSCEPTIBILITY[None, :], G, axis=0).astype(np.float32)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=6)
    refs = [O.forward_hard(Ws[g], md_o, R[g], m[g], S[g], n_seed=n_seed, inst=g) for g in range(G)]
    gD = np.stack([O.mse(refs[g]["D"], synth.target_curve(T, bips[g].n, seed=g, level=5e-5))[1] for g in range(G)])
    ctx = capi.gabm_create_bipartite(bips, model(seed=6))
    Rd, md_, Sd, gDd = to_dev(R, m, S, gD)
    D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed] * G)
    e = capi.gabm_get_state(ctx)[0]
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    off = np.concatenate([[0], np.cumsum([b.n for b in bips])])
    checked = 0
    for g in range(G):
        if refs[g]["margin"] <= EXACT_MARGIN:
            continue
        assert np.array_equal(e[off[g]:off[g + 1]], refs[g]["e_final"]), g
        assert np.allclose(D.cpu().numpy()[g], refs[g]["D"], rtol=1e-15, atol=0)
        ref = O.backward_hard(Ws[g], md_o, R[g], m[g], S[g], refs[g]["e_final"], gD[g], inst=g)
        check_adjoint(dR[g], ref["dR"], f"dR[{g}]")
        check_adjoint(dS[g], ref["dS"], f"dS[{g}]")
        checked += 1
    assert checked >= 2
