"""Full-size parity of the two largest workloads, in the configuration the library
runs them (recompute policy, day loops replayed as CUDA graphs, autotuned schedule):

* 32 county graphs with agent counts log-uniform in [5e4, 2e6] (the typed
  generator, ~12M agents and ~270M directed edges for this seed), each with its
  own parameters, 90 days;
* one 8M-agent graph with Chung-Lu power-law contacts (exponent 2.5, degrees up
  to 2000; ~155M directed edges), 120 days.

The oracle cannot run these horizons at this size in test time, so the checks are
properties that hold at any size (conservation, monotone compartments, deaths =
m x RM increments) over the whole horizon, plus sampled oracle comparisons: one
lockstep day from the oracle's own state (lambda within 1e-5 relative, decisions
equal except at near-ties) and the adjoint of a shorter replayed horizon (within
1e-3 of the oracle adjoint).  Sampled counties: the smallest, the largest and two
seeded picks.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import FLIP_MARGIN, LAM_RTOL, NEVER, check_adjoint, ensure_built, model, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _check_properties(counts, D, m, n):
    """Per-day invariants of one instance's hard trajectory."""
    assert np.all(counts.sum(axis=1) == n)
    S, RM = counts[:, 0], counts[:, 3]
    assert np.all(np.diff(S) <= 0) and np.all(np.diff(RM) >= 0)
    # D_t = m_t newRM(t), and newRM(t) = RM(t) - RM(t-1): RM counts agents with t - e >= L
    assert np.array_equal(D[1:], m[1:].astype(np.float64) * np.diff(RM))


def _lockstep(pop, md_o, t, R_t, S, e_start, lam_gpu, e_gpu, inst):
    ref = O.day_hard(pop, md_o, t, float(R_t), S, e_start, inst=inst)
    sus = e_start == NEVER
    lam_ref = float(R_t) * S[pop.age].astype(np.float64) * ref["Lam"]
    assert np.all(lam_gpu[~sus] == 0.0)
    pos = sus & (lam_ref > 0)
    rel = np.abs(lam_gpu[pos].astype(np.float64) - lam_ref[pos]) / lam_ref[pos]
    assert np.all(lam_gpu[sus & (lam_ref == 0)] == 0.0)
    diff = e_gpu != ref["e_out"]
    if diff.any():
        assert np.all(np.abs(ref["u"][diff] - ref["p"][diff]) < FLIP_MARGIN)
        assert np.all(sus[diff])
    assert diff.sum() <= max(1, 1e-5 * sus.sum())
    assert pos.sum() > 0
    return float(rel.max())


@pytest.fixture(scope="module")
def counties():
    return synth.uneven_counties(32, seed=0)


def test_uneven_counties_full_size(counties):
    pops = counties
    G, T = len(pops), 90
    sizes = np.array([p.n for p in pops])
    rng = np.random.default_rng(11)
    R = (rng.uniform(1.8, 3.2, (G, 1)) * rng.uniform(0.9, 1.1, (G, T))).astype(np.float32)
    m = np.repeat(rng.uniform(0.005, 0.05, (G, 1)), T, axis=1).astype(np.float32)
    S = (synth.SUSCEPTIBILITY[None, :] * rng.uniform(0.8, 1.2, (G, 9))).astype(np.float32)
    ctx = capi.gabm_create(pops, model(seed=5, policy=capi.GABM_RECOMPUTE))
    Rd, md_, Sd = to_dev(R, m, S)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [20] * G, want_counts=True)
    D, counts = D.cpu().numpy(), counts.cpu().numpy()
    for g in range(G):
        _check_properties(counts[g], D[g], m[g], sizes[g])
    assert (counts[:, -1, 0] < sizes - 1000).sum() >= G // 2   # most county epidemics took off
    # the autotuner keeps the trajectory; the replayed day loop gives the same deaths
    capi.gabm_autotune(ctx, 1)
    D2, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [20] * G)
    assert np.array_equal(D2.cpu().numpy(), D)

    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=5)
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.choice(G, 2, replace=False).tolist()))
    off = np.concatenate([[0], np.cumsum(sizes)])
    # the 90-day adjoint of every sampled county's own GPU trajectory against the oracle's
    # adjoint of that trajectory
    y = np.stack([synth.target_curve(T, pops[g].n, seed=g, level=5e-5) for g in range(G)])
    (yd,) = to_dev(y)
    _, gDd = capi.gabm_mse_loss(ctx, yd)
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    E = capi.gabm_get_state(ctx)[0]
    gD90 = gDd.cpu().numpy()
    for g in picks:
        ref = O.backward_hard(pops[g], md_o, R[g], m[g], S[g], E[off[g]:off[g + 1]], gD90[g], inst=g)
        check_adjoint(dR[g], ref["dR"], f"dR[{g}] (90 days)")
        check_adjoint(dm[g], ref["dm"], f"dm[{g}] (90 days)")
        check_adjoint(dS[g], ref["dS"], f"dS[{g}] (90 days)")
    # one lockstep day from the oracle's own states of the sampled counties (the others susceptible)
    t = 40
    e_start = np.full(off[-1], NEVER, np.int16)
    for g in picks:
        e_start[off[g]:off[g + 1]] = O.forward_hard(pops[g], md_o, R[g, :t], m[g, :t], S[g], n_seed=20,
                                                    inst=g)["e_final"]
    capi.gabm_set_state(ctx, t, e_start[None, :])
    capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
    lam = capi.gabm_get_lambda(ctx, t)[0]
    e_gpu = capi.gabm_get_state(ctx)[0]
    worst = 0.0
    for g in picks:
        sl = slice(off[g], off[g + 1])
        worst = max(worst, _lockstep(pops[g], md_o, t, R[g, t], S[g], e_start[sl], lam[sl], e_gpu[sl], g))
    assert worst <= LAM_RTOL, worst

    # adjoint of a 30-day horizon replayed from the oracle's final states
    Ta = 30
    E = np.full(off[-1], NEVER, np.int16)
    gD = np.zeros((G, Ta))
    grads = {}
    for g in picks:
        f = O.forward_hard(pops[g], md_o, R[g, :Ta], m[g, :Ta], S[g], n_seed=20, inst=g)
        y = synth.target_curve(Ta, pops[g].n, seed=g, level=5e-5)
        _, gD[g] = O.mse(f["D"], y)
        E[off[g]:off[g + 1]] = f["e_final"]
        grads[g] = O.backward_hard(pops[g], md_o, R[g, :Ta], m[g, :Ta], S[g], f["e_final"], gD[g], inst=g)
    capi.gabm_set_state(ctx, Ta, E[None, :])
    capi.gabm_forward(ctx, Ta, Rd[:, :Ta].contiguous(), md_[:, :Ta].contiguous(), Sd)
    (gDd,) = to_dev(gD)
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    for g in picks:
        check_adjoint(dR[g], grads[g]["dR"], f"dR[{g}]")
        check_adjoint(dm[g], grads[g]["dm"], f"dm[{g}]")
        check_adjoint(dS[g], grads[g]["dS"], f"dS[{g}]")


@pytest.fixture(scope="module")
def powerlaw8m():
    return synth.population_typed(8_000_000, seed=0, powerlaw=True)


def test_powerlaw_8M_full_size(powerlaw8m):
    pop = powerlaw8m
    assert pop.degrees().max() > 1000          # hubs: rows far longer than a warp pass
    T = 120
    R = np.full((1, T), 2.5, np.float32)
    m = np.full((1, T), 0.01, np.float32)
    S = synth.SUSCEPTIBILITY[None, :].astype(np.float32)
    ctx = capi.gabm_create([pop], model(seed=1, policy=capi.GABM_RECOMPUTE))
    Rd, md_, Sd = to_dev(R, m, S)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [20], want_counts=True)
    D, counts = D.cpu().numpy()[0], counts.cpu().numpy()[0]
    _check_properties(counts, D, m[0], pop.n)
    assert counts[-1, 0] < 0.9 * pop.n            # the epidemic took off
    (yd,) = to_dev(synth.target_curve(T, pop.n)[None, :])
    _, gD = capi.gabm_mse_loss(ctx, yd)
    # over 120 days the adjoint grows to ~1e36, past the sweep's rescaling threshold (2^64):
    # the scaled sweep follows the FP64 oracle's adjoint of the GPU's own trajectory over
    # the whole horizon
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gD)]
    cur, peak = capi.gabm_mem_stats(ctx)
    assert peak < 16 * 2 ** 30                     # the 120-day horizon needs no per-day snapshots
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=1)
    E = capi.gabm_get_state(ctx)[0]
    g_own = O.backward_hard(pop, md_o, R[0], m[0], S[0], E, gD.cpu().numpy()[0])
    assert np.abs(g_own["dR"]).max() > 2.0 ** 64    # values the sweep must rescale
    check_adjoint(dR, g_own["dR"], "dR (120 days)")
    check_adjoint(dm, g_own["dm"], "dm (120 days)")
    check_adjoint(dS, g_own["dS"], "dS (120 days)")

    t = 30
    e_start = O.forward_hard(pop, md_o, R[0, :t], m[0, :t], S[0], n_seed=20)["e_final"]
    capi.gabm_set_state(ctx, t, e_start[None, :])
    capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
    worst = _lockstep(pop, md_o, t, R[0, t], S[0], e_start, capi.gabm_get_lambda(ctx, t)[0],
                      capi.gabm_get_state(ctx)[0], 0)
    assert worst <= LAM_RTOL, worst

    Ta = 20
    f = O.forward_hard(pop, md_o, R[0, :Ta], m[0, :Ta], S[0], n_seed=20)
    _, gDa = O.mse(f["D"], synth.target_curve(Ta, pop.n, seed=3, level=5e-6))
    g = O.backward_hard(pop, md_o, R[0, :Ta], m[0, :Ta], S[0], f["e_final"], gDa)
    capi.gabm_set_state(ctx, Ta, f["e_final"][None, :])
    capi.gabm_forward(ctx, Ta, Rd[:, :Ta].contiguous(), md_[:, :Ta].contiguous(), Sd)
    (gDd,) = to_dev(gDa[None, :])
    dR, dm, dS = [x.cpu().numpy()[0] for x in capi.gabm_backward(ctx, gDd)]
    check_adjoint(dR, g["dR"], "dR")
    check_adjoint(dm, g["dm"], "dm")
    check_adjoint(dS, g["dS"], "dS")


def test_batched_500k_64_sets_full_size():
    """The batched ensemble at its full size: one shared 500k-agent typed contact graph, 64
    parameter sets (R ~ U[1.5, 4.0], m ~ U[0.005, 0.05]), 45 days, the lambda store, the
    autotuned schedule, day loops replayed as CUDA graphs.  For sampled sets (largest R,
    smallest R and two seeded picks), on the GPU's own trajectory:
    * three lockstep days: lambda within 1e-5 relative of the oracle's day from the same
      start-of-day state, decisions equal except at near-ties;
    * deaths equal m_t times the exits the final state implies;
    * the 45-day adjoint within 1e-3 of the oracle's adjoint of that trajectory."""
    pop = synth.population_typed(500_000, seed=0)
    B, T, L, n_seed = 64, 45, 11, 20
    rng = np.random.default_rng(0)
    R = np.repeat(rng.uniform(1.5, 4.0, (B, 1)), T, axis=1).astype(np.float32)
    m = np.repeat(rng.uniform(0.005, 0.05, (B, 1)), T, axis=1).astype(np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (B, 1)).astype(np.float32)
    y = np.stack([synth.target_curve(T, pop.n, seed=b) for b in range(B)])
    ctx = capi.gabm_create([pop], model(seed=0), sets_per_graph=B)
    Rd, md_, Sd, yd = to_dev(R, m, S, y)
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed] * B)
    capi.gabm_autotune(ctx, 1)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [n_seed] * B, want_counts=True)
    D, counts = D.cpu().numpy(), counts.cpu().numpy()
    _, gDd = capi.gabm_mse_loss(ctx, yd)
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    gD = gDd.cpu().numpy()
    E = capi.gabm_get_state(ctx)
    days = (15, 30, 44)
    lam = {t: capi.gabm_get_lambda(ctx, t) for t in days}
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=0)
    picks = sorted({int(np.argmax(R[:, 0])), int(np.argmin(R[:, 0]))} |
                   set(np.random.default_rng(1).choice(B, 2, replace=False).tolist()))
    worst, compared = 0.0, 0
    for s in picks:
        Es = E[s].astype(np.int64)
        _check_properties(counts[s], D[s], m[s], pop.n)
        exits = np.bincount(Es[(Es != NEVER) & (Es + L >= 0) & (Es + L < T)] + L, minlength=T)
        assert np.array_equal(D[s], m[s].astype(np.float64) * exits), s
        for t in days:
            e_start = np.where(Es < t, Es, NEVER).astype(np.int16)
            e_after = np.where(Es <= t, Es, NEVER).astype(np.int16)
            ref = O.day_hard(pop, md_o, t, float(R[s, t]), S[s], e_start, inst=s)
            sus = e_start == NEVER
            lam_ref = float(R[s, t]) * S[s][pop.age].astype(np.float64) * ref["Lam"]
            assert np.all(lam[t][s][~sus] == 0.0)
            assert np.all(lam[t][s][sus & (lam_ref == 0)] == 0.0)
            pos = sus & (lam_ref > 0)
            if pos.any():
                worst = max(worst, float(np.max(np.abs(lam[t][s][pos] - lam_ref[pos]) / lam_ref[pos])))
                compared += int(pos.sum())
            diff = e_after != ref["e_out"]
            if diff.any():
                assert np.all(np.abs(ref["u"][diff] - ref["p"][diff]) < FLIP_MARGIN), (s, t)
                assert np.all(sus[diff])
            assert diff.sum() <= max(1, 1e-5 * sus.sum()), (s, t)
        g = O.backward_hard(pop, md_o, R[s], m[s], S[s], E[s], gD[s], inst=s)
        check_adjoint(dR[s], g["dR"], f"dR[{s}]")
        check_adjoint(dm[s], g["dm"], f"dm[{s}]")
        check_adjoint(dS[s], g["dS"], f"dS[{s}]")
        assert np.abs(g["dR"]).max() > 0
    assert worst <= LAM_RTOL, worst
    assert compared > 100_000
