"""GPU parity of the set-batched kernels (B parameter sets per graph) against the
FP64 oracle, one oracle run per instance (instance id = graph * B + set keys its
Philox stream).

Bars as for one set per graph: lambda within 1e-5 relative in lockstep, flips only
at near-ties, bit-exact trajectories and counts where the oracle run has no
near-tie, and the adjoint within 1e-3 of the oracle adjoint.  Instances whose
oracle run has a near-tie (|u - p| <= 1e-6 somewhere) may take another
trajectory after it; those are checked in lockstep only.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import (EXACT_MARGIN, FLIP_MARGIN, LAM_RTOL, NEVER, check_adjoint, ensure_built, model, to_dev,
                     torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def _params(I, T, rng_seed):
    """Per-instance parameters of an ensemble: R ~ U[1.5, 4], m ~ U[0.005, 0.05], S scaled per age."""
    rng = np.random.default_rng(rng_seed)
    R = (rng.uniform(1.5, 4.0, (I, 1)) * rng.uniform(0.9, 1.1, (I, T))).astype(np.float32)
    m = np.repeat(rng.uniform(0.005, 0.05, (I, 1)), T, axis=1).astype(np.float32)
    S = (synth.SUSCEPTIBILITY[None, :] * rng.uniform(0.8, 1.2, (I, 9))).astype(np.float32)
    return R, m, S


def _hub_graph():
    """Directed weights plus one row with 1499 in-neighbours (compensated sums, transposed edges)."""
    pop = synth.random_directed(2000, 12.0, seed=4)
    hub_cols = np.arange(1, 1500, dtype=np.uint32)
    rowptr = pop.rowptr.astype(np.int64)
    col = np.concatenate([hub_cols, pop.col[rowptr[1]:]]).astype(np.uint32)
    w = np.concatenate([np.linspace(0.1, 2.0, hub_cols.size).astype(np.float32), pop.w[rowptr[1]:]])
    rp = rowptr.copy()
    rp[1:] = rowptr[1:] - rowptr[1] + hub_cols.size
    return synth.Population(n=pop.n, rowptr=rp.astype(np.uint64), col=col, w=w, age=pop.age)


def _oracle_runs(pops, B, R, m, S, n_seed, seed, want_hist=False):
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=seed)
    refs = []
    for g, pop in enumerate(pops):
        for s in range(B):
            i = g * B + s
            refs.append(O.forward_hard(pop, md_o, R[i], m[i], S[i], n_seed=n_seed[i], inst=i, want_hist=want_hist))
    return md_o, refs


@pytest.mark.parametrize("B", [2, 3, 8, 17, 64])
def test_batched_free_run_matches_oracle(B):
    """Every set width (two to 64 sets, one kernel template each): seeds, trajectories,
    counts and deaths of each instance equal its own oracle run."""
    pop = synth.population_small(n=3001, seed=31)
    T = 20
    R, m, S = _params(B, T, rng_seed=B)
    n_seed = [(5 + 3 * s) % 17 for s in range(B)]
    ctx = capi.gabm_create([pop], model(seed=5), sets_per_graph=B)
    Rd, md_, Sd = to_dev(R, m, S)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, n_seed, want_counts=True)
    D, counts = D.cpu().numpy(), counts.cpu().numpy()
    e = capi.gabm_get_state(ctx)
    assert e.shape == (B, pop.n)
    md_o, refs = _oracle_runs([pop], B, R, m, S, n_seed, seed=5)
    exact = 0
    for s, ref in enumerate(refs):
        seeds = np.sort(O.select_seeds(pop.n, 5, s, n_seed[s]))
        assert np.array_equal(np.sort(np.flatnonzero(e[s] == -4)), seeds), s
        assert np.all(counts[s].sum(axis=1) == pop.n)
        if ref["margin"] > EXACT_MARGIN:
            assert np.array_equal(e[s], ref["e_final"]), s
            assert np.array_equal(counts[s], ref["counts"]), s
            assert np.allclose(D[s], ref["D"], rtol=1e-15, atol=0), s
            exact += 1
    assert exact >= max(1, B // 2)
    assert (counts[:, -1, 0] < pop.n - 50).any()   # some epidemic took off
    # the state round-trips through set_state / get_state in caller order
    capi.gabm_set_state(ctx, T, e)
    assert np.array_equal(capi.gabm_get_state(ctx), e)


def _graph(kind, n, seed):
    """"typed": the four-interaction-type generator (households, schools, workplaces, random
    contacts); "small": households and random contacts only; "hub": directed, one long row."""
    if kind == "typed":
        return synth.population_typed(n, seed=seed)
    if kind == "small":
        return synth.population_small(n=n, seed=seed)
    return _hub_graph()


@pytest.mark.parametrize("graph,B", [("typed", 8), ("typed", 64), ("small", 64), ("hub", 4)])
def test_batched_lockstep_days(graph, B):
    """Each day from the oracle's start-of-day states of all sets: lambda per set within
    1e-5 relative, decisions equal except at near-ties."""
    pop = _graph(graph, 10_000, 2)
    T = 24
    R, m, S = _params(B, T, rng_seed=100 + B)
    n_seed = [20] * B
    md_o, refs = _oracle_runs([pop], B, R, m, S, n_seed, seed=3, want_hist=True)
    ctx = capi.gabm_create([pop], model(seed=3), sets_per_graph=B)
    Rd, md_, Sd = to_dev(R, m, S)
    worst, flips, drawn = 0.0, 0, 0
    days = range(0, T, 3) if B == 64 else range(T)
    for t in days:
        e_start = np.stack([r["e_hist"][t] for r in refs])
        capi.gabm_set_state(ctx, t, e_start)
        capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
        lam = capi.gabm_get_lambda(ctx, t).astype(np.float64)
        e_gpu = capi.gabm_get_state(ctx)
        for s in range(B):
            ref = O.day_hard(pop, md_o, t, float(R[s, t]), S[s], e_start[s], inst=s)
            sus = e_start[s] == NEVER
            lam_ref = float(R[s, t]) * S[s][pop.age].astype(np.float64) * ref["Lam"]
            assert np.all(lam[s][~sus] == 0.0)
            pos = sus & (lam_ref > 0)
            if pos.any():
                worst = max(worst, float(np.max(np.abs(lam[s][pos] - lam_ref[pos]) / lam_ref[pos])))
            assert np.all(lam[s][sus & (lam_ref == 0)] == 0.0)
            diff = e_gpu[s] != ref["e_out"]
            if diff.any():
                assert np.all(np.abs(ref["u"][diff] - ref["p"][diff]) < FLIP_MARGIN)
                assert np.all(sus[diff])
            flips += int(diff.sum())
            drawn += int(sus.sum())
    assert worst <= LAM_RTOL, worst
    assert flips <= max(1, 1e-5 * drawn)


def _adjoint_case(pops, B, T, seed, rng_seed):
    I = len(pops) * B
    R, m, S = _params(I, T, rng_seed)
    n_seed = [8 + (i % 5) for i in range(I)]
    md_o, refs = _oracle_runs(pops, B, R, m, S, n_seed, seed=seed)
    gDs, gs = [], []
    i = 0
    for g, pop in enumerate(pops):
        for s in range(B):
            y = synth.target_curve(T, pop.n, seed=rng_seed + i, level=5e-5)
            _, gD = O.mse(refs[i]["D"], y)
            gDs.append(gD)
            gs.append(O.backward_hard(pop, md_o, R[i], m[i], S[i], refs[i]["e_final"], gD, inst=i))
            i += 1
    ctx = capi.gabm_create(pops, model(seed=seed), sets_per_graph=B)
    Rd, md_, Sd = to_dev(R, m, S)
    capi.gabm_forward(ctx, T, Rd, md_, Sd, n_seed)
    e = capi.gabm_get_state(ctx)
    (gDd,) = to_dev(np.stack(gDs))
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    tab = [x.cpu().numpy() for x in capi.gabm_backward_table(ctx, gDd)]
    for a, b in zip((dR, dm, dS), tab[:3]):   # the table adjoint leaves the others unchanged
        assert np.array_equal(a, b)
    dc = tab[3]
    checked = 0
    off = np.concatenate([[0], np.cumsum([p.n for p in pops])])
    i = 0
    for g, pop in enumerate(pops):
        for s in range(B):
            if refs[i]["margin"] > EXACT_MARGIN:
                # the GPU ran the oracle's trajectory: its adjoint must match the oracle's
                assert np.array_equal(e[s, off[g]:off[g + 1]], refs[i]["e_final"]), i
                check_adjoint(dR[i], gs[i]["dR"], f"dR[{i}]")
                check_adjoint(dm[i], gs[i]["dm"], f"dm[{i}]")
                check_adjoint(dS[i], gs[i]["dS"], f"dS[{i}]")
                assert dc[i, 0] == 0.0
                check_adjoint(dc[i, 1:], gs[i]["dc"][1:], f"dc[{i}]")
                assert np.abs(gs[i]["dR"]).max() > 0
                checked += 1
            assert np.all(np.isfinite(dR[i])) and np.all(np.isfinite(dS[i]))
            i += 1
    return checked, I


@pytest.mark.parametrize("graph,B", [("typed", 6), ("typed", 64), ("small", 64), ("hub", 5)])
def test_batched_adjoint_matches_oracle(graph, B):
    pop = _graph(graph, 4000, 8)
    checked, I = _adjoint_case([pop], B, T=22, seed=9, rng_seed=40 + B)
    assert checked >= max(1, I // 2)


def test_batched_multi_graph():
    """Uneven graphs x sets: instance g * B + s has its own Philox stream and parameters."""
    pops = [synth.population_small(n=n, seed=50 + i) for i, n in enumerate((1500, 77, 2300))]
    checked, I = _adjoint_case(pops, 3, T=20, seed=12, rng_seed=70)
    assert checked >= I // 2


def _run_all(ctx, T, R, m, S, n_seed, y):
    Rd, md_, Sd, yd = to_dev(R, m, S, y)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, n_seed, want_counts=True)
    lam = [capi.gabm_get_lambda(ctx, t) for t in (0, T // 2, T - 1)]
    loss, gD = capi.gabm_mse_loss(ctx, yd)
    dR, dm, dS = capi.gabm_backward(ctx, gD)
    dc = capi.gabm_backward_table(ctx, gD)[3]
    out = dict(D=D.cpu().numpy(), counts=counts.cpu().numpy(), e=capi.gabm_get_state(ctx),
               dR=dR.cpu().numpy(), dm=dm.cpu().numpy(), dS=dS.cpu().numpy(), dc=dc.cpu().numpy())
    for k, v in enumerate(lam):
        out[f"lam{k}"] = v
    return out


def _assert_same(a, b, what):
    for k in a:
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("B", [3, 8, 20, 64])
def test_schedules_are_bitwise_equal(B):
    """Every sets-per-lane schedule sums each set in entry order and each tile's rows in
    ascending order: identical trajectories, lambdas and adjoints."""
    pop = synth.population_small(n=5003, seed=61)
    T = 20
    R, m, S = _params(B, T, rng_seed=300 + B)
    y = np.stack([synth.target_curve(T, pop.n, seed=b, level=5e-5) for b in range(B)])
    ctx = capi.gabm_create([pop], model(seed=21), sets_per_graph=B)
    Bp = 1 << (B - 1).bit_length()
    ref = None
    for spl in (2, 4, 8):
        if spl > Bp:
            with pytest.raises(capi.GabmError):
                capi.gabm_set_schedule(ctx, spl, spl)
            continue
        capi.gabm_set_schedule(ctx, spl, spl)
        assert capi.gabm_get_schedule(ctx)["fwd_sets_per_lane"] == spl
        out = _run_all(ctx, T, R, m, S, [10] * B, y)
        if ref is None:
            ref = out
            assert np.abs(out["dR"]).max() > 0
        else:
            _assert_same(ref, out, f"spl={spl}")
    # the backward in launches of fewer sets (each launch one column block of the rows)
    for chunk in (Bp // 2, Bp // 4):
        for spl in (2, 4, 8):
            if chunk < 2 or spl > chunk:
                continue
            capi.gabm_set_schedule(ctx, 4 if Bp >= 4 else 2, spl, bwd_sets_per_launch=chunk)
            assert capi.gabm_get_schedule(ctx)["bwd_sets_per_launch"] == chunk
            _assert_same(ref, _run_all(ctx, T, R, m, S, [10] * B, y), f"chunk={chunk} spl={spl}")
    with pytest.raises(capi.GabmError):
        capi.gabm_set_schedule(ctx, 2, 2, bwd_sets_per_launch=3)
    # mixed schedules, then the autotuner: same results, state as after the last forward
    capi.gabm_set_schedule(ctx, 2, Bp if Bp <= 8 else 8)
    _assert_same(ref, _run_all(ctx, T, R, m, S, [10] * B, y), "mixed")
    e_before = capi.gabm_get_state(ctx)
    chosen = capi.gabm_autotune(ctx, 1)
    assert chosen["fwd_sets_per_lane"] in (2, 4, 8) and chosen["bwd_sets_per_lane"] in (2, 4, 8)
    assert Bp % chosen["bwd_sets_per_launch"] == 0
    assert np.array_equal(capi.gabm_get_state(ctx), e_before)
    assert np.array_equal(capi.gabm_get_lambda(ctx, T // 2), ref["lam1"])
    (gDd,) = to_dev(np.stack([O.mse(ref["D"][b], y[b])[1] for b in range(B)]))
    dR, _, _ = capi.gabm_backward(ctx, gDd)
    assert np.array_equal(dR.cpu().numpy(), ref["dR"])


@pytest.mark.parametrize("B", [1, 16])
def test_cuda_graph_replay_equals_eager_launches(B, monkeypatch):
    """Day loops replayed from captured CUDA graphs give bitwise what eager launches give,
    across changes of T (re-capture) and repeated calls (replay)."""
    pop = synth.population_small(n=4001, seed=62)
    R, m, S = _params(B, 26, rng_seed=400 + B)
    y = np.stack([synth.target_curve(26, pop.n, seed=b, level=5e-5) for b in range(B)])
    graphs = capi.gabm_create([pop], model(seed=22), sets_per_graph=B)
    monkeypatch.setenv("GABM_CUDA_GRAPHS", "0")
    eager = capi.gabm_create([pop], model(seed=22), sets_per_graph=B)
    for T in (26, 13, 26, 26):
        sl = (slice(None), slice(0, T))
        a = _run_all(graphs, T, R[sl], m[sl], S, [7] * B, y[sl])
        b = _run_all(eager, T, R[sl], m[sl], S, [7] * B, y[sl])
        _assert_same(a, b, f"T={T}")
    # a replay issues the same kernels: the launch counter grows by the same amount
    n0g, n0e = capi.gabm_launch_count(graphs), capi.gabm_launch_count(eager)
    _run_all(graphs, 26, R, m, S, [7] * B, y)
    _run_all(eager, 26, R, m, S, [7] * B, y)
    assert capi.gabm_launch_count(graphs) - n0g == capi.gabm_launch_count(eager) - n0e


def test_batched_long_horizon_beyond_fp32_range():
    """Four sets over 200 days whose exact adjoints reach 1e39..1e51 (beyond fp32): the
    sets share a power-of-two scale per day, and every set without a near-tie matches
    the FP64 oracle adjoint."""
    pop = synth.population_small(n=3000, seed=3)
    T, B = 200, 4
    R = np.repeat(np.array([1.2, 1.3, 1.35, 1.45], np.float32)[:, None], T, axis=1)
    m = np.full((B, T), 0.02, np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (B, 1)).astype(np.float32)
    md_o, refs = _oracle_runs([pop], B, R, m, S, [10] * B, seed=1)
    y = synth.target_curve(T, pop.n, seed=2, level=5e-5)
    gDs = np.stack([O.mse(r["D"], y)[1] for r in refs])
    ctx = capi.gabm_create([pop], model(seed=1), sets_per_graph=B)
    Rd, md_, Sd, gDd = to_dev(R, m, S, gDs)
    capi.gabm_forward(ctx, T, Rd, md_, Sd, [10] * B)
    e = capi.gabm_get_state(ctx)
    dR, dm, dS = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gDd)]
    checked = 0
    for s, ref in enumerate(refs):
        if ref["margin"] <= EXACT_MARGIN:
            continue
        assert np.array_equal(e[s], ref["e_final"])
        g = O.backward_hard(pop, md_o, R[s], m[s], S[s], ref["e_final"], gDs[s], inst=s)
        assert np.abs(g["dR"]).max() > 3.4e38
        check_adjoint(dR[s], g["dR"], f"dR[{s}]")
        check_adjoint(dm[s], g["dm"], f"dm[{s}]")
        check_adjoint(dS[s], g["dS"], f"dS[{s}]")
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("B", [6, 64])
def test_recompute_policy_is_bitwise_the_store_policy(B):
    """Several sets per graph without the lambda store: the backward sums lambda again
    from the final exposure days, bitwise the forward's, so the adjoint is bitwise that of
    the store policy.  A backward needs a forward over days 0..T-1 (after a forward from a
    set state it is refused)."""
    pop = synth.population_small(n=5000, seed=13)
    T = 24
    R, m, S = _params(B, T, 90 + B)
    y = np.stack([synth.target_curve(T, pop.n, seed=s, level=5e-5) for s in range(B)])
    outs = {}
    for policy in (capi.GABM_STORE_LAMBDA, capi.GABM_RECOMPUTE):
        ctx = capi.gabm_create([pop], model(seed=3, policy=policy), sets_per_graph=B)
        Rd, md_, Sd, yd = to_dev(R, m, S, y)
        D, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [10] * B)
        _, gD = capi.gabm_mse_loss(ctx, yd)
        outs[policy] = [D.cpu().numpy()] + [x.cpu().numpy() for x in capi.gabm_backward(ctx, gD)]
        if policy == capi.GABM_RECOMPUTE:
            again = [x.cpu().numpy() for x in capi.gabm_backward(ctx, gD)]   # a second sweep, same result
            for a, b in zip(outs[policy][1:], again):
                assert np.array_equal(a, b)
            with pytest.raises(capi.GabmError) as ei:
                capi.gabm_backward_table(ctx, gD)
            assert ei.value.status == capi.GABM_EUNSUPPORTED
            capi.gabm_set_state(ctx, T, capi.gabm_get_state(ctx))
            capi.gabm_forward(ctx, T, Rd, md_, Sd)
            with pytest.raises(capi.GabmError) as ei:
                capi.gabm_backward(ctx, gD)
            assert ei.value.status == capi.GABM_ESTATE
    for a, b in zip(outs[capi.GABM_STORE_LAMBDA], outs[capi.GABM_RECOMPUTE]):
        assert np.array_equal(a, b)
