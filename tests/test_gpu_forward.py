"""GPU parity of the forward day step against the FP64 oracle (through the C ABI).

Bar: lambda within 1e-5 relative; infection decisions identical except where
|u - p_oracle| < 1e-6, at most a 1e-5 fraction of agents; counts, seeds and
Philox words bit-exact.
"""
import numpy as np
import pytest

import oracle as O
from paper_2207_09714_gb300 import capi, synth

from helpers import (EXACT_MARGIN, FLIP_FRACTION, LAM_RTOL, NEVER, compare_day, ensure_built, model,
                     to_dev, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    ensure_built()
    torch_cuda()


def test_device_philox_matches_oracle(golden_dir):
    torch = torch_cuda()
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0x0123456789ABCDEF
    out = capi.gabm_philox(seed, torch.from_numpy(ctr).cuda()).cpu().numpy()
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(0, 4099, 97):
        assert np.array_equal(out[i], O.philox4x32_10(ctr[i], key))
    import os
    for line in open(os.path.join(golden_dir, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        s = v[4] | (v[5] << 32)
        got = capi.gabm_philox(s, torch.tensor([v[0:4]], dtype=torch.uint32).cuda()).cpu().numpy()[0]
        assert [int(x) for x in got] == v[6:10]


def _params(T, R=2.5, m=0.01, inst=1):
    return (np.full((inst, T), R, np.float32), np.full((inst, T), m, np.float32),
            np.tile(synth.SUSCEPTIBILITY, (inst, 1)).astype(np.float32))


@pytest.mark.parametrize("n,n_seed", [(10_000, 20), (10_007, 1), (33, 33), (1, 0), (1, 1), (5000, 0)])
def test_seeds_match_oracle(n, n_seed):
    pop = synth.population_small(n=n, seed=3) if n > 1 else synth.Population(
        n=1, rowptr=np.zeros(2, np.uint64), col=np.zeros(0, np.uint32), w=np.zeros(0, np.float32),
        age=np.zeros(1, np.uint8))
    md = model(seed=11)
    ctx = capi.gabm_create([pop], md)
    R, m, S = _params(1, R=0.0)
    R, m, S = to_dev(R, m, S)
    capi.gabm_forward(ctx, 1, R, m, S, [n_seed])
    e = capi.gabm_get_state(ctx)[0]
    rows = O.select_seeds(n, 11, 0, n_seed)
    expect = np.full(n, NEVER, np.int16)
    expect[rows] = -4
    assert np.array_equal(e, expect)


def test_lockstep_days_10k():
    """Every day of the 10k-agent 30-day run: the GPU starts from the oracle's state."""
    pop = synth.population_small()
    T = 30
    md = model(seed=0)
    md_o = O.Model(4, 7, md.c, seed=0)
    R, m, S = _params(T)
    ref = O.forward_hard(pop, md_o, R[0], m[0], S[0], n_seed=20, want_hist=True)
    ctx = capi.gabm_create([pop], md)
    Rd, md_, Sd = to_dev(R, m, S)
    worst, flips, drawn = 0.0, 0, 0
    for t in range(T):
        capi.gabm_set_state(ctx, t, ref["e_hist"][t][None, :])
        D, counts = capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd,
                                      want_counts=True)
        rel, f, s = compare_day(pop, md_o, ctx, t, R[0], S[0], ref["e_hist"][t])
        worst, flips, drawn = max(worst, rel), flips + f, drawn + s
        assert np.array_equal(counts.cpu().numpy()[0, t], ref["counts"][t])
        assert D.cpu().numpy()[0, t] == pytest.approx(ref["D"][t], rel=1e-15, abs=1e-15)
    assert worst <= LAM_RTOL, worst
    assert flips <= max(1, FLIP_FRACTION * pop.n)
    assert ref["counts"][-1, 0] < pop.n - 1000  # the epidemic took off


def test_free_running_matches_oracle_exactly():
    pop = synth.population_small(n=10_007, seed=5)
    T = 30
    for seed in range(20):
        md_o = O.Model(4, 7, synth.infectiousness_table(), seed=seed)
        R, m, S = _params(T, R=2.7)
        ref = O.forward_hard(pop, md_o, R[0], m[0], S[0], n_seed=15)
        if ref["margin"] > EXACT_MARGIN:
            break
    assert ref["margin"] > EXACT_MARGIN
    ctx = capi.gabm_create([pop], model(seed=seed))
    Rd, md_, Sd = to_dev(R, m, S)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [15], want_counts=True)
    assert np.array_equal(capi.gabm_get_state(ctx)[0], ref["e_final"])
    assert np.array_equal(counts.cpu().numpy()[0], ref["counts"])
    assert np.allclose(D.cpu().numpy()[0], ref["D"], rtol=1e-15, atol=0)
    # host buffers through the same call give the same result
    D2, c2 = capi.gabm_forward(ctx, T, R, m, S, [15], want_counts=True)
    assert np.array_equal(D2, D.cpu().numpy()) and np.array_equal(c2, counts.cpu().numpy())
    # repeated runs are bitwise identical
    D3, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [15])
    assert np.array_equal(D3.cpu().numpy(), D.cpu().numpy())


@pytest.mark.parametrize("knobs", [{"GABM_FWD_SMEM_BITS": "1"}, {"GABM_SELL_SIGMA": "1"},
                                   {"GABM_SELL_SIGMA": "128"}])
def test_layout_and_bitmap_variants_are_bitwise_equal(knobs, monkeypatch):
    """The shared-memory copy of the infectious bitmap and other degree-sorting windows
    change only where data sit, not what is summed or in which order: same state, same D."""
    pop = synth.population_small(n=10_007, seed=5)
    T = 30
    R, m, S = _params(T, R=2.7)
    Rd, md_, Sd = to_dev(R, m, S)
    base = capi.gabm_create([pop], model(seed=3))
    D0, c0 = capi.gabm_forward(base, T, Rd, md_, Sd, [15], want_counts=True)
    for k, v in knobs.items():
        monkeypatch.setenv(k, v)
    var = capi.gabm_create([pop], model(seed=3))
    D1, c1 = capi.gabm_forward(var, T, Rd, md_, Sd, [15], want_counts=True)
    e0, e1 = capi.gabm_get_state(base)[0], capi.gabm_get_state(var)[0]
    if "GABM_SELL_SIGMA" in knobs:
        # another relabelling may sum a row's entries in another order: from one common
        # state, the day's lambdas agree within the lambda bar
        capi.gabm_forward(base, 12, Rd[:, :12].contiguous(), md_[:, :12].contiguous(), Sd, [15])
        e12 = capi.gabm_get_state(base)
        lams = []
        for ctx in (base, var):
            capi.gabm_set_state(ctx, 12, e12)
            capi.gabm_forward(ctx, 13, Rd[:, :13].contiguous(), md_[:, :13].contiguous(), Sd)
            lams.append(capi.gabm_get_lambda(ctx, 12)[0])
        assert (lams[0] > 0).sum() > 100
        assert np.allclose(lams[1], lams[0], rtol=LAM_RTOL, atol=0)
        return
    assert np.array_equal(e0, e1)
    assert np.array_equal(D0.cpu().numpy(), D1.cpu().numpy())
    assert np.array_equal(c0.cpu().numpy(), c1.cpu().numpy())
    for t in (0, 11, 29):
        assert np.array_equal(capi.gabm_get_lambda(base, t)[0], capi.gabm_get_lambda(var, t)[0])
    # the same switch through the schedule API
    capi.gabm_set_schedule(base, fwd_smem_bitmap=1)
    assert capi.gabm_get_schedule(base)["fwd_smem_bitmap"] == 1
    D2, _ = capi.gabm_forward(base, T, Rd, md_, Sd, [15])
    assert np.array_equal(D2.cpu().numpy(), D0.cpu().numpy())
    assert capi.gabm_autotune(base, 1)["fwd_smem_bitmap"] in (0, 1)
    assert np.array_equal(capi.gabm_get_state(base)[0], e0)


@pytest.mark.parametrize("order", [capi.GABM_ORDER_INPUT, capi.GABM_ORDER_BFS, capi.GABM_ORDER_COMMUNITY])
def test_agent_orders_agree(order):
    """Every device layout of the agents gives the oracle's day steps (ids stay the caller's)."""
    pop = synth.population_small(n=3001, seed=7)
    T = 20
    R, m, S = _params(T, R=3.0)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=2)
    ref = O.forward_hard(pop, md_o, R[0], m[0], S[0], n_seed=9, want_hist=True)
    ctx = capi.gabm_create([pop], model(seed=2, order=order))
    Rd, md_, Sd = to_dev(R, m, S)
    for t in (0, 7, 13, 19):
        capi.gabm_set_state(ctx, t, ref["e_hist"][t][None, :])
        capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
        rel, flips, _ = compare_day(pop, md_o, ctx, t, R[0], S[0], ref["e_hist"][t])
        assert rel <= LAM_RTOL and flips <= 1
    # seeds and the full run are keyed by the caller's ids in both layouts
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, [9], want_counts=True)
    assert np.array_equal(np.sort(np.flatnonzero(capi.gabm_get_state(ctx)[0] == -4)),
                          np.sort(O.select_seeds(pop.n, 2, 0, 9)))


def test_order_tuned_creation_keeps_the_fastest_layout():
    """gabm_create_order_tuned times every candidate layout and returns one that runs the
    workload exactly as a ctx created directly with that layout."""
    pop = synth.population_typed(20_000, seed=3)
    T = 15
    R, m, S = _params(T, R=3.0)
    Rd, md_, Sd = to_dev(R, m, S)
    ctx, times = capi.gabm_create_order_tuned([pop], model(seed=4), Rd, md_, Sd, [12])
    assert set(times) == {capi.GABM_ORDER_COMMUNITY, capi.GABM_ORDER_BFS}
    assert all(v > 0 for v in times.values())
    chosen = min(times, key=times.get)
    ref = capi.gabm_create([pop], model(seed=4, order=chosen))
    D0, _ = capi.gabm_forward(ctx, T, Rd, md_, Sd, [12])
    D1, _ = capi.gabm_forward(ref, T, Rd, md_, Sd, [12])
    assert np.array_equal(D0.cpu().numpy(), D1.cpu().numpy())
    assert np.array_equal(capi.gabm_get_state(ctx)[0], capi.gabm_get_state(ref)[0])


def test_directed_graph_and_hubs():
    """Asymmetric weights (a transposed weight would show) and rows longer than a warp pass."""
    pop = synth.random_directed(2000, 12.0, seed=4)
    # add a hub row with many in-neighbours
    hub_cols = np.arange(1, 1500, dtype=np.uint32)
    rowptr = pop.rowptr.astype(np.int64)
    col = np.concatenate([hub_cols, pop.col[rowptr[1]:]]).astype(np.uint32)
    w = np.concatenate([np.linspace(0.1, 2.0, hub_cols.size).astype(np.float32), pop.w[rowptr[1]:]])
    rp = rowptr.copy()
    rp[1:] = rowptr[1:] - rowptr[1] + hub_cols.size
    pop = synth.Population(n=pop.n, rowptr=rp.astype(np.uint64), col=col, w=w, age=pop.age)
    T = 25
    R, m, S = _params(T, R=3.0)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=1)
    ref = O.forward_hard(pop, md_o, R[0], m[0], S[0], n_seed=30, want_hist=True)
    ctx = capi.gabm_create([pop], model(seed=1))
    Rd, md_, Sd = to_dev(R, m, S)
    worst = 0.0
    for t in range(0, T, 3):
        capi.gabm_set_state(ctx, t, ref["e_hist"][t][None, :])
        capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
        rel, flips, _ = compare_day(pop, md_o, ctx, t, R[0], S[0], ref["e_hist"][t])
        worst = max(worst, rel)
        assert flips <= 1
    assert worst <= LAM_RTOL


def test_multi_graph_batch():
    """Uneven graphs concatenated in one ctx: each instance matches its own oracle run."""
    pops = [synth.population_small(n=n, seed=10 + i) for i, n in enumerate((1000, 4321, 77, 2500))]
    T = 25
    I = len(pops)
    rng = np.random.default_rng(4)
    R = rng.uniform(2.0, 3.5, (I, T)).astype(np.float32)
    m = rng.uniform(0.005, 0.05, (I, T)).astype(np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (I, 1)).astype(np.float32)
    S[2] *= 1.3
    n_seed = [5, 12, 3, 0]
    ctx = capi.gabm_create(pops, model(seed=4))
    Rd, md_, Sd = to_dev(R, m, S)
    D, counts = capi.gabm_forward(ctx, T, Rd, md_, Sd, n_seed, want_counts=True)
    D, counts = D.cpu().numpy(), counts.cpu().numpy()
    e = capi.gabm_get_state(ctx)[0]
    off = 0
    for g, pop in enumerate(pops):
        md_o = O.Model(4, 7, synth.infectiousness_table(), seed=4)
        ref = O.forward_hard(pop, md_o, R[g], m[g], S[g], n_seed=n_seed[g], inst=g, want_hist=True)
        seg = slice(off, off + pop.n)
        if ref["margin"] > EXACT_MARGIN:
            assert np.array_equal(e[seg], ref["e_final"])
            assert np.array_equal(counts[g], ref["counts"])
            assert np.allclose(D[g], ref["D"], rtol=1e-15, atol=0)
        off += pop.n
    # lockstep on one day for every graph at once
    t = 10
    e_start = np.concatenate([O.forward_hard(p, O.Model(4, 7, synth.infectiousness_table(), seed=4), R[g], m[g],
                                             S[g], n_seed=n_seed[g], inst=g, want_hist=True)["e_hist"][t]
                              for g, p in enumerate(pops)])
    capi.gabm_set_state(ctx, t, e_start[None, :])
    capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
    off = 0
    for g, pop in enumerate(pops):
        seg = slice(off, off + pop.n)
        md_o = O.Model(4, 7, synth.infectiousness_table(), seed=4)
        rel, flips, _ = compare_day(pop, md_o, ctx, t, R[g], S[g], e_start[seg], inst_slice=seg, inst=g)
        assert rel <= LAM_RTOL and flips <= 1
        off += pop.n


def test_degenerate_inputs():
    c = synth.infectiousness_table()
    # edgeless graph: nobody but the seeds is ever infected
    empty = synth.Population(n=300, rowptr=np.zeros(301, np.uint64), col=np.zeros(0, np.uint32),
                             w=np.zeros(0, np.float32), age=np.zeros(300, np.uint8))
    ctx = capi.gabm_create([empty], model())
    R, m, S = to_dev(*_params(20, R=5.0))
    D, counts = capi.gabm_forward(ctx, 20, R, m, S, [7], want_counts=True)
    assert np.all(counts.cpu().numpy()[0, :, 0] == 293)
    assert D.cpu().numpy()[0, 7] == pytest.approx(0.07, rel=1e-6)
    # R = 0: no transmission
    pop = synth.population_small(n=2000, seed=9)
    ctx = capi.gabm_create([pop], model())
    R, m, S = to_dev(*_params(15, R=0.0))
    _, counts = capi.gabm_forward(ctx, 15, R, m, S, [10], want_counts=True)
    assert np.all(counts.cpu().numpy()[0, :, 0] == 1990)
    # T = 1 and a short-L model (tau_EI = tau_IR = 1)
    md2 = model(c=np.array([0.0, 1.0], np.float32), tau_EI=1, tau_IR=1, seed=3)
    ctx = capi.gabm_create([pop], md2)
    R1, m1, S1 = _params(1, R=4.0)
    D, counts = capi.gabm_forward(ctx, 1, *to_dev(R1, m1, S1), [50], want_counts=True)
    ref = O.forward_hard(pop, O.Model(1, 1, md2.c, seed=3), R1[0], m1[0], S1[0], n_seed=50)
    assert np.array_equal(counts.cpu().numpy()[0], ref["counts"])
    # errors that need a live ctx
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_forward(ctx, 0, *to_dev(R1[:, :0], m1[:, :0], S1), [1])
    assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(ValueError):   # the binding checks shapes before the call
        capi.gabm_forward(ctx, 2, *to_dev(R1, m1, S1), [1])
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_forward(ctx, 1, *to_dev(R1, m1, S1), [pop.n + 1])
    assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_set_state(ctx, 3, np.full((1, pop.n), 5, np.int16))
    assert ei.value.status == capi.GABM_EINVAL


@pytest.fixture(scope="module")
def full_size():
    """The 1M-agent, 60-day workload (typed households/schools/workplaces/random contacts)."""
    pop = synth.population_typed(1_000_000, seed=0)
    T = 60
    R, m, S = _params(T, R=2.5, m=0.01)
    md_o = O.Model(4, 7, synth.infectiousness_table(), seed=0)
    ref = O.forward_hard(pop, md_o, R[0], m[0], S[0], n_seed=20, want_hist=True)
    return pop, T, R, m, S, md_o, ref


def test_full_size_lockstep_sampled_days(full_size):
    pop, T, R, m, S, md_o, ref = full_size
    ctx = capi.gabm_create([pop], model(seed=0))
    Rd, md_, Sd = to_dev(R, m, S)
    flips_total, drawn_total = 0, 0
    for t in (0, 20, 40, 50, 59):
        capi.gabm_set_state(ctx, t, ref["e_hist"][t][None, :])
        capi.gabm_forward(ctx, t + 1, Rd[:, :t + 1].contiguous(), md_[:, :t + 1].contiguous(), Sd)
        rel, flips, drawn = compare_day(pop, md_o, ctx, t, R[0], S[0], ref["e_hist"][t])
        assert rel <= LAM_RTOL, (t, rel)
        assert flips <= FLIP_FRACTION * pop.n
        flips_total += flips
        drawn_total += drawn
    assert drawn_total > 4_000_000


def test_full_size_free_run_properties(full_size):
    """At full size a few near-tie flips can make trajectories diverge, so the free run is
    checked through properties that hold at any size, plus closeness of the epidemic curve."""
    pop, T, R, m, S, md_o, ref = full_size
    ctx = capi.gabm_create([pop], model(seed=0))
    D, counts = capi.gabm_forward(ctx, T, *to_dev(R, m, S), [20], want_counts=True)
    counts = counts.cpu().numpy()[0]
    assert np.all(counts.sum(axis=1) == pop.n)
    assert np.all(np.diff(counts[:, 0]) <= 0) and np.all(np.diff(counts[:, 3]) >= 0)
    e = capi.gabm_get_state(ctx)[0]
    assert np.array_equal(np.sort(np.flatnonzero(e == -4)), np.sort(O.select_seeds(pop.n, 0, 0, 20)))
    assert np.all((e == NEVER) | ((e >= -4) & (e < T)))
    # day-by-day counts equal the oracle's until the first divergence (usually never)
    same = np.all(counts == ref["counts"], axis=1)
    first_diff = int(np.argmin(same)) if not same.all() else T
    assert first_diff >= 30
    assert abs(int(counts[-1, 0]) - int(ref["counts"][-1, 0])) <= 0.02 * (pop.n - int(ref["counts"][-1, 0]))
