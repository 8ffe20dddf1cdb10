"""Pins of the FP64 oracle against things other than itself (no GPU needed).

Each test checks the oracle against a published value, a closed form, an
exact enumeration, a mean-field limit, an invariant the paper states, or a
finite-difference derivative, chosen so that a plausible slip in the oracle
(a dropped normalisation, an off-by-one day, a transposed weight, a sign in
the adjoint) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import brute, meanfield
from paper_2207_09714_gb300 import synth

NEVER = O.NEVER


def _kat_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat_rows(golden_dir)
    assert len(rows) == 3
    for r in rows:
        out = O.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_uniform_exact_in_fp32_and_unbiased():
    ids = np.arange(200_000, dtype=np.uint32)
    u = O.uniform(12345, ids, day=3, inst=2, stream=0)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    k = u * 2.0 ** 24
    assert np.all(k == np.round(k)) and np.all(np.round(k).astype(np.int64) % 2 == 1)
    se = math.sqrt(1 / 12 / u.size)
    assert abs(u.mean() - 0.5) < 5 * se
    # different days / instances / streams give different draws
    assert not np.array_equal(u, O.uniform(12345, ids, day=4, inst=2, stream=0))
    assert not np.array_equal(u, O.uniform(12345, ids, day=3, inst=3, stream=0))
    assert not np.array_equal(u, O.uniform(12345, ids, day=3, inst=2, stream=1))
    # rough uniformity over 16 bins
    h = np.histogram(u, bins=16, range=(0, 1))[0]
    exp = u.size / 16
    assert np.all(np.abs(h - exp) < 5 * math.sqrt(exp))


def test_seed_selection_is_smallest_keys():
    n = 3000
    for inst in (0, 5):
        rows = O.select_seeds(n, seed=7, inst=inst, n_seed=25)
        h = O.hash_words(7, range(n), day=0, inst=inst, stream=1).astype(np.uint64)
        key = (h << np.uint64(32)) | np.arange(n, dtype=np.uint64)
        expect = np.argsort(key, kind="stable")[:25]
        assert np.array_equal(rows, expect)
    assert O.select_seeds(n, 7, 0, 0).size == 0
    assert np.array_equal(np.sort(O.select_seeds(50, 7, 0, 50)), np.arange(50))
    with pytest.raises(ValueError):
        O.select_seeds(50, 7, 0, 51)


def test_seed_selection_uniform_frequency():
    n, k, runs = 40, 4, 3000
    freq = np.zeros(n)
    for s in range(runs):
        freq[O.select_seeds(n, s, 0, k)] += 1
    p = k / n
    se = math.sqrt(p * (1 - p) / runs)
    assert np.all(np.abs(freq / runs - p) < 5 * se)


def test_seed_selection_follows_original_ids():
    n = 500
    rng = np.random.default_rng(3)
    perm = rng.permutation(n)            # old id i -> new row perm[i]
    orig_id = np.empty(n, np.uint32)
    orig_id[perm] = np.arange(n)          # new row r holds old agent orig_id[r]
    a = O.select_seeds(n, 11, 0, 9)
    b = O.select_seeds(n, 11, 0, 9, orig_id=orig_id)
    assert np.array_equal(np.sort(perm[a]), np.sort(b))


# ---------------------------------------------------------------- exact law
def _tiny_directed():
    # 5 agents, asymmetric weights: a transposed weight or wrong edge direction shows.
    n = 5
    edges = {(1, 0): 0.9, (2, 0): 0.3, (0, 1): 1.4, (3, 1): 0.5, (0, 2): 0.7, (1, 2): 1.1,
             (4, 3): 0.8, (2, 3): 1.3, (3, 4): 0.6, (0, 4): 0.2}
    # edges[(i, j)]: row i (destination) lists in-neighbour j
    rows = [[] for _ in range(n)]
    for (i, j), w in sorted(edges.items()):
        rows[i].append((j, w))
    rowptr = np.zeros(n + 1, np.uint64)
    col, ww = [], []
    for i in range(n):
        for j, w in rows[i]:
            col.append(j); ww.append(w)
        rowptr[i + 1] = len(col)
    age = np.array([0, 3, 6, 8, 2], np.uint8)
    return synth.Population(n=n, rowptr=rowptr, col=np.array(col, np.uint32),
                            w=np.array(ww, np.float32), age=age)


TINY = dict(tau_EI=1, tau_IR=2, c=np.array([0.0, 0.4, 0.6], np.float32))
TINY_R = np.array([3.0, 2.0, 4.0, 1.5, 3.5, 2.5], np.float32)
TINY_M = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6], np.float32)
TINY_S = np.array([1.2, 0.5, 1.0, 0.8, 1.5, 0.7, 1.1, 0.9, 1.3], np.float32)


def test_day_probabilities_match_enumerator():
    pop = _tiny_directed()
    md = O.Model(TINY["tau_EI"], TINY["tau_IR"], TINY["c"], seed=0)
    W = brute.dense_weights(pop)
    rng = np.random.default_rng(0)
    for trial in range(40):
        t = int(rng.integers(0, 6))
        e = np.array([NEVER if rng.random() < 0.5 else int(rng.integers(-3, t)) for _ in range(5)],
                     np.int16)
        out = O.day_hard(pop, md, t, TINY_R[t], TINY_S, e)
        p_exact = brute.infection_probs(W, [int(a) for a in pop.age], TINY_S, TINY["c"], 3,
                                        TINY_R[t], t, [int(v) for v in e])
        for i in range(5):
            if e[i] == NEVER:
                assert abs(out["p"][i] - p_exact[i]) <= 1e-15
            else:
                assert out["p"][i] == 0.0 and out["e_out"][i] == e[i]


def test_monte_carlo_matches_exact_law():
    pop = _tiny_directed()
    e0 = np.array([-1, NEVER, NEVER, NEVER, NEVER], np.int16)
    ED, ED2, P_inf, final = brute.exact_law(pop, TINY["tau_EI"], TINY["tau_IR"], TINY["c"],
                                            TINY_R, TINY_M, TINY_S, e0, T=6)
    assert abs(sum(final.values()) - 1.0) < 1e-12
    runs = 20_000
    Dsum = np.zeros(6)
    inf = np.zeros(5)
    for s in range(runs):
        md = O.Model(TINY["tau_EI"], TINY["tau_IR"], TINY["c"], seed=s)
        r = O.forward_hard(pop, md, TINY_R, TINY_M, TINY_S, e0=e0)
        Dsum += r["D"]
        inf += (r["e_final"] != NEVER) & (r["e_final"] >= 0)
    for t in range(6):
        var = ED2[t] - ED[t] ** 2
        se = math.sqrt(max(var, 0.0) / runs)
        assert abs(Dsum[t] / runs - ED[t]) <= 5 * se + 1e-12, (t, Dsum[t] / runs, ED[t])
    for i in range(5):
        se = math.sqrt(P_inf[i] * (1 - P_inf[i]) / runs)
        assert abs(inf[i] / runs - P_inf[i]) <= 5 * se + 1e-12, (i, inf[i] / runs, P_inf[i])


def test_two_agent_closed_form():
    # One seed, one susceptible, one symmetric interaction of weight w: Dbar = w, and the
    # susceptible escapes the seed's whole remaining infectious period with probability
    # exp(-R S (1 - kappa)), kappa = seed infectiousness spent before day 0.
    c = synth.infectiousness_table()
    w = 0.8
    pop = synth.Population(n=2, rowptr=np.array([0, 1, 2], np.uint64), col=np.array([1, 0], np.uint32),
                           w=np.array([w, w], np.float32), age=np.array([4, 6], np.uint8))
    R = np.full(12, 0.7, np.float32)
    m = np.full(12, 0.01, np.float32)
    e0 = np.array([-4, NEVER], np.int16)
    kappa = float(np.sum(c[1:4].astype(np.float64)))
    S1 = float(synth.SUSCEPTIBILITY[6])
    p_escape = math.exp(-0.7 * S1 * (1.0 - kappa))
    runs = 20_000
    esc = 0
    for s in range(runs):
        r = O.forward_hard(pop, O.Model(4, 7, c, seed=s), R, m, synth.SUSCEPTIBILITY, e0=e0)
        esc += r["e_final"][1] == NEVER
    se = math.sqrt(p_escape * (1 - p_escape) / runs)
    assert abs(esc / runs - p_escape) < 5 * se
    # per-day probability: p = 1 - exp(-R S c[t + 4])
    for t in range(0, 8):
        out = O.day_hard(pop, O.Model(4, 7, c), t, 0.7, synth.SUSCEPTIBILITY,
                         np.array([-4, NEVER], np.int16))
        k = t + 4
        ck = float(c[k]) if k < 11 else 0.0
        assert abs(out["p"][1] - (1 - math.exp(-0.7 * S1 * ck))) < 1e-15


def test_zero_transmission_and_empty_graph():
    pop = synth.population_small(n=2000, seed=1)
    c = synth.infectiousness_table()
    T = 25
    R0 = np.zeros(T, np.float32)
    m = np.full(T, 0.01, np.float32)
    r = O.forward_hard(pop, O.Model(4, 7, c), R0, m, synth.SUSCEPTIBILITY, n_seed=20)
    assert np.all(r["counts"][:, 0] == pop.n - 20)
    assert np.sum(r["e_final"] != NEVER) == 20
    empty = synth.Population(n=300, rowptr=np.zeros(301, np.uint64), col=np.zeros(0, np.uint32),
                             w=np.zeros(0, np.float32), age=np.zeros(300, np.uint8))
    r = O.forward_hard(empty, O.Model(4, 7, c), np.full(T, 3.0, np.float32), m,
                       synth.SUSCEPTIBILITY, n_seed=5)
    assert np.all(r["counts"][:, 0] == 295)
    assert r["D"][7] == pytest.approx(float(m[7]) * 5)  # seeds reach RM after tau_IR days


def test_conservation_monotonicity_and_state_rules():
    pop = synth.population_small()
    c = synth.infectiousness_table()
    T = 30
    R = np.full(T, 2.5, np.float32)
    m = np.full(T, 0.01, np.float32)
    r = O.forward_hard(pop, O.Model(4, 7, c, seed=0), R, m, synth.SUSCEPTIBILITY, n_seed=20,
                       want_hist=True)
    cnt = r["counts"]
    assert np.all(cnt.sum(axis=1) == pop.n)
    assert np.all(np.diff(cnt[:, 0]) <= 0)
    assert np.all(np.diff(cnt[:, 3]) >= 0)
    eh = r["e_hist"]
    for t in range(T):
        changed = eh[t + 1] != eh[t]
        assert np.all(eh[t][changed] == NEVER)
        assert np.all(eh[t + 1][changed] == t)
    # D_t = m_t x (agents entering RM on day t) = m_t x increase of RM
    dRM = np.diff(np.concatenate([cnt[:, 3], [0]]))[:-1]
    assert np.allclose(r["D"][1:], m[1:] * dRM, rtol=0, atol=1e-12)
    assert np.array_equal(r["e_final"], eh[T])


def test_permutation_invariance():
    pop = synth.population_small(n=5000, seed=2)
    c = synth.infectiousness_table()
    T = 30
    R = np.full(T, 2.8, np.float32)
    m = np.full(T, 0.02, np.float32)
    rng = np.random.default_rng(9)
    perm = rng.permutation(pop.n)
    pp = synth.permute(pop, perm)
    orig_id = np.empty(pop.n, np.uint32)
    orig_id[perm] = np.arange(pop.n)
    md = O.Model(4, 7, c, seed=5)
    a = O.forward_hard(pop, md, R, m, synth.SUSCEPTIBILITY, n_seed=15)
    b = O.forward_hard(pp, md, R, m, synth.SUSCEPTIBILITY, n_seed=15, orig_id=orig_id)
    assert np.array_equal(a["D"], b["D"])
    assert np.array_equal(a["counts"], b["counts"])
    assert np.array_equal(a["e_final"], b["e_final"][perm])
    assert a["counts"][-1, 0] < pop.n - 100  # the epidemic did take off


@pytest.fixture(scope="module")
def complete_runs():
    n, R0 = 2048, 2.5
    pop = synth.complete_graph(n, age_bin=2)   # S[2] = 1
    c = synth.infectiousness_table()
    T = 120
    ns = int(0.01 * n)
    R = np.full(T, R0, np.float32)
    m = np.full(T, 0.01, np.float32)
    runs = [O.forward_hard(pop, O.Model(4, 7, c, seed=s), R, m, synth.SUSCEPTIBILITY, n_seed=ns)
            for s in range(16)]
    return dict(n=n, R0=R0, c=c, T=T, ns=ns, runs=runs)


def test_mean_field_curve(complete_runs):
    d = complete_runs
    new, E, I = meanfield.daily_recurrence(d["n"], d["R0"], d["c"], 4, 7, d["ns"], d["T"])
    I_sim = np.mean([r["counts"][:, 2] for r in d["runs"]], axis=0) / d["n"]
    E_sim = np.mean([r["counts"][:, 1] for r in d["runs"]], axis=0) / d["n"]
    assert np.abs(I_sim - I / d["n"]).max() < 0.02
    assert np.abs(E_sim - E / d["n"]).max() < 0.02


def test_final_size_relation(complete_runs):
    d = complete_runs
    z_sim = np.mean([np.mean(r["e_final"] != NEVER) for r in d["runs"]])
    for r in d["runs"]:
        assert r["counts"][-1, 1] + r["counts"][-1, 2] == 0  # epidemic over
    z = meanfield.final_size(d["n"], d["R0"], d["c"], 4, d["ns"])
    assert 0.85 < z < 0.95
    assert abs(z_sim - z) < 0.02


# ---------------------------------------------------------------- adjoint
def test_dy_dlambda_matches_finite_difference():
    for lam in (1e-6, 1e-3, 0.05, 0.7, 3.0):
        for u in (1e-5, 0.01, 0.3, 0.5, 0.97):
            h = 1e-3 * lam
            d1 = (O.y_soft(lam + h, u) - O.y_soft(lam - h, u)) / (2 * h)
            d2 = (O.y_soft(lam + 2 * h, u) - O.y_soft(lam - 2 * h, u)) / (4 * h)
            fd = (4 * d1 - d2) / 3   # Richardson: truncation error O(h^4)
            an = O.dy_dlambda(lam, u)
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-11, (lam, u, fd, an)
    # finite limit at p = 0 equals (1 - u) / u
    assert O.dy_dlambda(0.0, 0.25) == pytest.approx(3.0, rel=1e-15)


def test_mse_gradient():
    rng = np.random.default_rng(1)
    D = rng.random(9); y = rng.random(9)
    loss, gD = O.mse(D, y)
    assert loss == pytest.approx(np.mean((D - y) ** 2), rel=1e-15)
    for t in range(9):
        h = 1e-6
        Dp = D.copy(); Dp[t] += h
        Dm = D.copy(); Dm[t] -= h
        fd = (O.mse(Dp, y)[0] - O.mse(Dm, y)[0]) / (2 * h)
        assert abs(fd - gD[t]) < 1e-8


def _soft_setup():
    pop = synth.population_small(n=240, seed=4, er_mean_degree=6)
    c = synth.infectiousness_table()
    T = 22
    rng = np.random.default_rng(8)
    R = rng.uniform(1.5, 3.5, T).astype(np.float32)
    m = rng.uniform(0.01, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY.copy()
    y = rng.uniform(0, 0.3, T)
    md = O.Model(4, 7, c, seed=3)
    return pop, md, R, m, S, y


def _soft_loss(pop, md, R, m, S, y):
    f = O.forward_soft(pop, md, R, m, S, n_seed=6)
    return O.mse(f["D"], y)[0]


def _seed_days(pop, md, n_seed, inst=0):
    """Initial exposure days of the seeded state: -tau_EI for the seeds, NEVER elsewhere."""
    e0 = np.full(pop.n, NEVER, np.int16)
    e0[O.select_seeds(pop.n, md.seed, inst, n_seed)] = -md.tau_EI
    return e0


def test_soft_adjoint_matches_central_differences():
    pop, md, R, m, S, y = _soft_setup()
    f = O.forward_soft(pop, md, R, m, S, n_seed=6)
    loss, gD = O.mse(f["D"], y)
    g = O.backward_soft(pop, md, R, m, S, gD, f["s_hist"], f["y_hist"], f["dydl_hist"],
                        f["Lam_hist"], f["newRM"], e0=_seed_days(pop, md, 6))
    assert np.abs(g["dR"]).max() > 0 and np.abs(g["dS"]).max() > 0
    assert g["dc"][0] == 0.0 and np.abs(g["dc"][1:]).min() > 0

    # Central differences with Richardson extrapolation; the steps are powers of two that
    # are multiples of the parameter's fp32 spacing, so the perturbed fp32 inputs are exact.
    for name, vec, n_check in (("R", R, len(R)), ("m", m, len(m)), ("S", S, 9)):
        for idx in range(n_check):
            base = float(vec[idx])
            h = 2.0 ** (math.floor(math.log2(max(1.0, abs(base)))) - 12)
            # Richardson extrapolation of central differences with steps h and 2h
            def L_at(delta):
                v = vec.copy()
                v[idx] = np.float32(base + delta)
                assert float(v[idx]) == base + delta  # exact in fp32
                args = dict(R=R, m=m, S=S)
                args[name] = v
                return _soft_loss(pop, md, args["R"], args["m"], args["S"], y)
            d1 = (L_at(h) - L_at(-h)) / (2 * h)
            d2 = (L_at(2 * h) - L_at(-2 * h)) / (4 * h)
            est = (4 * d1 - d2) / 3
            an = {"R": g["dR"], "m": g["dm"], "S": g["dS"]}[name][idx]
            ref = max(abs(an), 1e-9 * max(np.abs(g["dR"]).max(), 1.0))
            assert abs(est - an) <= 1e-6 * ref + 1e-12, (name, idx, est, an)

    # the infectiousness table c[1..L-1] (c[0] = 0 is fixed by A2)
    for k in range(1, md.L):
        base = float(md.c[k])
        h = 2.0 ** (math.floor(math.log2(max(1.0, abs(base)))) - 12)
        def Lc_at(delta):
            c = md.c.copy()
            c[k] = np.float32(base + delta)
            assert float(c[k]) == base + delta
            return _soft_loss(pop, O.Model(md.tau_EI, md.tau_IR, c, seed=md.seed), R, m, S, y)
        d1 = (Lc_at(h) - Lc_at(-h)) / (2 * h)
        d2 = (Lc_at(2 * h) - Lc_at(-2 * h)) / (4 * h)
        est = (4 * d1 - d2) / 3
        an = g["dc"][k]
        assert abs(est - an) <= 1e-6 * max(abs(an), 1e-9) + 1e-12, ("c", k, est, an)


def test_hard_adjoint_is_soft_adjoint_at_hard_values():
    pop = synth.population_small(n=3000, seed=6)
    c = synth.infectiousness_table()
    T = 35
    rng = np.random.default_rng(2)
    R = rng.uniform(2.0, 3.5, T).astype(np.float32)
    m = rng.uniform(0.005, 0.05, T).astype(np.float32)
    S = synth.SUSCEPTIBILITY
    md = O.Model(4, 7, c, seed=9)
    f = O.forward_hard(pop, md, R, m, S, n_seed=12, want_Lam=True)
    E = f["e_final"].astype(np.int64)
    y = rng.uniform(0, 2, T)
    loss, gD = O.mse(f["D"], y)
    h = O.backward_hard(pop, md, R, m, S, f["e_final"], gD)
    n = pop.n
    seeds = (E != NEVER) & (E < 0)
    s_hist = np.zeros((T + 1, n)); y_hist = np.zeros((T, n)); dydl = np.zeros((T, n))
    for t in range(T):
        S_t = ~seeds & ((E == NEVER) | (E >= t))
        s_hist[t] = S_t
        y_hist[t] = (E == t)
        u = O.uniform(md.seed, np.arange(n), day=t)
        lam = R[t].astype(np.float64) * S[pop.age].astype(np.float64) * f["Lam_hist"][t]
        dydl[t] = np.where(S_t, [O.dy_dlambda(a, b) if s else 0.0 for a, b, s in zip(lam, u, S_t)], 0.0)
    s_hist[T] = ~seeds & (E == NEVER)
    g = O.backward_soft(pop, md, R, m, S, gD, s_hist, y_hist, dydl, f["Lam_hist"],
                        f["newRM"].astype(np.float64), e0=np.where(seeds, E, NEVER))
    for k in ("dR", "dm", "dS", "dc"):
        ref = np.abs(h[k]).max()
        assert ref > 0
        assert np.allclose(g[k], h[k], rtol=1e-10, atol=1e-12 * ref), k
    assert np.array_equal(h["dm"], gD * f["newRM"])


def test_agent_location_expansion():
    """The one-hop weights of an agent-location graph, checked by hand on a small case:
    agents 0, 1, 2 share location A (weights 1, 2, 3), agents 1 and 2 also share B
    (weights 0.5, 4); agent 3 is alone at C."""
    from oracle import bipartite as OB
    bip = synth.Bipartite(n=4, n_loc=3, rowptr=np.array([0, 1, 3, 5, 6], np.uint64),
                          loc=np.array([0, 0, 1, 0, 1, 2], np.uint32),
                          w=np.array([1.0, 2.0, 0.5, 3.0, 4.0, 7.0], np.float32), age=np.zeros(4, np.uint8))
    W = OB.expand(bip)
    dense = np.zeros((4, 4))
    for i in range(4):
        for p in range(int(W.rowptr[i]), int(W.rowptr[i + 1])):
            dense[i, W.col[p]] = W.w64[p]
    ref = np.array([[0, 2, 3, 0], [2, 0, 6 + 2, 0], [3, 8, 0, 0], [0, 0, 0, 0]], np.float64)
    assert np.array_equal(dense, ref)
    assert OB.mean_weighted_degree(bip) == pytest.approx(ref.sum() / 4, rel=1e-15)
    # on a generated population: symmetric, no self pairs, Dbar from the incidence alone
    big = synth.population_bipartite(3000, seed=2)
    Wb = OB.expand(big)
    A = sp.csr_matrix((Wb.w64, Wb.col.astype(np.int64), Wb.rowptr.astype(np.int64)), shape=(big.n, big.n))
    assert abs(A - A.T).max() < 1e-12 and A.diagonal().max() == 0
    assert OB.mean_weighted_degree(big) == pytest.approx(Wb.w64.sum() / big.n, rel=1e-12)
