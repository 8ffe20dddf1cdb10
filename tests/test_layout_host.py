"""Device layouts of the agents, computed on the host through the C ABI (no GPU): every
order is a permutation, the community order keeps densely connected groups in nearby
rows, and bad arguments are rejected.  Results never depend on the layout (Sec. 2.3:
the aggregation is permutation invariant); these checks are about locality only."""
import numpy as np
import pytest

from paper_2207_09714_gb300 import build as gbuild
from paper_2207_09714_gb300 import capi, synth

ORDERS = (capi.GABM_ORDER_INPUT, capi.GABM_ORDER_BFS, capi.GABM_ORDER_COMMUNITY)


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    return capi.load_library()


def _cliques(n, k, er, seed):
    """n agents in cliques of k (random membership) plus Erdos-Renyi contacts of mean degree er."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    us, vs = [], []
    for c0 in range(0, n, k):
        a, b = np.meshgrid(perm[c0:c0 + k], perm[c0:c0 + k])
        us.append(a[a < b]); vs.append(b[a < b])
    e = int(n * er / 2)
    u = np.concatenate(us + [rng.integers(0, n, e)])
    v = np.concatenate(vs + [rng.integers(0, n, e)])
    pop = synth.csr_from_undirected(n, u, v, rng.uniform(0.5, 1.5, u.size), np.zeros(n, np.uint8), name="cliques")
    group = np.empty(n, np.int64)
    group[perm] = np.arange(n) // k
    return pop, group


def _edge_distance(pop, order):
    pos = np.empty(pop.n, np.int64)
    pos[order] = np.arange(pop.n)
    rows = np.repeat(np.arange(pop.n), np.diff(pop.rowptr.astype(np.int64)))
    return rows, np.abs(pos[rows] - pos[pop.col.astype(np.int64)])


@pytest.mark.parametrize("order", ORDERS)
def test_every_layout_is_a_permutation(order):
    for pop in (synth.population_typed(3000, seed=2), synth.random_directed(777, 5.0, seed=1),
                synth.population_typed(2000, seed=5, powerlaw=True, pl_kmax=400)):
        for sets in (1, 8):
            got = capi.gabm_agent_layout(pop, order, sets)
            assert got.shape == (pop.n,)
            assert np.array_equal(np.sort(got), np.arange(pop.n))
    one = synth.csr_from_undirected(1, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0), np.zeros(1, np.uint8))
    assert capi.gabm_agent_layout(one, order).tolist() == [0]


def test_community_order_keeps_groups_together():
    pop, group = _cliques(20_000, 20, 3.0, seed=1)
    rows, d = {}, {}
    for order in ORDERS:
        r, dist = _edge_distance(pop, capi.gabm_agent_layout(pop, order))
        rows[order], d[order] = r, dist
    same = group[rows[capi.GABM_ORDER_COMMUNITY]] == group[pop.col.astype(np.int64)]
    near = {o: float(np.mean(d[o][same] <= 1024)) for o in ORDERS}
    # each clique sits inside (or across the edge of) one 1024-row degree window
    assert near[capi.GABM_ORDER_COMMUNITY] >= 0.95, near
    assert near[capi.GABM_ORDER_COMMUNITY] > near[capi.GABM_ORDER_BFS] + 0.2, near
    assert near[capi.GABM_ORDER_BFS] > near[capi.GABM_ORDER_INPUT], near


def test_long_rows_are_grouped_with_one_set_per_graph():
    """Rows of more than 128 entries share tiles with each other only: they fill
    ceil(count / 32) tiles, 32 to a tile (the last group may be partial)."""
    pop = synth.population_typed(60_000, seed=3, powerlaw=True, pl_kmax=2000)
    deg = np.diff(pop.rowptr.astype(np.int64))
    n_long = int((deg > 128).sum())
    assert n_long >= 8
    for sets, grouped in ((1, True), (8, False)):
        order = capi.gabm_agent_layout(pop, capi.GABM_ORDER_COMMUNITY, sets)
        tiles = np.unique(np.flatnonzero(deg[order] > 128) // 32)
        if grouped:
            assert tiles.size == -(-n_long // 32)
        else:   # several sets per graph keep the degree windows only
            assert tiles.size >= 1


def test_layout_rejects_bad_arguments():
    pop = synth.population_typed(500, seed=1)
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_agent_layout(pop, 7)
    assert ei.value.status == capi.GABM_EINVAL
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_agent_layout(pop, capi.GABM_ORDER_BFS, 0)
    assert ei.value.status == capi.GABM_EINVAL
    bad = synth.Population(n=pop.n, rowptr=pop.rowptr, col=pop.col.copy(), w=pop.w, age=pop.age)
    bad.col[3] = pop.n + 5
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_agent_layout(bad, capi.GABM_ORDER_COMMUNITY)
    assert ei.value.status == capi.GABM_EINVAL
