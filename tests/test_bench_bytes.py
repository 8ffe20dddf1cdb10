"""The bench's algorithmic byte counts (the roofline's numerator) against a per-row count
written from the day kernels' access rules, on small trajectories (no GPU).

Forward day t, per row: state, flag read and clear and row length (8 bytes, every row);
a susceptible row with an in-neighbour infectious on day t reads its entries (8 bytes
each) and its age and caller id (5); an exposure on day t writes its state (2); the
lambda store writes 4 bytes per susceptible row; a row infectious on day t + 1 pushes
tomorrow's flags over its out-entries (4-byte column + 1-byte flag each; out-entries =
in-entries on these symmetric graphs).

Reverse day t, per row: state and row length (6 bytes, every row); a row that needs
gx(t+1) (not a seed, exposed on day t + 2 - L or later or never, and t + 1 < T) reads its
entries and writes its ring slot; a susceptible row reads its age, the ring slots k = 2..L-1
with t + k < T, the stored lambda, A when it is exposed after day t, writes A when it is
exposed on day t, and writes r; 72 bytes of per-tile partial sums per tile."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2207_09714_gb300 import synth  # noqa: E402

NEVER = 32767


def _per_row_counts(pop, E, T, L, n_rows, store):
    deg = np.diff(pop.rowptr.astype(np.int64))
    rp = pop.rowptr.astype(np.int64)
    col = pop.col.astype(np.int64)

    def infectious(i, d):
        return E[i] != NEVER and 1 <= d - E[i] < L

    fwd, bwd = np.zeros(T), np.zeros(T)
    for t in range(T):
        f = 8.0 * n_rows
        b = 6.0 * n_rows + 72.0 * (n_rows // 32)
        ring_reads = sum(1 for k in range(2, L) if t + k < T)
        for i in range(pop.n):
            e = int(E[i])
            seed = e != NEVER and e < 0
            never = e == NEVER
            sus = not seed and e >= t
            if sus and any(infectious(j, t) for j in col[rp[i]:rp[i + 1]]):
                f += 8.0 * deg[i] + 5.0
            if e == t:
                f += 2.0
            if store and sus:
                f += 4.0
            if infectious(i, t + 1):
                f += 5.0 * deg[i]
            if t + 1 < T and not seed and (never or e >= t + 2 - L):
                b += 8.0 * deg[i] + 4.0
            if sus:
                b += 1.0 + 4.0 * ring_reads + 4.0 + (4.0 if store else 0.0)
                if not never and e != t:
                    b += 4.0
                if e == t:
                    b += 4.0
        fwd[t], bwd[t] = f, b
    return fwd, bwd


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_trajectory_bytes_match_a_per_row_count(seed):
    rng = np.random.default_rng(seed)
    pop = synth.population_typed(400 + 37 * seed, seed=seed)
    T, L = 18, 11
    # a trajectory's final exposure days: seeds before day 0, exposures, never exposed
    E = np.full(pop.n, NEVER, np.int64)
    k = rng.choice(pop.n, size=pop.n // 3, replace=False)
    E[k] = rng.integers(-L, T, size=k.size)
    n_rows = ((pop.n + 31) // 32) * 32
    for store in (True, False):
        fwd, bwd, _, _ = bench.trajectory_bytes(E, pop.degrees().astype(np.float64), T, L, n_rows, store,
                                                frontier=bench.frontier_counts(pop, E, T, L))
        f_ref, b_ref = _per_row_counts(pop, E, T, L, n_rows, store)
        assert np.array_equal(fwd, f_ref), (store, np.flatnonzero(fwd != f_ref))
        assert np.array_equal(bwd, b_ref), (store, np.flatnonzero(bwd != b_ref))
