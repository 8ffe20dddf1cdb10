"""gabm_seed_state_noalloc: the entry point for callers that cannot let a library
allocate device memory (fixed memory budgets, memory owned by another framework's
pool).  Its output must equal the day-0 state the regular entry points build.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2207_09714_gb300 import build as gbuild
from paper_2207_09714_gb300 import capi, synth

from helpers import ensure_built, model, to_dev, torch_cuda


def _reference_state(pop, n_seed, seed):
    """Day-0 state from gabm_create + gabm_forward: one graph copy per instance
    (instance i = graph i), one day at R = 0 so nobody but the seeds is exposed."""
    I = len(n_seed)
    ctx = capi.gabm_create([pop] * I, model(seed=seed, order=capi.GABM_ORDER_INPUT))
    R = np.zeros((I, 1), np.float32)
    m = np.zeros((I, 1), np.float32)
    S = np.tile(synth.SUSCEPTIBILITY, (I, 1)).astype(np.float32)
    capi.gabm_forward(ctx, 1, *to_dev(R, m, S), n_seed)
    return capi.gabm_get_state(ctx)[0].reshape(I, pop.n)


@pytest.mark.gpu
def test_noalloc_state_matches_regular_entry_points():
    ensure_built()
    torch = torch_cuda()
    cases = [(synth.population_small(n=10_007, seed=3), [20, 1, 0, 3335], 77),
             (synth.population_small(n=4096, seed=4), [4096, 7], 5)]
    for pop, n_seed, seed in cases:
        ref = _reference_state(pop, n_seed, seed)
        out = torch.empty((len(n_seed), pop.n), dtype=torch.int16, device="cuda")
        for _ in range(2):   # two calls in a row share (and must clear) the fixed scratch
            out.fill_(123)
            capi.gabm_seed_state_noalloc(seed, pop.n, n_seed, 4, out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    gbuild.build()
    L = capi.load_library()
    seeds = np.zeros(capi.GABM_NUM_AGES + 20, np.int32)
    p = seeds.ctypes.data_as(ctypes.c_void_p)
    too_many = L.gabm_seed_state_noalloc(1, 100, 17, p, 4, None, None)
    assert too_many == capi.GABM_EINVAL
    assert "num_instances" in L.gabm_noalloc_last_error().decode()
    assert L.gabm_seed_state_noalloc(1, 1 << 28, 16, p, 4, None, None) == capi.GABM_EINVAL
    assert L.gabm_seed_state_noalloc(1, 0, 1, p, 4, None, None) == capi.GABM_EINVAL
