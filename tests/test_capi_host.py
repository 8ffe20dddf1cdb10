"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/gabm.h declares, and host-side validation rejects bad input
before any CUDA call."""
import ctypes

import numpy as np
import pytest

from paper_2207_09714_gb300 import build as gbuild
from paper_2207_09714_gb300 import capi, synth


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return capi.load_library()


def test_exports_every_declared_symbol(lib):
    names = capi.header_functions()
    assert {"gabm_create", "gabm_forward", "gabm_backward", "gabm_mse_loss", "gabm_destroy"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name
    assert capi.gabm_version().startswith("gabm-gb300")


def _md(**kw):
    base = dict(tau_EI=4, tau_IR=7, c=synth.infectiousness_table())
    base.update(kw)
    return capi.ModelDesc(**base)


def _expect(status, graphs, md, sets=1):
    with pytest.raises(capi.GabmError) as ei:
        capi.gabm_create(graphs, md, sets_per_graph=sets)
    assert ei.value.status == status, str(ei.value)
    assert capi.load_library().gabm_last_error(None).decode()  # message is set
    return str(ei.value)


def test_create_rejects_bad_graphs(lib):
    pop = synth.population_small(n=200, seed=1)

    def mutate(**kw):
        d = dict(n=pop.n, rowptr=pop.rowptr.copy(), col=pop.col.copy(), w=pop.w.copy(), age=pop.age.copy())
        d.update(kw)
        return synth.Population(**d)

    rp = pop.rowptr.copy(); rp[5], rp[6] = rp[6], rp[5] + 0
    rp[5] = rp[6] + 3
    assert "rowptr" in _expect(capi.GABM_EINVAL, [mutate(rowptr=rp)], _md())
    rp0 = pop.rowptr.copy(); rp0[0] = 1
    _expect(capi.GABM_EINVAL, [mutate(rowptr=rp0)], _md())
    col = pop.col.copy(); col[10] = pop.n
    assert "out of range" in _expect(capi.GABM_EINVAL, [mutate(col=col)], _md())
    w = pop.w.copy(); w[3] = -1.0
    _expect(capi.GABM_EINVAL, [mutate(w=w)], _md())
    w = pop.w.copy(); w[4] = np.nan
    _expect(capi.GABM_EINVAL, [mutate(w=w)], _md())
    age = pop.age.copy(); age[7] = 9
    _expect(capi.GABM_EINVAL, [mutate(age=age)], _md())
    # the second graph is bad: still rejected, nothing created
    _expect(capi.GABM_EINVAL, [pop, mutate(age=age)], _md())


def test_create_rejects_bad_models(lib):
    pop = synth.population_small(n=64, seed=2)
    c = synth.infectiousness_table()
    c1 = c.copy(); c1[0] = 0.1
    assert "c[0]" in _expect(capi.GABM_EINVAL, [pop], _md(c=c1))
    c2 = c.copy(); c2[3] = -0.2
    _expect(capi.GABM_EINVAL, [pop], _md(c=c2))
    _expect(capi.GABM_EINVAL, [pop], _md(tau_EI=0, c=c[:7]))
    _expect(capi.GABM_EINVAL, [pop], _md(tau_EI=20, tau_IR=20, c=np.zeros(40, np.float32)))
    _expect(capi.GABM_EUNSUPPORTED, [pop], _md(gumbel_tau=0.5))
    _expect(capi.GABM_EUNSUPPORTED, [pop], _md(relax_mode=capi.GABM_SOFT, lambda_policy=capi.GABM_RECOMPUTE))
    _expect(capi.GABM_EUNSUPPORTED, [pop], _md(relax_mode=capi.GABM_SOFT), sets=2)
    _expect(capi.GABM_EINVAL, [pop], _md(lambda_policy=7))
    _expect(capi.GABM_EINVAL, [pop], _md(), sets=0)
    _expect(capi.GABM_EINVAL, [], _md())
    # progression variants: the sampled R/M split (tau_IM) and stochastic I-stage durations (p_IR)
    c11 = synth.infectiousness_table(4, 7)
    _expect(capi.GABM_EINVAL, [pop], _md(tau_IM=-2))
    _expect(capi.GABM_EINVAL, [pop], _md(tau_IM=40, c=np.r_[0.0, np.full(43, 0.02)].astype(np.float32)))
    pmf = np.full(7, 1 / 7, np.float32)
    _expect(capi.GABM_EINVAL, [pop], _md(p_IR=np.r_[pmf[:6], -1.0].astype(np.float32)))
    _expect(capi.GABM_EINVAL, [pop], _md(p_IR=np.zeros(7, np.float32)))
    for kw, sets in ((dict(tau_IM=9, c=synth.infectiousness_table(4, 9), relax_mode=capi.GABM_SOFT), 1),
                     (dict(tau_IM=9, c=synth.infectiousness_table(4, 9)), 2),
                     (dict(p_IR=pmf, lambda_policy=capi.GABM_RECOMPUTE), 1),
                     (dict(p_IR=pmf, tau_IM=5, c=c11), 1)):
        _expect(capi.GABM_EUNSUPPORTED, [pop], _md(**kw), sets=sets)
    with pytest.raises(ValueError):
        capi.gabm_create([pop], _md(tau_IM=9))   # c must have tau_EI + max(tau_IR, tau_IM) = 13 entries
    # SIRS reinfection (tau_RS)
    _expect(capi.GABM_EINVAL, [pop], _md(tau_RS=-1))
    for kw, sets in ((dict(tau_RS=5, relax_mode=capi.GABM_SOFT), 1), (dict(tau_RS=5), 3),
                     (dict(tau_RS=5, lambda_policy=capi.GABM_RECOMPUTE), 1), (dict(tau_RS=5, p_IR=pmf), 1),
                     (dict(tau_RS=5, tau_IM=9, c=synth.infectiousness_table(4, 9)), 1)):
        _expect(capi.GABM_EUNSUPPORTED, [pop], _md(**kw), sets=sets)
    # parameter sets per graph: up to 64; without the lambda store only on symmetric weights
    _expect(capi.GABM_EUNSUPPORTED, [pop], _md(), sets=65)
    _expect(capi.GABM_EUNSUPPORTED, [synth.random_directed(64, 4.0, seed=3)],
            _md(lambda_policy=capi.GABM_RECOMPUTE), sets=4)


def test_null_handles_are_safe(lib):
    P = ctypes.c_void_p
    assert lib.gabm_forward(None, 5, None, None, None, None, None, None, 0) == capi.GABM_EINVAL
    assert lib.gabm_backward(None, None, None, None, None, 0) == capi.GABM_EINVAL
    assert lib.gabm_mse_loss(None, None, None, None, 0) == capi.GABM_EINVAL
    assert lib.gabm_get_state(None, None, 0) == capi.GABM_EINVAL
    assert lib.gabm_launch_count(None) == 0
    lib.gabm_destroy(None)
    assert lib.gabm_philox(0, None, None, 0, None) == capi.GABM_OK
    assert lib.gabm_philox(0, None, None, -1, None) == capi.GABM_EINVAL
    out = P()
    assert lib.gabm_create(None, 1, 1, None, None, ctypes.byref(out)) == capi.GABM_EINVAL
