"""Memory-wave planner (host code of the library, no GPU needed): every q point in exactly
one wave, each wave's projections + polarization workspace + outputs within the budget,
oversized q rejected."""
import numpy as np
import pytest

import synth_inputs as S

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gw():
    try:
        import paper_1003_0316_gb300 as g
    except ImportError as e:      # library not built here
        pytest.skip(str(e))
    return g


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_waves_cover_and_fit(gw, prec):
    wl = S.batched_uneven()
    Ks = [wl.K(i) for i in range(wl.nq)]
    nbs = list(wl.nb)
    budget = 200 * 2 ** 30
    waves = gw.plan_waves(Ks, nbs, wl.nw, prec, budget)
    assert sorted(q for w in waves for q in w) == list(range(wl.nq))
    elem = 16 if prec == "fp64" else 8
    for w in waves:
        ws = gw.polarization_workspace([Ks[q] for q in w], [nbs[q] for q in w], wl.nw, prec)
        need = ws + sum(Ks[q] * nbs[q] * elem + wl.nw * nbs[q] ** 2 * 16 for q in w)
        assert need <= budget
    # total projections of the workload exceed the budget, so there are several waves
    assert len(waves) >= sum(Ks[q] * nbs[q] * elem for q in range(wl.nq)) / budget
    assert gw.plan_waves(Ks, nbs, wl.nw, prec, budget) == waves


def test_waves_reject_oversized_q(gw):
    with pytest.raises(gw.GWError) as e:
        gw.plan_waves([10 ** 7], [4096], 16, "bf16x3", 2 ** 30)
    assert e.value.code == gw.GW_EINVAL
